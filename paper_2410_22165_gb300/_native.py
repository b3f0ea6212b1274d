"""ctypes binding of libeconojax.so (the C ABI of include/econojax.h).

Argument marshalling only: every computation runs in the CUDA library.  The
library is never replaced by a Python fallback; if it is missing or fails to
load, this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libeconojax.so")

EJ_MAX_A, EJ_MAX_R, EJ_MAX_P, EJ_MAX_NB = 1024, 16, 32, 4
EJ_MAX_ORDERS, EJ_MAX_ACTIONS, EJ_MAX_LEVELS = 16, 256, 512

STATUS = {0: "EJ_OK", 1: "EJ_ERR_ARG", 2: "EJ_ERR_CUDA", 3: "EJ_ERR_UNSUPPORTED"}

FIELDS = ["coin", "esc", "income", "uprev", "nord", "counts", "sc", "inv", "inve", "sg",
          "t", "gstep", "episode", "pop", "rates", "ugprev", "level_count", "book", "key"]


class EjParams(C.Structure):
    _fields_ = [
        ("E", C.c_int32), ("A", C.c_int32), ("R", C.c_int32), ("P", C.c_int32),
        ("nb", C.c_int32), ("T_ep", C.c_int32), ("T_tax", C.c_int32), ("expire", C.c_int32),
        ("max_orders", C.c_int32), ("Rk", C.c_int32), ("Rd", C.c_int32),
        ("allow_noop", C.c_int32), ("gov_enabled", C.c_int32), ("tax_levels", C.c_int32),
        ("start_coin", C.c_float), ("eta", C.c_float), ("omega", C.c_float),
        ("labor_gather", C.c_float), ("labor_craft", C.c_float), ("labor_trade", C.c_float),
        ("craft_coin", C.c_float), ("gather_rho", C.c_float), ("price_tick", C.c_float),
        ("price_ticks", C.c_int32 * EJ_MAX_P), ("thresholds", C.c_float * (EJ_MAX_NB - 1)),
        ("skill_gain", C.c_float), ("skill_max", C.c_float), ("skill_init", C.c_int32),
    ]


class EjSizes(C.Structure):
    _fields_ = [
        ("n_actions", C.c_int32), ("obs_dim", C.c_int32), ("gobs_dim", C.c_int32),
        ("mask_words", C.c_int32), ("levels", C.c_int32), ("book_cap", C.c_int32),
        ("threads", C.c_int32), ("smem_bytes", C.c_int32), ("state_bytes", C.c_uint64),
    ]


class EjRollout(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("obs", "gobs", "mask", "act", "gact", "logp", "glogp",
                                           "value", "gvalue", "rew", "grew", "done")]


class EjPpoParams(C.Structure):
    _fields_ = [("gamma", C.c_float), ("lam", C.c_float), ("clip", C.c_float), ("vf_coef", C.c_float),
                ("vclip", C.c_float), ("ent_coef", C.c_float), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("epochs", C.c_int32),
                ("minibatches", C.c_int32), ("seed", C.c_uint64)]


NET_POP, NET_GOV = 0, 1
NETS_SHARED, NETS_INDEPENDENT, NETS_CTDE = 0, 1, 2
FP32, BF16 = 0, 1


class EjError(RuntimeError):
    pass


_lib = None

# Exported symbols and their prototypes: (restype, argtypes).
_VP = C.c_void_p
_PROTOS = {
    "ej_params_default": (C.c_int, [C.POINTER(EjParams)]),
    "ej_sizes": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjSizes)]),
    "ej_state_field": (C.c_int, [C.POINTER(EjParams), C.c_int32, C.POINTER(C.c_uint64),
                                 C.POINTER(C.c_uint64), C.POINTER(C.c_int32)]),
    "env_reset": (C.c_int, [C.POINTER(EjParams), _VP, _VP, C.c_uint64, _VP, _VP, _VP, _VP]),
    "env_step": (C.c_int, [C.POINTER(EjParams), _VP, C.c_int32, _VP, _VP, _VP, _VP,
                           _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ej_step_host_workspace_bytes": (C.c_int, [C.POINTER(EjParams), C.c_int32, C.POINTER(C.c_uint64)]),
    "env_step_host": (C.c_int, [C.POINTER(EjParams), _VP, C.c_int32, C.c_int32, _VP, _VP, _VP, _VP, _VP, _VP,
                                _VP, _VP, _VP, _VP, _VP, C.c_uint64, _VP]),
    "ej_fill_draws": (C.c_int, [C.POINTER(EjParams), C.c_uint64, C.c_uint32, C.c_int32,
                                _VP, _VP, _VP, _VP, _VP, _VP]),
    "ej_net_floats": (C.c_int, [C.POINTER(EjParams), C.c_int32, C.c_int32, C.POINTER(C.c_uint64)]),
    "policy_forward": (C.c_int, [C.POINTER(EjParams), _VP, C.c_int32, C.c_int32, C.c_int32, _VP, _VP,
                                 _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "rollout": (C.c_int, [C.POINTER(EjParams), _VP, C.c_int32, C.c_int32, C.c_int32, _VP, _VP,
                          C.c_void_p, _VP]),
    "rollout_split": (C.c_int, [C.POINTER(EjParams), _VP, C.c_int32, C.c_int32, C.c_int32, _VP, _VP,
                                C.c_void_p, C.c_int32, _VP]),
    "ej_ppo_params_default": (C.c_int, [C.POINTER(EjPpoParams)]),
    "ej_ppo_workspace_bytes": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32,
                                         C.POINTER(C.c_uint64)]),
    "ej_ppo_workspace_offsets": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32,
                                           C.POINTER(C.c_uint64)]),
    "ppo_advantages": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_void_p, _VP, _VP]),
    "ppo_minibatch_grad": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32,
                                     C.c_int32, C.c_int32, _VP, C.c_void_p, _VP, C.c_uint32, C.c_int32,
                                     _VP, _VP, _VP]),
    "policy_segmented": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "policy_forward_segments": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                          C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          _VP]),
    "ppo_minibatch_moments": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32,
                                        C.c_void_p, _VP, C.c_uint32, C.c_int32, _VP, _VP]),
    "ppo_minibatch_grad_global": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32,
                                            C.c_int32, C.c_int32, _VP, C.c_void_p, _VP, C.c_uint32, C.c_int32,
                                            _VP, _VP, _VP, _VP]),
    "adam_step": (C.c_int, [C.c_uint64, _VP, _VP, _VP, _VP, C.c_int32, C.c_float, C.c_float, C.c_float,
                            C.c_float, _VP]),
    "ppo_update": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32, C.c_int32,
                             _VP, _VP, _VP, _VP, _VP, _VP, C.c_int32, C.c_uint32, C.c_void_p, _VP, _VP, _VP]),
    "ppo_minibatch_grad_static": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32,
                                            C.c_int32, C.c_int32, _VP, C.c_void_p, C.c_uint32, C.c_int32,
                                            _VP, _VP, _VP]),
    "policy_forward_agents": (C.c_int, [C.POINTER(EjParams), _VP, C.c_int32, C.c_int32, C.c_int32, _VP, _VP,
                                        _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "rollout_agents": (C.c_int, [C.POINTER(EjParams), _VP, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _VP, _VP,
                                 C.c_void_p, _VP]),
    "ej_ppo_workspace_bytes_agents": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32,
                                                C.c_int32, C.POINTER(C.c_uint64)]),
    "ppo_minibatch_grad_agents": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32,
                                            C.c_int32, C.c_int32, _VP, C.c_void_p, _VP, C.c_uint32, C.c_int32,
                                            _VP, _VP, _VP]),
    "ppo_update_agents": (C.c_int, [C.POINTER(EjParams), C.POINTER(EjPpoParams), C.c_int32, C.c_int32, C.c_int32,
                                    C.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, C.c_int32, C.c_uint32, C.c_void_p,
                                    _VP, _VP, _VP]),
    "ej_device_status": (C.c_int, [C.POINTER(C.c_int32), C.c_int32]),
    "ej_last_error": (C.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Load the library (building nothing).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise EjError(
            f"{path} is missing: build it with `python -m paper_2410_22165_gb300.build` "
            "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_PROTOS)


def check(status: int, what: str = ""):
    if status != 0:
        msg = load().ej_last_error().decode(errors="replace")
        raise EjError(f"{what}: {STATUS.get(status, status)}: {msg}")


def make_params(**kw) -> EjParams:
    p = EjParams()
    check(load().ej_params_default(C.byref(p)), "ej_params_default")
    for k, v in kw.items():
        if k == "price_ticks":
            vals = [int(x) for x in v]
            p.price_ticks = (C.c_int32 * EJ_MAX_P)(*(vals + [0] * (EJ_MAX_P - len(vals))))
        elif k == "thresholds":
            vals = [float(x) for x in v]
            p.thresholds = (C.c_float * (EJ_MAX_NB - 1))(*(vals + [0.0] * (EJ_MAX_NB - 1 - len(vals))))
        else:
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
    return p


def params_dict(p: EjParams) -> dict:
    d = {}
    for name, _ in EjParams._fields_:
        v = getattr(p, name)
        if name == "price_ticks":
            v = [int(x) for x in v[: p.P]]
        elif name == "thresholds":
            v = [float(x) for x in v[: p.nb - 1]]
        d[name] = v
    return d


def sizes(p: EjParams) -> EjSizes:
    s = EjSizes()
    check(load().ej_sizes(C.byref(p), C.byref(s)), "ej_sizes")
    return s


def state_field(p: EjParams, field: str):
    off, cnt, esz = C.c_uint64(), C.c_uint64(), C.c_int32()
    check(load().ej_state_field(C.byref(p), FIELDS.index(field), C.byref(off), C.byref(cnt),
                                C.byref(esz)), "ej_state_field")
    return off.value, cnt.value, esz.value
