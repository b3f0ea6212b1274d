"""ctypes wrapper of the C environment oracle (test infrastructure only).

The rules themselves live in ``oracle/ej_oracle.c``; this file only moves
numpy arrays in and out.  Parameters are given as a plain dict (see
``default_params``) so that the oracle shares no struct with the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

MAX_R, MAX_P, MAX_NB = 16, 32, 8


class _Params(C.Structure):
    _fields_ = [
        ("R", C.c_int), ("P", C.c_int), ("nb", C.c_int), ("T_ep", C.c_int),
        ("T_tax", C.c_int), ("expire", C.c_int), ("max_orders", C.c_int),
        ("Rk", C.c_int), ("Rd", C.c_int), ("allow_noop", C.c_int),
        ("gov_enabled", C.c_int), ("tax_levels", C.c_int),
        ("start_coin", C.c_double), ("eta", C.c_double), ("omega", C.c_double),
        ("labor_gather", C.c_double), ("labor_craft", C.c_double),
        ("labor_trade", C.c_double), ("craft_coin", C.c_double),
        ("gather_rho", C.c_double), ("price_tick", C.c_double),
        ("price_ticks", C.c_int * MAX_P), ("thresholds", C.c_double * (MAX_NB - 1)),
        ("skill_gain", C.c_double), ("skill_max", C.c_double),
    ]


class _Info(C.Structure):
    _fields_ = [
        ("t", C.c_int), ("episode", C.c_int), ("n_book", C.c_int),
        ("rates32", C.c_float * MAX_NB), ("rates64", C.c_double * MAX_NB),
        ("ug_prev", C.c_double),
    ]


def default_params(**over):
    """Table 2 of the paper (environment half), plus the readings for what it
    does not print: craft coin 10 per unit of skill, brackets [50, 100] (the
    worked example of Section 3), 21 rate levels."""
    p = dict(
        R=2, P=5, nb=3, T_ep=1000, T_tax=100, expire=30, max_orders=15, Rk=2, Rd=2,
        allow_noop=1, gov_enabled=1, tax_levels=21, start_coin=15.0, eta=0.27,
        omega=1.0, labor_gather=1.0, labor_craft=1.0, labor_trade=0.05,
        craft_coin=10.0, gather_rho=1.1, price_tick=2.0, price_ticks=[1, 2, 3, 4, 5],
        thresholds=[50.0, 100.0], skill_gain=0.0, skill_max=5.0, skill_init=0,
    )
    p.update(over)
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        P, D, F, I, U = C.POINTER, C.c_double, C.c_float, C.c_int32, C.c_uint32
        L.orc_env_new.restype = C.c_void_p
        L.orc_env_new.argtypes = [P(_Params), C.c_int]
        L.orc_env_free.argtypes = [C.c_void_p]
        L.orc_env_reset.argtypes = [C.c_void_p, P(F), P(F)]
        L.orc_env_step.argtypes = [C.c_void_p, P(I), P(I), P(F), P(U), P(F), P(F),
                                   P(D), P(D), P(I), P(D), P(D), P(U)]
        L.orc_env_run.argtypes = [C.c_void_p, C.c_int, P(I), P(I), P(F), P(U), P(F), P(F),
                                  P(D), P(D), P(I), P(D), P(D), P(U)]
        L.orc_env_observe.argtypes = [C.c_void_p, P(D), P(D), P(U)]
        L.orc_env_get_info.argtypes = [C.c_void_p, P(_Info)]
        L.orc_env_get_agents.argtypes = [C.c_void_p, P(F), P(D), P(F), P(D), P(I), P(I),
                                         P(I), P(I), P(I), P(D)]
        L.orc_env_get_book.restype = C.c_int
        L.orc_env_get_book.argtypes = [C.c_void_p, P(I), C.c_int]
        L.orc_env_get_trades.argtypes = [C.c_void_p, P(I), P(C.c_int64)]
        for name in ("orc_num_actions", "orc_obs_dim", "orc_gobs_dim", "orc_mask_words"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [P(_Params)]
        L.orc_gini.restype = D
        L.orc_gini.argtypes = [P(D), C.c_int]
        L.orc_isoelastic.restype = D
        L.orc_isoelastic.argtypes = [D, D, D]
        L.orc_bracket_tax.restype = D
        L.orc_bracket_tax.argtypes = [D, P(D), P(D), C.c_int]
        _lib = L
    return _lib


def _cparams(p: dict) -> _Params:
    s = _Params()
    for name, _ in _Params._fields_:
        if name == "price_ticks":
            arr = (C.c_int * MAX_P)(*([int(x) for x in p[name]] + [0] * (MAX_P - len(p[name]))))
            s.price_ticks = arr
        elif name == "thresholds":
            vals = [float(x) for x in p[name]]
            s.thresholds = (C.c_double * (MAX_NB - 1))(*(vals + [0.0] * (MAX_NB - 1 - len(vals))))
        else:
            setattr(s, name, p[name])
    return s


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def num_actions(p):
    return lib().orc_num_actions(C.byref(_cparams(p)))


def obs_dim(p):
    return lib().orc_obs_dim(C.byref(_cparams(p)))


def gobs_dim(p):
    return lib().orc_gobs_dim(C.byref(_cparams(p)))


def mask_words(p):
    return lib().orc_mask_words(C.byref(_cparams(p)))


def gini(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_gini(_ptr(x, C.c_double), len(x))


def isoelastic(coin, labor, eta):
    return lib().orc_isoelastic(coin, labor, eta)


def bracket_tax(income, rates, thresholds):
    r = np.ascontiguousarray(rates, dtype=np.float64)
    t = np.ascontiguousarray(list(thresholds) + [0.0], dtype=np.float64)
    return lib().orc_bracket_tax(float(income), _ptr(r, C.c_double), _ptr(t, C.c_double), len(r))


class OracleEnv:
    """One environment of A population agents plus the government."""

    def __init__(self, params: dict, A: int):
        self.p = dict(params)
        self.A = int(A)
        self._cp = _cparams(self.p)
        self.h = lib().orc_env_new(C.byref(self._cp), self.A)
        self.R = self.p["R"]
        self.nb = self.p["nb"]
        self.D = obs_dim(self.p)
        self.G = gobs_dim(self.p)
        self.W = mask_words(self.p)
        self.nA = num_actions(self.p)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_env_free(h)
            self.h = None

    def reset(self, sg, sc):
        sg = np.ascontiguousarray(sg, dtype=np.float32).reshape(self.A, self.R)
        sc = np.ascontiguousarray(sc, dtype=np.float32).reshape(self.A)
        lib().orc_env_reset(self.h, _ptr(sg, C.c_float), _ptr(sc, C.c_float))

    def observe(self):
        obs = np.zeros((self.A, self.D))
        gobs = np.zeros(self.G)
        mask = np.zeros((self.A, self.W), dtype=np.uint32)
        lib().orc_env_observe(self.h, _ptr(obs, C.c_double), _ptr(gobs, C.c_double),
                              _ptr(mask, C.c_uint32))
        return obs, gobs, mask

    def step(self, act, gov_act, gather_u, tb, next_sg=None, next_sc=None):
        A = self.A
        act = np.ascontiguousarray(act, dtype=np.int32).reshape(A)
        gov = np.ascontiguousarray(gov_act, dtype=np.int32).reshape(self.nb)
        gu = np.ascontiguousarray(gather_u, dtype=np.float32).reshape(A)
        tb = np.ascontiguousarray(tb, dtype=np.uint32).reshape(A)
        nsg = None if next_sg is None else np.ascontiguousarray(next_sg, dtype=np.float32)
        nsc = None if next_sc is None else np.ascontiguousarray(next_sc, dtype=np.float32)
        rew = np.zeros(A)
        grew = np.zeros(1)
        done = np.zeros(1, dtype=np.int32)
        obs = np.zeros((A, self.D))
        gobs = np.zeros(self.G)
        mask = np.zeros((A, self.W), dtype=np.uint32)
        lib().orc_env_step(self.h, _ptr(act, C.c_int32), _ptr(gov, C.c_int32),
                           _ptr(gu, C.c_float), _ptr(tb, C.c_uint32),
                           _ptr(nsg, C.c_float), _ptr(nsc, C.c_float),
                           _ptr(rew, C.c_double), _ptr(grew, C.c_double),
                           _ptr(done, C.c_int32), _ptr(obs, C.c_double),
                           _ptr(gobs, C.c_double), _ptr(mask, C.c_uint32))
        return dict(rew=rew, grew=float(grew[0]), done=int(done[0]), obs=obs, gobs=gobs, mask=mask)

    def run(self, act, gov_act, gather_u, tb, later_sg=None, later_sc=None, outputs=True):
        """Run n steps; inputs are [n, A] / [n, nb]; later skills [k, A, R] / [k, A]."""
        act = np.ascontiguousarray(act, dtype=np.int32)
        n = act.shape[0]
        A = self.A
        gov = np.ascontiguousarray(gov_act, dtype=np.int32)
        gu = np.ascontiguousarray(gather_u, dtype=np.float32)
        tb = np.ascontiguousarray(tb, dtype=np.uint32)
        lsg = None if later_sg is None else np.ascontiguousarray(later_sg, dtype=np.float32)
        lsc = None if later_sc is None else np.ascontiguousarray(later_sc, dtype=np.float32)
        out = {}
        if outputs:
            out = dict(rew=np.zeros((n, A)), grew=np.zeros(n), done=np.zeros(n, dtype=np.int32),
                       obs=np.zeros((n, A, self.D)), gobs=np.zeros((n, self.G)),
                       mask=np.zeros((n, A, self.W), dtype=np.uint32))
        g = out.get
        lib().orc_env_run(self.h, n, _ptr(act, C.c_int32), _ptr(gov, C.c_int32),
                          _ptr(gu, C.c_float), _ptr(tb, C.c_uint32),
                          _ptr(lsg, C.c_float), _ptr(lsc, C.c_float),
                          _ptr(g("rew"), C.c_double), _ptr(g("grew"), C.c_double),
                          _ptr(g("done"), C.c_int32), _ptr(g("obs"), C.c_double),
                          _ptr(g("gobs"), C.c_double), _ptr(g("mask"), C.c_uint32))
        return out

    def info(self):
        s = _Info()
        lib().orc_env_get_info(self.h, C.byref(s))
        return dict(t=s.t, episode=s.episode, n_book=s.n_book,
                    rates32=np.array(s.rates32[: self.nb], dtype=np.float32),
                    rates64=np.array(s.rates64[: self.nb]), ug_prev=s.ug_prev)

    def agents(self):
        A, R = self.A, self.R
        f = dict(coin32=np.zeros(A, np.float32), coin64=np.zeros(A),
                 income32=np.zeros(A, np.float32), income64=np.zeros(A),
                 esc_ticks=np.zeros(A, np.int32), inv=np.zeros((A, R), np.int32),
                 inv_esc=np.zeros((A, R), np.int32), n_orders=np.zeros(A, np.int32),
                 counts=np.zeros((A, 3), np.int32), u_prev=np.zeros(A))
        lib().orc_env_get_agents(
            self.h, _ptr(f["coin32"], C.c_float), _ptr(f["coin64"], C.c_double),
            _ptr(f["income32"], C.c_float), _ptr(f["income64"], C.c_double),
            _ptr(f["esc_ticks"], C.c_int32), _ptr(f["inv"], C.c_int32),
            _ptr(f["inv_esc"], C.c_int32), _ptr(f["n_orders"], C.c_int32),
            _ptr(f["counts"], C.c_int32), _ptr(f["u_prev"], C.c_double))
        return f

    def book(self):
        cap = self.A * (self.p["max_orders"] + 1) + 16
        rows = np.zeros((cap, 6), dtype=np.int32)
        n = lib().orc_env_get_book(self.h, _ptr(rows, C.c_int32), cap)
        b = rows[:n].copy()
        return b

    def trades(self):
        n = np.zeros(self.R, np.int32)
        v = np.zeros(self.R, np.int64)
        lib().orc_env_get_trades(self.h, _ptr(n, C.c_int32), _ptr(v, C.c_int64))
        return n, v
