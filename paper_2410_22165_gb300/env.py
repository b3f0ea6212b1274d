"""Vectorised EconoJax environments on the GPU (torch tensors in, torch tensors out).

Thin wrapper of the C ABI: it allocates the caller-owned buffers as torch
tensors and passes their device pointers and the current CUDA stream to
``env_reset`` / ``env_step``.  No step of the environment runs in Python.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native as N

_DT = {4: torch.int32}
_FIELD_DTYPE = {
    "coin": torch.float32, "esc": torch.int32, "income": torch.float32, "uprev": torch.float32,
    "nord": torch.int32, "counts": torch.int32, "sc": torch.float32, "inv": torch.int32,
    "inve": torch.int32, "sg": torch.float32, "t": torch.int32, "gstep": torch.int32,
    "episode": torch.int32, "pop": torch.int32, "rates": torch.float32, "ugprev": torch.float32,
    "level_count": torch.int32, "book": torch.int32, "key": torch.int32,
}


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _host_ptr(t):
    if t.is_cuda:
        raise ValueError("expected a host tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class VecEnv:
    """E environments of A agents each (populations may be smaller per env)."""

    def __init__(self, E: int, A: int = 100, device="cuda", **params):
        self.p = N.make_params(E=E, A=A, **params)
        self.sizes = N.sizes(self.p)
        self.device = torch.device(device)
        self.E, self.A = E, A
        self.nA = self.sizes.n_actions
        self.D = self.sizes.obs_dim
        self.G = self.sizes.gobs_dim
        self.W = self.sizes.mask_words
        # 256-byte aligned (the caching allocator aligns to at least 512 bytes)
        self.state = torch.zeros(int(self.sizes.state_bytes), dtype=torch.uint8, device=self.device)
        assert self.state.data_ptr() % 256 == 0

    @property
    def params(self) -> dict:
        return N.params_dict(self.p)

    def alloc_outputs(self, n: int, obs=True, gobs=True, mask=True, rew=True, done=True):
        E, A, dev = self.E, self.A, self.device
        out = {}
        if rew:
            out["rew"] = torch.empty((n, E, A), dtype=torch.float32, device=dev)
            out["grew"] = torch.empty((n, E), dtype=torch.float32, device=dev)
        if done:
            out["done"] = torch.empty((n, E), dtype=torch.uint8, device=dev)
        if obs:
            out["obs"] = torch.empty((n, E, A, self.D), dtype=torch.float32, device=dev)
        if gobs:
            out["gobs"] = torch.empty((n, E, self.G), dtype=torch.float32, device=dev)
        if mask:
            out["mask"] = torch.empty((n, E, A, self.W), dtype=torch.int32, device=dev)
        return out

    def reset(self, seed: int = 0, pop_sizes: torch.Tensor | None = None, out=None, stream=None):
        """env_reset: returns {obs [E,A,D], gobs [E,G], mask [E,A,W]}."""
        if out is None:
            o = self.alloc_outputs(1, rew=False, done=False)
            out = {k: v[0] for k, v in o.items()}
        if pop_sizes is not None:
            pop_sizes = pop_sizes.to(device=self.device, dtype=torch.int32).contiguous()
        N.check(N.load().env_reset(C.byref(self.p), _ptr(self.state), _ptr(pop_sizes),
                                   C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _ptr(out.get("obs")),
                                   _ptr(out.get("gobs")), _ptr(out.get("mask")), _stream(stream)),
                "env_reset")
        return out

    def step(self, n_steps: int = 1, act=None, gov_act=None, gather_u=None, tb=None, out=None,
             stream=None):
        """env_step over n_steps.  Inputs [n,E,A] / [n,E,nb] or None (in-kernel draws).
        Returns the output dict ([n, ...] tensors)."""
        if out is None:
            out = self.alloc_outputs(n_steps)
        N.check(N.load().env_step(
            C.byref(self.p), _ptr(self.state), int(n_steps), _ptr(act), _ptr(gov_act),
            _ptr(gather_u), _ptr(tb), _ptr(out.get("rew")), _ptr(out.get("grew")),
            _ptr(out.get("done")), _ptr(out.get("obs")), _ptr(out.get("gobs")),
            _ptr(out.get("mask")), _stream(stream)), "env_step")
        return out

    def step_host(self, n_steps: int, host_in: dict, host_out: dict, chunk: int = 100, sync: bool = True,
                  stream=None):
        """env_step_host: env_step over n_steps with inputs and outputs in
        (pinned) host memory.  host_in: act [n,E,A], gov_act [n,E,nb],
        gather_u [n,E,A], tb [n,E,A] (any may be missing: in-kernel draws as
        in step); host_out: any of rew, grew, done, obs, gobs, mask (shapes of
        step's outputs).  The library runs the steps in chunks, copying chunk
        k+1's inputs in and chunk k-1's outputs out while chunk k runs; the
        staging workspace is allocated here (caller-owned).  With sync,
        returns when host_out is filled; otherwise the caller synchronises
        the stream."""
        chunk = max(1, min(chunk, n_steps))
        ws = getattr(self, "_host_ws", None)
        if ws is None or ws[0] != chunk:
            nbytes = C.c_uint64()
            N.check(N.load().ej_step_host_workspace_bytes(C.byref(self.p), chunk, C.byref(nbytes)),
                    "ej_step_host_workspace_bytes")
            ws = (chunk, torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device))
            self._host_ws = ws
        hp = lambda d, k: None if d.get(k) is None else C.c_void_p(_host_ptr(d[k]))
        N.check(N.load().env_step_host(
            C.byref(self.p), _ptr(self.state), int(n_steps), int(chunk), hp(host_in, "act"),
            hp(host_in, "gov_act"), hp(host_in, "gather_u"), hp(host_in, "tb"), hp(host_out, "rew"),
            hp(host_out, "grew"), hp(host_out, "done"), hp(host_out, "obs"), hp(host_out, "gobs"),
            hp(host_out, "mask"), _ptr(ws[1]), ws[1].numel(), _stream(stream)), "env_step_host")
        if sync:
            (torch.cuda.current_stream(self.device) if stream is None else stream).synchronize()
        return host_out

    def fill_draws(self, seed: int, g0: int, n_steps: int, stream=None, policy=False):
        """The draws env_step makes itself, as tensors (same counter mapping)."""
        E, A, dev = self.E, self.A, self.device
        d = dict(act=torch.empty((n_steps, E, A), dtype=torch.int32, device=dev),
                 gather_u=torch.empty((n_steps, E, A), dtype=torch.float32, device=dev),
                 tb=torch.empty((n_steps, E, A), dtype=torch.int32, device=dev),
                 gov_act=torch.empty((n_steps, E, self.p.nb), dtype=torch.int32, device=dev))
        if policy:
            d["policy_u"] = torch.empty((n_steps, E, A), dtype=torch.float32, device=dev)
        N.check(N.load().ej_fill_draws(C.byref(self.p), C.c_uint64(seed), C.c_uint32(g0),
                                       int(n_steps), _ptr(d["act"]), _ptr(d["gather_u"]),
                                       _ptr(d["tb"]), _ptr(d.get("policy_u")), _ptr(d["gov_act"]),
                                       _stream(stream)), "ej_fill_draws")
        return d

    def field(self, name: str) -> torch.Tensor:
        """View of one state field (shapes as documented in econojax.h)."""
        off, cnt, esz = N.state_field(self.p, name)
        dt = _FIELD_DTYPE[name]
        v = self.state[off: off + cnt * esz].view(dt)
        E, A_s, R = self.E, (self.A + 3) & ~3, self.p.R
        shapes = {"counts": (E, 3, A_s), "inv": (E, R, A_s), "inve": (E, R, A_s), "sg": (E, R, A_s),
                  "rates": (E, N.EJ_MAX_NB), "level_count": (E, self.sizes.levels),
                  "book": (E, self.sizes.book_cap)}
        if name in shapes:
            return v.view(shapes[name])
        if name in ("t", "gstep", "episode", "pop", "ugprev", "key"):
            return v
        return v.view(E, A_s)
