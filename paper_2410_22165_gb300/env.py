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
                  copy_streams: int = 1):
        """env_step over n_steps with inputs and outputs in (pinned) host memory.

        host_in: act [n,E,A], gov_act [n,E,nb], gather_u [n,E,A], tb [n,E,A];
        host_out: any of rew, grew, done, obs, gobs, mask (shapes of step's outputs).
        The steps run in chunks through two sets of device buffers, so that
        chunk k's outputs copy out while chunk k+1 runs and chunk k+2's inputs
        copy in; each chunk's output copies are split over `copy_streams`
        streams (several copy engines on the host link).  With sync, returns
        when host_out is filled; otherwise the caller synchronises the device."""
        dev = self.device
        keys_in = ("act", "gov_act", "gather_u", "tb")
        chunk = max(1, min(chunk, n_steps))
        st = getattr(self, "_host_io", None)
        ncs = max(1, int(copy_streams))
        if (st is None or st["chunk"] != chunk or set(st["out"][0]) != set(host_out)
                or len(st["outs"]) != ncs):
            bufs_in = [{k: torch.empty((chunk,) + tuple(host_in[k].shape[1:]), dtype=host_in[k].dtype, device=dev)
                        for k in keys_in} for _ in range(2)]
            names = set(host_out)
            bufs_out = [self.alloc_outputs(chunk, obs="obs" in names, gobs="gobs" in names, mask="mask" in names,
                                           rew=bool({"rew", "grew"} & names), done="done" in names)
                        for _ in range(2)]
            st = dict(chunk=chunk, inp=bufs_in, out=bufs_out,
                      streams=[torch.cuda.Stream(device=dev) for _ in range(2)],
                      outs=[torch.cuda.Stream(device=dev) for _ in range(ncs)],
                      ev=[[torch.cuda.Event() for _ in range(2)] for _ in range(2)],
                      ev_out=[[torch.cuda.Event() for _ in range(2)] for _ in range(ncs)])
            self._host_io = st
        s_in, s_comp = st["streams"]
        ev_in, ev_comp = st["ev"]
        main = torch.cuda.current_stream(dev)
        for s in (s_in, s_comp, *st["outs"]):
            s.wait_stream(main)
        n_chunks = (n_steps + chunk - 1) // chunk
        for c in range(n_chunks):
            b, lo = c % 2, c * chunk
            n = min(chunk, n_steps - lo)
            bi, bo = st["inp"][b], st["out"][b]
            with torch.cuda.stream(s_in):
                if c >= 2:
                    s_in.wait_event(ev_comp[b])          # chunk c-2 has finished reading these inputs
                for k in keys_in:
                    bi[k][:n].copy_(host_in[k][lo:lo + n], non_blocking=True)
                ev_in[b].record(s_in)
            with torch.cuda.stream(s_comp):
                s_comp.wait_event(ev_in[b])
                if c >= 2:
                    for ev_out in st["ev_out"]:
                        s_comp.wait_event(ev_out[b])     # chunk c-2's outputs have left these buffers
                out = {k: v[:n] for k, v in bo.items()}
                self.step(n, act=bi["act"][:n], gov_act=bi["gov_act"][:n], gather_u=bi["gather_u"][:n],
                          tb=bi["tb"][:n], out=out, stream=s_comp)
                ev_comp[b].record(s_comp)
            # output copies: each tensor's steps split evenly over the copy streams
            for j, so in enumerate(st["outs"]):
                with torch.cuda.stream(so):
                    so.wait_event(ev_comp[b])
                    a0, a1 = (n * j) // ncs, (n * (j + 1)) // ncs
                    if a1 > a0:
                        for k, v in host_out.items():
                            v[lo + a0:lo + a1].copy_(bo[k][a0:a1], non_blocking=True)
                    st["ev_out"][j][b].record(so)
        for s in (s_in, s_comp, *st["outs"]):
            main.wait_stream(s)
        if sync:
            torch.cuda.synchronize(dev)
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
