"""Binding of the serving loop (continuous batching of evaluation requests).

The scheduling, admission and completion tracking run in libpeps.so
(serve.cu); this module marshals arguments and allocates each request's
output tensors with torch (the caller's memory).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import peps as _p


def _lib():
    L = _p.lib()
    if not getattr(L, "_server_sigs", False):
        P, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.peps_server_create.argtypes = [i, d, ctypes.POINTER(P)]
        L.peps_server_destroy.argtypes = [P]
        L.peps_server_submit.argtypes = [P, P, P, i, P, P, P, P, P, ctypes.POINTER(ctypes.c_longlong)]
        L.peps_server_poll.argtypes = [P, i, P, P, i, ctypes.POINTER(i)]
        L.peps_server_stats.argtypes = [P, P]
        u64 = ctypes.c_uint64
        L.peps_server_submit_chain.argtypes = [P, P, P, i, i, u64, u64, u64, P, P, P, P, P,
                                               ctypes.POINTER(ctypes.c_longlong)]
        L.peps_server_set_packing.argtypes = [P, i, i]
        L.peps_server_set_policy.argtypes = [P, i]
        for f in ("peps_server_create", "peps_server_destroy", "peps_server_submit", "peps_server_poll",
                  "peps_server_stats", "peps_server_submit_chain", "peps_server_set_packing",
                  "peps_server_set_policy"):
            getattr(L, f).restype = ctypes.c_int
        L._server_sigs = True
    return L


class Server:
    """Requests of any number of models run on ``nlanes`` CUDA streams; a
    request is admitted when a lane is free and its HBM footprint fits under
    ``hbm_budget_gb``."""

    def __init__(self, nlanes=4, hbm_budget_gb=32.0):
        import torch
        self.torch = torch
        h = ctypes.c_void_p()
        _p.check(_lib().peps_server_create(int(nlanes), float(hbm_budget_gb), ctypes.byref(h)))
        self.h = h
        self.outputs = {}

    def submit(self, model, S, logabs=True, eloc=True, O=False):
        """Queues an evaluation of configurations S (CUDA int64 [n, words]) of
        ``model`` (a PEPS); returns the request id.  Outputs are fetched with
        :meth:`result` once :meth:`poll` has returned the id."""
        torch = self.torch
        S = model._S(S)
        n = S.shape[0]
        dev = S.device
        out = dict(
            S=S,
            logabs=torch.empty(n, dtype=torch.float64, device=dev) if logabs else None,
            sign=torch.empty(n, dtype=torch.int8, device=dev) if logabs else None,
            eloc=torch.empty(n, dtype=torch.float64, device=dev) if eloc else None,
            O=torch.empty((n, model.N, model.D ** 4), dtype=model.real, device=dev) if O else None,
            status=torch.empty(n, dtype=torch.int32, device=dev),
        )
        # inputs and output buffers must be ready before the lanes' streams use them
        torch.cuda.current_stream().synchronize()
        rid = ctypes.c_longlong()
        _p.check(_lib().peps_server_submit(self.h, model.h, _p._ptr(S), n, _p._ptr(out["logabs"]),
                                           _p._ptr(out["sign"]), _p._ptr(out["eloc"]), _p._ptr(out["O"]),
                                           _p._ptr(out["status"]), ctypes.byref(rid)))
        self.outputs[rid.value] = out
        return rid.value

    def submit_chain(self, model, S, nsweeps, seed, chain0=0, sweep0=0, logabs=True, eloc=True, O=False):
        """Queues a chain request: S (CUDA int64 [n, words], the chains' state,
        kept on the device by the caller) takes ``nsweeps`` Metropolis sweeps
        in place, then is evaluated.  Returns the request id."""
        torch = self.torch
        assert isinstance(S, torch.Tensor) and S.is_cuda and S.dtype == torch.int64 and S.is_contiguous()
        n = S.shape[0]
        dev = S.device
        out = dict(
            S=S,
            logabs=torch.empty(n, dtype=torch.float64, device=dev) if logabs else None,
            sign=torch.empty(n, dtype=torch.int8, device=dev) if logabs else None,
            eloc=torch.empty(n, dtype=torch.float64, device=dev) if eloc else None,
            O=torch.empty((n, model.N, model.D ** 4), dtype=model.real, device=dev) if O else None,
            status=torch.empty(n, dtype=torch.int32, device=dev),
        )
        torch.cuda.current_stream().synchronize()
        rid = ctypes.c_longlong()
        _p.check(_lib().peps_server_submit_chain(self.h, model.h, _p._ptr(S), n, int(nsweeps), int(seed),
                                                 int(chain0), int(sweep0), _p._ptr(out["logabs"]),
                                                 _p._ptr(out["sign"]), _p._ptr(out["eloc"]), _p._ptr(out["O"]),
                                                 _p._ptr(out["status"]), ctypes.byref(rid)))
        self.outputs[rid.value] = out
        return rid.value

    def set_packing(self, max_configs, max_requests=8):
        """Pack co-admitted requests of at most ``max_configs`` configurations
        (up to ``max_requests`` of distinct models) into one launch; 0 turns it off."""
        _p.check(_lib().peps_server_set_packing(self.h, int(max_configs), int(max_requests)))

    def set_policy(self, policy):
        """Admission order: "fifo" (first come first served, the default) or
        "expected" (smallest expected run time less time waited first)."""
        code = {"fifo": 0, "expected": 1}[policy]
        _p.check(_lib().peps_server_set_policy(self.h, code))

    def poll(self, wait=False, max_items=256):
        """[(request id, latency ms)] of requests finished since the last poll."""
        ids = np.zeros(max_items, dtype=np.int64)
        lat = np.zeros(max_items, dtype=np.float64)
        nd = ctypes.c_int()
        _p.check(_lib().peps_server_poll(self.h, 1 if wait else 0, _p._ptr(ids), _p._ptr(lat), int(max_items),
                                         ctypes.byref(nd)))
        done = [(int(ids[k]), float(lat[k])) for k in range(nd.value)]
        for rid, ms in done:
            if ms < 0 and rid in self.outputs:
                self.outputs[rid]["failed"] = _lib().peps_last_error().decode()
        return done

    def result(self, rid):
        """The outputs of a finished request; raises if it could not be launched."""
        out = self.outputs.pop(rid)
        if "failed" in out:
            raise _p.PepsError(2, f"request {rid} was not run: {out['failed']}")
        return out

    def drain(self):
        done = []
        while True:
            got = self.poll(wait=True)
            if not got:
                return done
            done += got

    def stats(self):
        st = np.zeros(8, dtype=np.float64)
        _p.check(_lib().peps_server_stats(self.h, _p._ptr(st)))
        keys = ["submitted", "completed", "queued", "running", "p50_ms", "p99_ms", "hbm_in_use_gb", "hbm_peak_gb"]
        return dict(zip(keys, st.tolist()))

    def close(self):
        if getattr(self, "h", None):
            _lib().peps_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_arrivals(rate_hz, duration_s, seed):
    """Arrival times of a Poisson process (exponential gaps), seeded."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return out
        out.append(t)
