"""Thin Python binding of libpeps.so (argument marshalling only).

Every step of the computation runs in the CUDA library; this module only
converts arguments.  There is no fallback: if libpeps.so is missing or no
GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpeps.so")

PEPS_OK, PEPS_EINVAL, PEPS_ENOMEM, PEPS_ECUDA, PEPS_ETIMEOUT, PEPS_ENUMERIC = range(6)
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed_tf32": 2, "mixed_bf16": 3}


class PepsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


STATUS_NAMES = {0: "PEPS_OK", 1: "PEPS_EINVAL", 2: "PEPS_ENOMEM", 3: "PEPS_ECUDA", 4: "PEPS_ETIMEOUT",
                5: "PEPS_ENUMERIC"}


class Params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("d", ctypes.c_int), ("D", ctypes.c_int),
                ("Dc", ctypes.c_int), ("J1", ctypes.c_double), ("J2", ctypes.c_double), ("prec", ctypes.c_int),
                ("workspace_gb", ctypes.c_double)]


_lib = None
P = ctypes.c_void_p


def lib():
    """Loads libpeps.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libpeps.so not found at {LIB_PATH}: run paper_1611_09467_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    i, d = ctypes.c_int, ctypes.c_double
    sigs = {
        "peps_create": [ctypes.POINTER(Params), P, P, ctypes.POINTER(P)],
        "peps_destroy": [P],
        "peps_set_tensors": [P, P],
        "peps_go_step": [P, P, d, ctypes.c_uint64, ctypes.c_uint64, P],
        "peps_amplitudes": [P, P, i, P, P, P],
        "peps_local_energy": [P, P, i, P, P],
        "peps_log_derivatives": [P, P, i, P],
        "peps_evaluate": [P, P, i, P, P, P, P, P],
        "peps_gradient": [P, P, i, ctypes.POINTER(d), P, P, P, P, P, P, ctypes.POINTER(i)],
        "peps_mc_sweep": [P, P, i, i, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, P],
        "peps_synchronize": [P],
        "peps_profile_enable": [P, i],
        "peps_profile_read": [P, P, P, i],
        "peps_debug_host_op": [i, i, i, P, P, P, P, P, P],
        "peps_amplitudes_static": [ctypes.POINTER(Params), P, P, i, P, P, P, P],
        "peps_debug_host_zip": [i, i, i, P, P, P, P, P],
    }
    for name, argt in sigs.items():
        f = getattr(L, name)
        f.argtypes = argt
        f.restype = ctypes.c_int
    L.peps_status_str.argtypes = [ctypes.c_int]
    L.peps_status_str.restype = ctypes.c_char_p
    L.peps_last_error.argtypes = []
    L.peps_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def exported_symbols():
    """Names declared in include/peps.h that the loaded library exports."""
    L = lib()
    names = ["peps_create", "peps_destroy", "peps_set_tensors", "peps_amplitudes", "peps_local_energy",
             "peps_log_derivatives", "peps_evaluate", "peps_gradient", "peps_mc_sweep", "peps_synchronize",
             "peps_status_str", "peps_last_error", "peps_debug_host_op", "peps_debug_host_zip",
             "peps_profile_enable", "peps_profile_read", "peps_amplitudes_static"]
    return {n: hasattr(L, n) for n in names}


def check(code):
    if code != PEPS_OK:
        raise PepsError(code, lib().peps_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def host_op(op, D, Dc, inputs, out_shape):
    """Runs one contraction program on host FP64 buffers (no GPU)."""
    ins = [_f64(x) for x in inputs] + [None] * (5 - len(inputs))
    out = np.zeros(out_shape, dtype=np.float64)
    check(lib().peps_debug_host_op(op, D, Dc, *[_ptr(x) for x in ins], _ptr(out)))
    return out


def host_zip(lr, D, Dc, dims, C, M, T, out_shape):
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    out = np.zeros(out_shape, dtype=np.float64)
    check(lib().peps_debug_host_zip(int(lr), D, Dc, _ptr(dims), _ptr(_f64(C)), _ptr(_f64(M)), _ptr(_f64(T)),
                                    _ptr(out)))
    return out


def amplitudes_static(A_dev, S, Lx, Ly, D, Dc, prec="fp64"):
    """ln|psi| and sign through the allocation-free entry point.

    ``A_dev`` is a CUDA tensor [N, 2, D^4] (float64 for fp64, float32 for
    fp32); ``S`` a CUDA int64 tensor [n, ceil(N/64)].  Outputs are allocated
    here by torch (the caller's memory); the library call itself allocates
    nothing."""
    import torch
    n = S.shape[0]
    params = Params(Lx, Ly, 2, D, Dc, 1.0, 0.0, PRECISIONS[prec], 0.0)
    la = torch.empty(n, dtype=torch.float64, device=S.device)
    sg = torch.empty(n, dtype=torch.int8, device=S.device)
    st = torch.empty(n, dtype=torch.int32, device=S.device)
    stream = torch.cuda.current_stream().cuda_stream
    check(lib().peps_amplitudes_static(ctypes.byref(params), _ptr(A_dev), _ptr(S), n, _ptr(la), _ptr(sg), _ptr(st),
                                       ctypes.c_void_p(stream)))
    return la, sg, st


class PEPS:
    """A PEPS (Eq. 1) on the GPU, with the boundary-MPS cut-off Dc (Fig. 1d).

    ``A`` is the padded float64 array [N][2][D][D][D][D] (index order l, r, u, d).
    Configurations are torch int64 tensors [n, ceil(N/64)] on the current
    CUDA device holding the bit-packed spins.
    """

    def __init__(self, A, Lx, Ly, D, Dc, J1=1.0, J2=0.0, prec="fp32", workspace_gb=0.0):
        import torch
        self.torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.Lx, self.Ly, self.D, self.Dc = Lx, Ly, D, Dc
        self.N = Lx * Ly
        self.nwords = (self.N + 63) // 64
        self.prec = prec
        self.real = torch.float64 if prec == "fp64" else torch.float32   # mixed paths store FP32
        self.params = Params(Lx, Ly, 2, D, Dc, float(J1), float(J2), PRECISIONS[prec], float(workspace_gb))
        A = _f64(A).copy()
        assert A.shape == (self.N, 2, D, D, D, D), A.shape
        self.A = A                                   # the FP64 tensors the context holds
        stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        check(lib().peps_create(ctypes.byref(self.params), _ptr(A), ctypes.c_void_p(stream), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().peps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _S(self, S):
        torch = self.torch
        if not isinstance(S, torch.Tensor):
            S = torch.from_numpy(np.ascontiguousarray(np.asarray(S).view(np.int64)))
        S = S.to(device="cuda", dtype=torch.int64).contiguous()
        assert S.dim() == 2 and S.shape[1] == self.nwords
        return S

    def set_tensors(self, A):
        A = _f64(A).copy()
        assert A.shape == (self.N, 2, self.D, self.D, self.D, self.D), A.shape
        check(lib().peps_set_tensors(self.h, _ptr(A)))
        self.A = A

    def go_step(self, grad, dt, seed, step, copy_back=True):
        """One gradient-optimisation update (Sec. III) with the derivative
        ``grad`` (CUDA FP64 [N][2][D^4], e.g. ``gradient(S)["grad"]``), in
        place on the device; the context then holds the new tensors.  With
        ``copy_back`` they are also copied to the host and returned (FP64)."""
        torch = self.torch
        g = grad.to(device="cuda", dtype=torch.float64).contiguous()
        shape = (self.N, 2, self.D, self.D, self.D, self.D)
        assert g.numel() == int(np.prod(shape)), g.shape
        out = np.empty(shape, dtype=np.float64) if copy_back else None
        check(lib().peps_go_step(self.h, _ptr(g), float(dt), int(seed), int(step), _ptr(out)))
        if copy_back:
            self.A = out
            return out.copy()
        self.A = None          # the host copy is stale until the next copy_back
        return None

    def evaluate(self, S, logabs=True, eloc=True, O=False):
        torch = self.torch
        S = self._S(S)
        n = S.shape[0]
        dev = S.device
        la = torch.empty(n, dtype=torch.float64, device=dev) if logabs else None
        sg = torch.empty(n, dtype=torch.int8, device=dev) if logabs else None
        el = torch.empty(n, dtype=torch.float64, device=dev) if eloc else None
        Ob = torch.empty((n, self.N, self.D ** 4), dtype=self.real, device=dev) if O else None
        st = torch.empty(n, dtype=torch.int32, device=dev)
        check(lib().peps_evaluate(self.h, _ptr(S), n, _ptr(la), _ptr(sg), _ptr(el), _ptr(Ob), _ptr(st)))
        return dict(logabs=la, sign=sg, eloc=el, O=Ob, status=st)

    def amplitudes(self, S):
        r = self.evaluate(S, logabs=True, eloc=False)
        return r["logabs"], r["sign"], r["status"]

    def local_energy(self, S):
        r = self.evaluate(S, logabs=False, eloc=True)
        return r["eloc"], r["status"]

    def log_derivatives(self, S):
        return self.evaluate(S, logabs=False, eloc=False, O=True)["O"]

    def gradient(self, S, per_config=False):
        torch = self.torch
        S = self._S(S)
        n = S.shape[0]
        dev = S.device
        grad = torch.empty((self.N, 2, self.D ** 4), dtype=torch.float64, device=dev)
        cov = torch.empty_like(grad)
        la = sg = el = st = None
        if per_config:
            la = torch.empty(n, dtype=torch.float64, device=dev)
            sg = torch.empty(n, dtype=torch.int8, device=dev)
            el = torch.empty(n, dtype=torch.float64, device=dev)
            st = torch.empty(n, dtype=torch.int32, device=dev)
        e = ctypes.c_double()
        used = ctypes.c_int()
        check(lib().peps_gradient(self.h, _ptr(S), n, ctypes.byref(e), _ptr(grad), _ptr(cov), _ptr(la), _ptr(sg),
                                  _ptr(el), _ptr(st), ctypes.byref(used)))
        out = dict(energy_per_site=e.value, grad=grad, cov=cov, n_used=used.value)
        if per_config:
            out.update(logabs=la, sign=sg, eloc=el, status=st)
        return out

    def mc_sweep(self, S, nsweeps, seed, chain0=0, sweep0=0):
        """In place on S (a CUDA int64 tensor); returns the accepted-move counts."""
        torch = self.torch
        assert isinstance(S, torch.Tensor) and S.is_cuda and S.dtype == torch.int64 and S.is_contiguous()
        n = S.shape[0]
        acc = torch.zeros(n, dtype=torch.int64, device=S.device)
        check(lib().peps_mc_sweep(self.h, _ptr(S), n, int(nsweeps), int(seed), int(chain0), int(sweep0), _ptr(acc)))
        return acc

    KERNELS = ["boundary", "row_sandwich", "pair_sandwich", "finalize", "grad_accum", "energy_sum",
               "grad_finalize", "mc_sweep"]

    def profile(self, on=True):
        check(lib().peps_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, reset=True):
        """{kernel: (milliseconds, launches)} since the last reset (synchronises the stream)."""
        ms = np.zeros(8, dtype=np.float64)
        n = np.zeros(8, dtype=np.int64)
        check(lib().peps_profile_read(self.h, _ptr(ms), _ptr(n), 1 if reset else 0))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KERNELS)}

    def synchronize(self):
        check(lib().peps_synchronize(self.h))
