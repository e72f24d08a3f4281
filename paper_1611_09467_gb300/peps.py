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
        "peps_gradient_sums": [P, P, i, P, i, P, P, P, P],
        "peps_set_graphs": [P, i],
        "peps_measure_peaks": [P],
        "peps_measure_tf32_mma_shape": [i, P],
        "peps_set_env_cache": [P, i],
        "peps_set_truncation": [P, i],
        "peps_correlations": [P, P, i, P, i, P, P, P],
        "peps_su_create": [ctypes.POINTER(Params), P, ctypes.POINTER(P)],
        "peps_su_destroy": [P],
        "peps_su_evolve": [P, P, P, d, i, ctypes.POINTER(d)],
        "peps_su_to_peps": [P, P, P, P],
        "peps_graph_stats": [P, P],
        "peps_autotune": [P, P, i, ctypes.c_char_p, ctypes.c_size_t],
        "peps_tuned_config": [P, P, ctypes.POINTER(d)],
        "peps_packer_create": [P, ctypes.POINTER(P)],
        "peps_packer_destroy": [P],
        "peps_packer_evaluate": [P, i, P, P, P, P, P, P, P, P],
        "peps_gradient_finalize": [P, P, ctypes.POINTER(d), ctypes.POINTER(d), P, P, ctypes.POINTER(i)],
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
    L.peps_gradient_sums_len.argtypes = [P]
    L.peps_gradient_sums_len.restype = ctypes.c_size_t
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
             "peps_profile_enable", "peps_profile_read", "peps_amplitudes_static", "peps_go_step",
             "peps_gradient_sums", "peps_gradient_sums_len", "peps_gradient_finalize", "peps_set_graphs",
             "peps_graph_stats", "peps_correlations", "peps_set_env_cache", "peps_set_truncation", "peps_measure_peaks",
             "peps_server_create",
             "peps_server_destroy", "peps_server_submit", "peps_server_submit_chain", "peps_server_set_packing", "peps_server_set_policy",
             "peps_server_poll", "peps_server_stats", "peps_su_create", "peps_su_destroy", "peps_su_evolve", "peps_su_to_peps",
             "peps_autotune", "peps_tuned_config", "peps_packer_create", "peps_packer_destroy",
             "peps_packer_evaluate"]
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


def measure_peaks():
    """Measured TFLOP/s of the pipes the kernels use on the current GPU:
    {"fp32_simt", "fp64_simt", "tf32_tcgen05"}."""
    out = np.zeros(3, dtype=np.float64)
    check(lib().peps_measure_peaks(_ptr(out)))
    return dict(fp32_simt=float(out[0]), fp64_simt=float(out[1]), tf32_tcgen05=float(out[2]))


def measure_mma_shape(n):
    """Measured TFLOP/s of dense TF32 tcgen05.mma instructions M = 128, N = n,
    K = 8 (operands in shared memory) on the current GPU."""
    out = np.zeros(1, dtype=np.float64)
    check(lib().peps_measure_tf32_mma_shape(int(n), _ptr(out)))
    return float(out[0])


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

    def gradient(self, S, per_config=False, out=None):
        """Energy per site and gradient over the batch S.  ``out`` (a dict a
        previous call returned, same batch size) reuses its tensors as the
        outputs, so repeated calls keep one signature for graph replay."""
        torch = self.torch
        S = self._S(S)
        n = S.shape[0]
        dev = S.device
        if out is not None:
            grad, cov = out["grad"], out["cov"]
            la, sg, el, st = (out.get(k) for k in ("logabs", "sign", "eloc", "status"))
        else:
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
        res = dict(energy_per_site=e.value, grad=grad, cov=cov, n_used=used.value)
        if la is not None:
            res.update(logabs=la, sign=sg, eloc=el, status=st)
        return res

    def gradient_sums(self, S, sums=None, accumulate=False):
        """The additive sums behind gradient() (layout in include/peps.h:
        sum E, count, sum E^2, 0, sum Delta [N][2][D^4], sum E Delta), as a CUDA
        float64 tensor; with ``sums`` given and ``accumulate``, added to it."""
        torch = self.torch
        S = self._S(S)
        if sums is None:
            sums = torch.empty(int(lib().peps_gradient_sums_len(self.h)), dtype=torch.float64, device=S.device)
        check(lib().peps_gradient_sums(self.h, _ptr(S), S.shape[0], _ptr(sums), 1 if accumulate else 0,
                                       None, None, None, None))
        return sums

    def gradient_from_sums(self, sums):
        """Energy per site, its variance, the gradient 2(<E Delta> - <E><Delta>)
        and its half from sums (e.g. added over ranks)."""
        torch = self.torch
        grad = torch.empty((self.N, 2, self.D ** 4), dtype=torch.float64, device=sums.device)
        cov = torch.empty_like(grad)
        e, v = ctypes.c_double(), ctypes.c_double()
        used = ctypes.c_int()
        check(lib().peps_gradient_finalize(self.h, _ptr(sums), ctypes.byref(e), ctypes.byref(v), _ptr(grad),
                                           _ptr(cov), ctypes.byref(used)))
        return dict(energy_per_site=e.value, energy_var=v.value, grad=grad, cov=cov, n_used=used.value)

    def correlations(self, S, sites, corr=True):
        """Local M^2 per configuration ([n] float64, NaN where status != 0) and,
        with ``corr``, the [nc, nc] sums of the local S_p.S_q over the
        configurations with status 0 (Sec. IV)."""
        torch = self.torch
        S = self._S(S)
        n = S.shape[0]
        sites = np.ascontiguousarray(sites, dtype=np.int32)
        m2 = torch.empty(n, dtype=torch.float64, device=S.device)
        C = torch.empty((len(sites), len(sites)), dtype=torch.float64, device=S.device) if corr else None
        st = torch.empty(n, dtype=torch.int32, device=S.device)
        check(lib().peps_correlations(self.h, _ptr(S), n, _ptr(sites), len(sites), _ptr(m2), _ptr(C), _ptr(st)))
        return dict(m2=m2, corr=C, status=st)

    def set_truncation(self, fit_sweeps=0):
        """0: zip-up SVD truncation; > 0: that many variational-fit sweeps after it."""
        check(lib().peps_set_truncation(self.h, int(fit_sweeps)))

    def set_env_cache(self, on=True):
        """Keep boundary environments across calls for unchanged configurations."""
        check(lib().peps_set_env_cache(self.h, 1 if on else 0))

    def set_graphs(self, on=True):
        """CUDA-graph replay of evaluate/gradient calls with a repeated signature."""
        check(lib().peps_set_graphs(self.h, 1 if on else 0))

    def graph_stats(self):
        v = np.zeros(3, dtype=np.int64)
        check(lib().peps_graph_stats(self.h, _ptr(v)))
        return dict(cached=int(v[0]), captures=int(v[1]), replays=int(v[2]))

    def autotune(self, S):
        """Times the kernel variants, grid and workspace on the probe batch S and
        keeps the fastest; returns the report (every trial and the choice)."""
        buf = ctypes.create_string_buffer(4096)
        S = self._S(S)
        check(lib().peps_autotune(self.h, _ptr(S), S.shape[0], buf, 4096))
        return buf.value.decode()

    def tuned_config(self):
        v = np.zeros(4, dtype=np.int32)
        ws = ctypes.c_double()
        check(lib().peps_tuned_config(self.h, _ptr(v), ctypes.byref(ws)))
        return dict(two_row_kernel=["tensor-core", "fused", "generic"][v[0]],
                    single_row_kernel=["fused", "generic"][v[1]], boundary_ctas=int(v[2]),
                    configs_per_chunk=int(v[3]), workspace_gb=ws.value)

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


class Packer:
    """Packed evaluation of requests of several models (boundary sweeps of all
    requests in one kernel launch) on the current torch stream."""

    def __init__(self):
        import torch
        self.torch = torch
        h = ctypes.c_void_p()
        check(lib().peps_packer_create(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().peps_packer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def evaluate(self, requests, eloc=True, O=False):
        """requests: [(PEPS, S)].  Returns one dict per request as PEPS.evaluate."""
        torch = self.torch
        k = len(requests)
        outs = []
        arr = lambda t: (ctypes.c_void_p * k)(*t)
        ctxs, Ss, ns, la, sg, el, Ob, st = [], [], [], [], [], [], [], []
        for m, S in requests:
            S = m._S(S)
            n = S.shape[0]
            o = dict(S=S, logabs=torch.empty(n, dtype=torch.float64, device=S.device),
                     sign=torch.empty(n, dtype=torch.int8, device=S.device),
                     eloc=torch.empty(n, dtype=torch.float64, device=S.device) if eloc else None,
                     O=torch.empty((n, m.N, m.D ** 4), dtype=m.real, device=S.device) if O else None,
                     status=torch.empty(n, dtype=torch.int32, device=S.device))
            outs.append(o)
            ctxs.append(m.h.value)
            Ss.append(S.data_ptr())
            ns.append(n)
            la.append(o["logabs"].data_ptr())
            sg.append(o["sign"].data_ptr())
            el.append(o["eloc"].data_ptr() if eloc else None)
            Ob.append(o["O"].data_ptr() if O else None)
            st.append(o["status"].data_ptr())
        nn = (ctypes.c_int * k)(*ns)
        check(lib().peps_packer_evaluate(self.h, k, arr(ctxs), arr(Ss), nn, arr(la), arr(sg), arr(el), arr(Ob),
                                         arr(st)))
        for o in outs:
            o.pop("S")
        return outs


class SimpleUpdate:
    """Simple-update imaginary-time evolution (Sec. III) on the GPU.

    ``Gam`` [N][2][D^4] float64 (the Gamma tensors, padded like A) and ``lam``
    [nbonds][D] float64 (bond weights; horizontal bonds row-major, then
    vertical) are held as CUDA tensors in ``self.Gam`` and ``self.lam``."""

    def __init__(self, Gam, lam, Lx, Ly, D, J1=1.0, J2=0.0):
        import torch
        self.torch = torch
        self.Lx, self.Ly, self.D, self.N = Lx, Ly, D, Lx * Ly
        self.Gam = torch.as_tensor(np.ascontiguousarray(Gam, dtype=np.float64)).reshape(self.N, 2, D ** 4).cuda()
        self.lam = torch.as_tensor(np.ascontiguousarray(lam, dtype=np.float64)).reshape(-1, D).cuda()
        params = Params(Lx, Ly, 2, D, D, float(J1), float(J2), 0, 0.0)
        h = ctypes.c_void_p()
        check(lib().peps_su_create(ctypes.byref(params), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                   ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().peps_su_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def evolve(self, dtau, nsteps, measure=True):
        """nsteps Trotter steps; returns max|A' - A| / max|A| over the last one
        (or None without ``measure``)."""
        c = ctypes.c_double()
        check(lib().peps_su_evolve(self.h, _ptr(self.Gam), _ptr(self.lam), float(dtau), int(nsteps),
                                   ctypes.byref(c) if measure else None))
        return c.value if measure else None

    def to_peps(self):
        """The PEPS tensors A [N][2][D^4] (CUDA float64, unit norm per site)."""
        A = self.torch.empty_like(self.Gam)
        check(lib().peps_su_to_peps(self.h, _ptr(self.Gam), _ptr(self.lam), _ptr(A)))
        return A
