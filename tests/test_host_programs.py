"""CPU tests of the C ABI library: it loads, exports every declared symbol, and
its contraction programs (the index descriptors the kernels run) compute the
contractions they claim (host executor, no GPU)."""
import os
import re

import numpy as np
import pytest

from paper_1611_09467_gb300 import build, peps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def test_exports_every_declared_symbol():
    with open(os.path.join(ROOT, "include", "peps.h")) as f:
        header = f.read()
    declared = set(re.findall(r"\b(peps_[a-z_]+)\s*\(", header))
    L = peps.lib()
    missing = [n for n in declared if not hasattr(L, n)]
    assert not missing, missing
    assert len(declared) >= 12
    assert peps.lib().peps_status_str(5) == b"PEPS_ENUMERIC"


def test_phase_timing_build_exports_its_counters():
    """The diagnostic build behind phase_timing.py compiles (every source with
    -DPEPS_PHASE_TIMING, into its own directory) and exports the counter
    reader; the library itself does not have it."""
    import ctypes
    path = build.build(phase_timing=True)
    assert path != build.LIB and os.path.exists(path)
    D = ctypes.CDLL(path)
    assert hasattr(D, "peps_phase_read") and hasattr(D, "peps_create")
    assert not hasattr(peps.lib(), "peps_phase_read")


def _pad(t, shape):
    out = np.zeros(shape)
    out[tuple(slice(0, s) for s in t.shape)] = t
    return out


@pytest.mark.parametrize("D,Dc", [(2, 3), (3, 4), (2, 5)])
def test_single_row_programs(D, Dc):
    rng = np.random.default_rng(D * 10 + Dc)
    F = rng.standard_normal((Dc, D, Dc))
    G = rng.standard_normal((Dc, D, Dc))
    Mu = rng.standard_normal((Dc, D, Dc))
    Md = rng.standard_normal((Dc, D, Dc))
    T = rng.standard_normal((D, D, D, D))
    # F_c[b,r,b'] = sum F[a,l,a'] Mu[a,u,b] T[l,r,u,d] Md[a',d,b']
    ref = np.einsum("xly,xub,lrud,ydc->brc", F, Mu, T, Md)
    got = peps.host_op(0, D, Dc, [F, Mu, T, Md], (Dc, D, Dc))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
    ref = np.einsum("xub,lrud,ydc,brc->xly", Mu, T, Md, G)
    got = peps.host_op(1, D, Dc, [G, Mu, T, Md], (Dc, D, Dc))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
    ref = np.einsum("xly,xub,ydc,brc->lrud", F, Mu, Md, G)
    got = peps.host_op(2, D, Dc, [F, Mu, Md, G], (D, D, D, D))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("D,Dc", [(2, 3), (3, 2), (2, 4)])
def test_two_row_programs(D, Dc):
    rng = np.random.default_rng(100 + D * 10 + Dc)
    E = rng.standard_normal((Dc, D, D, Dc))
    H = rng.standard_normal((Dc, D, D, Dc))
    Mu = rng.standard_normal((Dc, D, Dc))
    Md = rng.standard_normal((Dc, D, Dc))
    T1 = rng.standard_normal((D, D, D, D))
    T2 = rng.standard_normal((D, D, D, D))
    # E_c[b,r1,r2,b'] = sum E[a,l1,l2,a'] Mu[a,u1,b] T1[l1,r1,u1,m] T2[l2,r2,m,d2] Md[a',d2,b']
    ref = np.einsum("aepq,aub,erum,psmd,qdc->brsc", E, Mu, T1, T2, Md)
    got = peps.host_op(3, D, Dc, [E, Mu, T1, T2, Md], (Dc, D, D, Dc))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
    ref = np.einsum("aub,erum,psmd,qdc,brsc->aepq", Mu, T1, T2, Md, H)
    got = peps.host_op(4, D, Dc, [H, Mu, T1, T2, Md], (Dc, D, D, Dc))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dirn", ["down", "up"])
@pytest.mark.parametrize("dims", [(3, 2, 4, 2, 2, 3, 2), (1, 1, 3, 1, 1, 2, 2), (4, 3, 1, 2, 3, 1, 1)])
def test_zip_programs(dirn, dims):
    """One zip-up column, both directions, with actual (unpadded) dims inside padded storage."""
    D, Dc = 3, 4
    k, a, b, i, l, r, o = dims
    rng = np.random.default_rng(sum(dims))
    Mt = rng.standard_normal((a, i, b))
    M = _pad(Mt, (Dc, D, Dc))
    # T[l][r][u][d]; 'in' leg = u (top-down, dirn='down') or d (bottom-up)
    if dirn == "down":
        Tt = rng.standard_normal((l, r, i, o))
        T = _pad(Tt, (D, D, D, D))
        Tin = Tt
        strides = (D ** 3, D ** 2, D, 1)
    else:
        Tt = rng.standard_normal((l, r, o, i))
        T = _pad(Tt, (D, D, D, D))
        Tin = Tt.transpose(0, 1, 3, 2)
        strides = (D ** 3, D ** 2, 1, D)
    # left to right: C[k][a][l] -> X[(k,o)][(b,r)]
    C = rng.standard_normal((k, a, l))
    ref = np.einsum("kal,aib,lrio->kobr", C, Mt, Tin).reshape(k * o, b * r)
    got = peps.host_zip(1, D, Dc, list(dims) + list(strides), C, M, T, (k * o, b * r))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
    # right to left: C[b][r][k] -> X[(o,k)][(a,l)]
    C = rng.standard_normal((b, r, k))
    ref = np.einsum("aib,lrio,brk->okal", Mt, Tin, C).reshape(o * k, a * l)
    got = peps.host_zip(0, D, Dc, list(dims) + list(strides), C, M, T, (o * k, a * l))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def _params(**kw):
    base = dict(Lx=4, Ly=4, d=2, D=2, Dc=4, J1=1.0, J2=0.5, prec=0, workspace_gb=0.0)
    base.update(kw)
    return peps.Params(**base)


def _create(params, A):
    import ctypes
    h = ctypes.c_void_p()
    code = peps.lib().peps_create(ctypes.byref(params), A.ctypes.data if A is not None else None, None,
                                  ctypes.byref(h))
    return code, h.value, peps.lib().peps_last_error().decode()


@pytest.mark.parametrize("kw,msg", [
    (dict(Lx=1), "Lx, Ly"), (dict(Ly=65), "Lx, Ly"), (dict(d=3), "d must be 2"),
    (dict(D=0), "D must be"), (dict(D=17), "D must be"), (dict(Dc=0), "Dc"), (dict(Dc=33), "Dc"),
    (dict(D=16, Dc=17), "Dc*D"), (dict(prec=3), "precision"), (dict(J2=float("nan")), "coupling"),
])
def test_create_rejects_invalid_parameters(kw, msg):
    """Argument checks of peps_create run before any device call: each bad
    parameter returns PEPS_EINVAL with a message and leaves no handle."""
    p = _params(**kw)
    D = min(max(p.D, 1), 16)
    A = np.zeros((max(p.Lx, 1) * max(p.Ly, 1), 2) + (D,) * 4)
    code, h, err = _create(p, A)
    assert code == 1 and h is None, (code, err)
    assert msg in err


def test_create_rejects_invalid_tensors():
    """Non-finite entries and non-zero entries past an open edge (bond
    dimension one there, Eq. 1) are rejected on the host."""
    from paper_1611_09467_gb300 import inputs
    A = inputs.make_tensors(4, 4, 2, 7)
    bad = A.copy()
    bad[5, 1, 0, 1, 1, 0] = np.nan
    code, h, err = _create(_params(), bad)
    assert (code, h) == (1, None) and "non-finite" in err
    bad = A.copy()
    bad[0, 0, 1, 0, 0, 0] = 1.0          # site 0 has no left neighbour: l must be 0
    code, h, err = _create(_params(), bad)
    assert (code, h) == (1, None) and "open edge" in err
    code, h, err = _create(_params(), None)
    assert (code, h) == (1, None) and "null" in err


def test_calls_reject_null_context_and_bad_batches():
    import ctypes
    L = peps.lib()
    la = np.zeros(1)
    assert L.peps_amplitudes(None, la.ctypes.data, 1, la.ctypes.data, la.ctypes.data, None) == 1
    assert "null context" in L.peps_last_error().decode()
    p = _params(Lx=1)
    assert L.peps_amplitudes_static(ctypes.byref(p), None, None, 0, None, None, None, None) == 1
    assert "out of range" in L.peps_last_error().decode()
    p = _params(prec=2)
    assert L.peps_amplitudes_static(ctypes.byref(p), None, None, 0, None, None, None, None) == 1
    assert "precision" in L.peps_last_error().decode()
    p = _params()
    assert L.peps_amplitudes_static(ctypes.byref(p), None, None, -1, None, None, None, None) == 1
    assert L.peps_go_step(None, None, 0.001, 1, 0, None) == 1
    assert "null argument" in L.peps_last_error().decode()
    assert [L.peps_status_str(c).decode() for c in range(6)] == [
        "PEPS_OK", "PEPS_EINVAL", "PEPS_ENOMEM", "PEPS_ECUDA", "PEPS_ETIMEOUT", "PEPS_ENUMERIC"]


def test_create_without_a_device_fails_cleanly():
    """With valid arguments and no GPU, peps_create reports the CUDA error
    instead of falling back to any host path."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1611_09467_gb300 import inputs
    code, h, err = _create(_params(), inputs.make_tensors(4, 4, 2, 7))
    assert code == 3 and h is None, (code, err)


def test_server_argument_checks():
    """The serving calls reject bad arguments before touching the device."""
    import ctypes
    from paper_1611_09467_gb300 import serve
    L = serve._lib()
    h = ctypes.c_void_p()
    assert L.peps_server_create(0, 1.0, ctypes.byref(h)) == 1 and h.value is None
    assert L.peps_server_create(65, 1.0, ctypes.byref(h)) == 1
    assert L.peps_server_create(2, 0.0, ctypes.byref(h)) == 1
    assert "nlanes" in L.peps_last_error().decode()
    nd = ctypes.c_int(7)
    assert L.peps_server_poll(None, 0, None, None, 0, ctypes.byref(nd)) == 1
    assert L.peps_server_submit(None, None, None, 1, None, None, None, None, None, None) == 1
    assert "bad request" in L.peps_last_error().decode()
    st = np.zeros(8)
    assert L.peps_server_stats(None, st.ctypes.data) == 1
    assert L.peps_server_set_policy(None, 1) == 1
