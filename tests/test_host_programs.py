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
