"""Sampled spin correlations and M^2 (Sec. IV, peps_correlations) against
the FP64 oracle (oracle/correlations.py), configuration by configuration."""
import numpy as np
import pytest

from oracle import correlations as C
from paper_1611_09467_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_09467_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def packed(spins):
    return torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()


@pytest.mark.parametrize("L,D,Dc,margin,prec,near", [(6, 3, 4, 1, "fp64", False), (4, 2, 4, 0, "fp64", False),
                                                     (8, 4, 8, 2, "fp64", False), (8, 4, 8, 1, "fp32", True)])
def test_correlations_match_the_oracle(L, D, Dc, margin, prec, near):
    """Local M^2 of every configuration and the summed local S_p.S_q over the
    central sites: FP64 within 1e-10 (M^2) and 1e-9 (sums, relative to their
    size); FP32 on near-product tensors (well-conditioned cuts) within 1e-5.
    One configuration with S^z != 0 gets status 1, NaN M^2, and stays out of
    the sums."""
    from paper_1611_09467_gb300.peps import PEPS
    N = L * L
    A = inputs.near_product_tensors(L, L, D, 501) if near else inputs.make_tensors(L, L, D, 501)
    spins = inputs.random_sz0(12, N, 502)
    spins[5, np.flatnonzero(spins[5] == 0)[0]] = 1          # S^z != 0
    bad = True
    sites = C.central_sites(L, L, margin)
    p = PEPS(A, L, L, D, Dc, J1=1.0, J2=0.5, prec=prec)
    r = p.correlations(packed(spins), sites)
    torch.cuda.synchronize()
    m2 = r["m2"].cpu().numpy()
    corr = r["corr"].cpu().numpy()
    st = r["status"].cpu().numpy()
    tol_m2, tol_c = (1e-10, 1e-9) if prec == "fp64" else (1e-5, 1e-5)
    ref_sum = np.zeros((len(sites), len(sites)))
    worst = 0.0
    for k in range(len(spins)):
        if bad and k == 5:
            assert st[k] == 1 and np.isnan(m2[k])
            continue
        assert st[k] == 0
        ref = C.staggered_m2(A, spins[k], L, L, Dc, sites)
        worst = max(worst, abs(m2[k] - ref))
        assert abs(m2[k] - ref) < tol_m2, (k, m2[k], ref)
        ref_sum += C.correlations(A, spins[k], L, L, Dc, sites)
    print(f"{L}x{L} D={D} Dc={Dc} {prec}: {len(sites)} central sites, max |dM^2| {worst:.2e}, "
          f"max |d sum| {np.abs(corr - ref_sum).max():.2e}")
    assert np.abs(corr - ref_sum).max() < tol_c * max(1.0, np.abs(ref_sum).max())
    p.close()
