"""The allocation-free amplitude entry point, for callers that cannot call
cudaMalloc (code inside another runtime's memory arena, real-time code that
must not allocate after start-up).

It must return what peps_amplitudes returns, on two calls in a row (its
static scratch keeps the previous call's contents).  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_1611_09467_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_09467_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
def test_static_amplitudes_match_context_path(prec, tol):
    from paper_1611_09467_gb300.peps import PEPS, amplitudes_static
    Ly = Lx = 6
    D, Dc = 3, 4          # truncated regime
    A = inputs.make_tensors(Ly, Lx, D, 91)
    spins = inputs.random_sz0(40, Ly * Lx, 92)
    spins[3, :3] = 1      # one configuration with S^z != 0 -> status 1
    S = torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()
    p = PEPS(A, Lx, Ly, D, Dc, J1=1.0, J2=0.5, prec=prec)
    la_ref, sg_ref, st_ref = p.amplitudes(S)
    dt = torch.float64 if prec == "fp64" else torch.float32
    A_dev = torch.from_numpy(A.reshape(Ly * Lx, 2, -1)).to(device="cuda", dtype=dt)
    for _ in range(2):
        la, sg, st = amplitudes_static(A_dev, S, Lx, Ly, D, Dc, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(sg.cpu(), sg_ref.cpu())
        assert torch.equal(st.cpu(), st_ref.cpu())
        assert (la.cpu() - la_ref.cpu()).abs().max().item() < tol
    p.close()


@pytest.mark.parametrize("prec,L,D,Dc,n,tol", [("fp32", 16, 8, 16, 40, 1e-6), ("fp64", 10, 6, 12, 64, 1e-10)])
def test_static_slots_reused_and_zero_amplitude(prec, L, D, Dc, n, tol):
    """More configurations than static slots, so every CTA walks several
    configurations through one slot and each finds the previous one's data
    there: 16x16 D=8 Dc=16 in FP32 takes ~0.6 MB per slot (about a dozen slots
    in 8 MiB) and 10x10 D=6 Dc=12 in FP64 ~0.4 MB (about twenty).  One site's
    spin-1 block is zero, so the configurations with that spin have W = 0
    (status 5, ln|psi| = -inf, sign 0) and sit between ordinary ones.
    Near-product tensors keep the FP32 contraction well conditioned."""
    from paper_1611_09467_gb300.peps import PEPS, amplitudes_static
    N = L * L
    A = inputs.near_product_tensors(L, L, D, 93)
    A[N // 3, 1] = 0.0
    spins = inputs.random_sz0(n, N, 94)
    hit = spins[:, N // 3] == 1
    assert 0 < hit.sum() < n
    S = torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()
    p = PEPS(A, L, L, D, Dc, J1=1.0, J2=0.5, prec=prec)
    la_ref, sg_ref, st_ref = p.amplitudes(S)
    dt = torch.float64 if prec == "fp64" else torch.float32
    A_dev = torch.from_numpy(A.reshape(N, 2, -1)).to(device="cuda", dtype=dt)
    for _ in range(2):
        la, sg, st = amplitudes_static(A_dev, S, L, L, D, Dc, prec=prec)
        torch.cuda.synchronize()
        st_h = st.cpu().numpy()
        assert (st_h[hit] == 5).all() and (st_h[~hit] == 0).all()
        assert np.isinf(la.cpu().numpy()[hit]).all() and (sg.cpu().numpy()[hit] == 0).all()
        assert torch.equal(sg.cpu(), sg_ref.cpu())
        assert torch.equal(st.cpu(), st_ref.cpu())
        ok = torch.from_numpy(~hit)
        assert (la.cpu()[ok] - la_ref.cpu()[ok]).abs().max().item() < tol
    p.close()


def test_static_rejects_oversized_lattice():
    """FP64, 64x64, D=8, Dc=32 needs ~12 MB of scratch per CTA, more than the
    8 MiB array: rejected before anything is read (A_dev is a placeholder)."""
    from paper_1611_09467_gb300.peps import PepsError, amplitudes_static
    S = torch.zeros((1, 64), dtype=torch.int64, device="cuda")
    A_dev = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(PepsError, match="static array"):
        amplitudes_static(A_dev, S, 64, 64, 8, 32, prec="fp64")
