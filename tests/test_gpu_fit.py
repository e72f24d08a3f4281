"""The variational-fit truncation mode (peps_set_truncation) against the
oracle's fit mode (absorb_row_fit): FP64 ln|psi|, E and Delta to the FP64
bounds on truncated lattices, both sweep directions (rows absorbed
left-to-right and right-to-left, top-down and bottom-up), exactness when
nothing is cut, and FP32 on near-product tensors."""
import numpy as np
import pytest

from oracle import peps_oracle as O
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


@pytest.mark.parametrize("Ly,Lx,D,Dc,sweeps,prec,near", [
    (4, 4, 2, 4, 2, "fp64", False),      # exact regime
    (6, 6, 3, 4, 1, "fp64", False),      # truncated
    (5, 4, 3, 5, 2, "fp64", False),      # odd number of rows, rectangular
    (6, 5, 4, 8, 1, "fp64", True),
    (6, 6, 4, 8, 2, "fp32", True),
])
def test_fit_mode_matches_the_oracle(Ly, Lx, D, Dc, sweeps, prec, near):
    from paper_1611_09467_gb300.peps import PEPS
    N = Ly * Lx
    A = inputs.near_product_tensors(Ly, Lx, D, 611) if near else inputs.make_tensors(Ly, Lx, D, 611)
    spins = inputs.random_sz0(6, N, 612)
    p = PEPS(A, Lx, Ly, D, Dc, J1=1.0, J2=0.5, prec=prec)
    p.set_truncation(sweeps)
    r = p.evaluate(packed(spins), logabs=True, eloc=True, O=True)
    z = PEPS(A, Lx, Ly, D, Dc, J1=1.0, J2=0.5, prec=prec).evaluate(packed(spins), logabs=True, eloc=False)
    torch.cuda.synchronize()
    tl, te, to = (1e-10, 1e-8, 1e-8) if prec == "fp64" else (2e-5, 1e-4, 1e-4)
    moved = 0.0
    for k in range(len(spins)):
        ev = O.evaluate(A, spins[k], Ly, Lx, Dc, 1.0, 0.5, fit_sweeps=sweeps)
        scale = 1.0 + sum(abs(J) / 4 + (abs(J) / 2 * abs(ev.ratios[(i, j)]) if spins[k][i] != spins[k][j] else 0)
                          for i, j, J, _ in O.all_bonds(Ly, Lx, 1.0, 0.5))
        dl = abs(r["logabs"][k].item() - ev.logabs)
        de = abs(r["eloc"][k].item() - ev.eloc)
        ref = ev.O.reshape(N, -1)
        do = float(np.abs(r["O"][k].cpu().numpy() - ref).max())
        print(f"{Ly}x{Lx} D={D} Dc={Dc} {prec} sweeps={sweeps} k={k}: d ln|psi| {dl:.2e}, dE/scale {de / scale:.2e}, "
              f"dDelta/max {do / np.abs(ref).max():.2e}")
        assert r["sign"][k].item() == ev.sign
        assert dl < tl
        assert de < te * scale
        assert do < to * np.abs(ref).max()
        moved = max(moved, abs(r["logabs"][k].item() - z["logabs"][k].item()))
    if Dc < D ** (Lx // 2):
        assert moved > 1e-8            # a different truncation from the zip-up's
    p.close()
