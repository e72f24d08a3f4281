"""The gradient-optimisation update on the device (Sec. III) against the
oracle: the update bit for bit (the keyed draws are integer hashes, and
A - (p dt) sign is evaluated in the same order on both sides), then the
refreshed context against a fresh context built on the updated tensors."""
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


@pytest.mark.parametrize("Ly,Lx,D,Dc,prec", [(4, 4, 2, 4, "fp64"), (5, 4, 3, 6, "fp32"),
                                             (6, 6, 8, 16, "mixed_tf32")])
def test_go_step_matches_oracle_and_refreshes_the_context(Ly, Lx, D, Dc, prec):
    from paper_1611_09467_gb300.peps import PEPS
    N = Ly * Lx
    A = inputs.make_tensors(Ly, Lx, D, seed=141)
    rng = np.random.default_rng(142)
    g = rng.standard_normal(A.shape) * inputs.edge_mask(Ly, Lx, D)
    g[N // 2, 1] = 0.0                       # a block that no sample selected
    g = g.reshape(N, 2, -1)
    p = PEPS(A, Lx, Ly, D, Dc, J1=1.0, J2=0.5, prec=prec)
    A1 = p.go_step(torch.from_numpy(g).cuda(), 0.004, seed=9, step=3)
    ref = O.go_step(A, g, 0.004, 9, 3)
    assert np.array_equal(A1, ref)
    assert not np.array_equal(A1, A)
    spins = inputs.random_sz0(8, N, 143)
    S = torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()
    r1 = p.evaluate(S, logabs=True, eloc=True)
    q = PEPS(A1, Lx, Ly, D, Dc, J1=1.0, J2=0.5, prec=prec)
    r2 = q.evaluate(S, logabs=True, eloc=True)
    torch.cuda.synchronize()
    for k in ("logabs", "sign", "eloc", "status"):
        assert torch.equal(r1[k], r2[k]), k
    p.close()
    q.close()
