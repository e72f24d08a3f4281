"""The simple-update initialiser on the GPU (peps_su_*) against the FP64
oracle (oracle/simple_update.py): bond weights and the state after a number of
Trotter steps, with and without next-nearest gates, then a converged run.

Singular vectors are fixed only up to sign, so the tensors are compared
through what does not depend on that choice: the bond weights (singular
values) and the wavefunction of the PEPS (exact contraction, up to an overall
sign)."""
import math

import numpy as np
import pytest

from oracle import peps_oracle as O
from oracle import simple_update as SU

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_09467_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def lam_array(lam, Ly, Lx):
    h, v = O.nn_bonds(Ly, Lx)
    return np.stack([lam[b] for b in h + v])


def gpu_state(Gam, lam, Ly, Lx, D, J1, J2):
    from paper_1611_09467_gb300.peps import SimpleUpdate
    return SimpleUpdate(Gam, lam_array(lam, Ly, Lx), Lx, Ly, D, J1=J1, J2=J2)


def wavefunction(A, L):
    _, psi = O.exact_sz0_wavefunction(A, L, L)
    return psi / np.linalg.norm(psi)


@pytest.mark.parametrize("D,J2,steps,dtau", [(2, 0.0, 20, 0.01), (3, 0.5, 8, 0.01), (2, 0.5, 5, 0.2)])
def test_su_steps_match_the_oracle(D, J2, steps, dtau):
    """4x4 from the same seeded tensors: after the Trotter steps every bond
    weight agrees to 1e-10 and the S^z = 0 wavefunction of the PEPS to 1e-9
    (overall sign free); with J2 = 0.5 the next-nearest gates (SWAP routes)
    run too.  dtau = 0.2 makes large single steps."""
    L = 4
    Gam, lam = SU.init_state(L, L, D, 311)
    s = gpu_state(Gam, lam, L, L, D, 1.0, J2)
    for _ in range(steps):
        SU.trotter_step(Gam, lam, L, L, 1.0, J2, dtau, D)
    s.evolve(dtau, steps, measure=False)
    lg = s.lam.cpu().numpy()
    lo = lam_array(lam, L, L)
    print("max weight difference %.2e" % np.abs(lg - lo).max())
    assert np.abs(lg - lo).max() < 1e-10
    A_gpu = s.to_peps().cpu().numpy().reshape(L * L, 2, D, D, D, D)
    A_or = SU.to_peps(Gam, lam, L, L)
    pg, po = wavefunction(A_gpu, L), wavefunction(A_or, L)
    d = min(np.linalg.norm(pg - po), np.linalg.norm(pg + po))
    print("wavefunction difference %.2e" % d)
    assert d < 1e-9
    mask = np.broadcast_to(__import__("paper_1611_09467_gb300.inputs", fromlist=["x"]).edge_mask(L, L, D),
                           A_gpu.shape)
    assert (A_gpu[~mask] == 0).all()
    s.close()


def test_su_converges_to_the_oracles_energy():
    """4x4 J2 = 0 D = 2 with the paper's schedule (dtau = 0.01 until the
    relative change is below 1e-6, then 0.001 likewise): the exact energy of
    the GPU's converged PEPS equals the oracle's converged one within 1e-5
    (both stop at the same criterion, not the same step) and lies within 0.01
    of Table I's SU value (-0.54557)."""
    L, D = 4, 2
    H, _ = O.hamiltonian_sz0(L, L, 1.0, 0.0)

    def energy(A):
        _, psi = O.exact_sz0_wavefunction(A, L, L)
        return float(psi @ (H @ psi) / (psi @ psi)) / (L * L)

    Gam, lam = SU.init_state(L, L, D, 301)
    s = gpu_state(Gam, lam, L, L, D, 1.0, 0.0)
    steps = 0
    for dtau in (0.01, 0.001):
        for _ in range(200):
            ch = s.evolve(dtau, 50)
            steps += 50
            if ch < 1e-6:
                break
        print("dtau %.3f: relative change %.2e after %d steps" % (dtau, ch, steps))
    e_gpu = energy(s.to_peps().cpu().numpy().reshape(L * L, 2, D, D, D, D))
    for dtau in (0.01, 0.001):
        for _ in range(200):
            if SU.evolve(Gam, lam, L, L, 1.0, 0.0, D, dtau, 50) < 1e-6:
                break
    e_or = energy(SU.to_peps(Gam, lam, L, L))
    print("energy per site: gpu %.7f oracle %.7f" % (e_gpu, e_or))
    assert abs(e_gpu - e_or) < 1e-5
    assert abs(e_gpu - (-0.54557)) < 0.01
    s.close()


def test_su_full_size_step_rate():
    """16x16, D = 8, J2/J1 = 0.5 (the large workload's shape): Trotter steps
    run and keep the weights normalised; the step rate is printed."""
    import time
    from paper_1611_09467_gb300 import inputs
    L, D = 16, 8
    Gam, lam = SU.init_state(L, L, D, 321)
    s = gpu_state(Gam, lam, L, L, D, 1.0, 0.5)
    s.evolve(0.01, 2, measure=False)
    torch.cuda.synchronize()
    t = time.perf_counter()
    ch = s.evolve(0.01, 10)
    dt = time.perf_counter() - t
    nb = s.lam.shape[0]
    print("16x16 D=8 J2=0.5: %.1f Trotter steps/s (%d bonds, %d next-nearest routes), change %.2e"
          % (10 / dt, nb, 2 * (L - 1) ** 2, ch))
    w = s.lam.cpu().numpy()
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0, atol=1e-12)
    assert np.isfinite(s.Gam.cpu().numpy()).all()
    s.close()
