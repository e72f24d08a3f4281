"""Pins of the oracle's gradient-optimisation (GO) update (Sec. III): its keyed
draw, the update rule, the step-length schedule of the paper's run, and that
the update descends the exact energy."""
import math

import numpy as np
import pytest

from oracle import peps_oracle as O
from paper_1611_09467_gb300 import inputs


def test_go_draw_is_splitmix64():
    """The vectorised mix equals the scalar SplitMix64 output function (itself
    pinned by the published first output for seed 0); the draws are uniform
    on [0, 1), reproducible for a key, and differ between steps."""
    rng = np.random.default_rng(1)
    z = rng.integers(0, 2 ** 63, size=2000, dtype=np.uint64) * np.uint64(2) \
        + rng.integers(0, 2, size=2000, dtype=np.uint64)
    vec = O._mix64_vec(z)
    assert all(int(v) == O._mix64(int(x)) for x, v in zip(z, vec))
    assert int(O._mix64_vec(np.uint64(0x9E3779B97F4A7C15))) == 0xE220A8397B1DCDAF
    u = O.go_uniform(11, 3, 200_000)
    assert 0.0 <= u.min() and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1.0 / 12) < 2e-3
    assert np.array_equal(u, O.go_uniform(11, 3, 200_000))
    assert not np.array_equal(u[:1000], O.go_uniform(11, 4, 1000))


def test_go_step_moves_against_the_sign_by_less_than_dt():
    """Every element moves by p*dt, 0 <= p < 1, against the sign of its
    derivative; zero derivative, no move; the moves' p have mean 1/2."""
    Ly = Lx = 6
    D = 4
    A = inputs.make_tensors(Ly, Lx, D, seed=5)
    rng = np.random.default_rng(6)
    g = rng.standard_normal(A.shape) * inputs.edge_mask(Ly, Lx, D)   # zero past open edges
    g[3, 1] = 0.0                                                    # a block no sample selected
    dt = 0.004
    B = O.go_step(A, g.reshape(Ly * Lx, 2, -1), dt, seed=9, step=2)
    d = B - A
    moving = g != 0
    assert np.all(np.sign(d[moving]) == -np.sign(g[moving]))
    assert np.all(np.abs(d) < dt)
    assert np.all(d[~moving] == 0.0)
    # ~10^4 moving elements: the mean of p is 1/2 within 5 standard errors
    assert abs(np.mean(np.abs(d[moving]) / dt) - 0.5) < 0.015


def test_go_schedule_matches_the_papers_run():
    """dt = 0.005 for 50 steps, then multiplied by 0.968 per step down to 0.001
    over the next 50, then 0.001 (Sec. III, the 10x10 D=8 run of Fig. 4)."""
    assert O.go_dt(0) == O.go_dt(49) == 0.005
    assert O.go_dt(50) == pytest.approx(0.005 * 0.968)
    assert O.go_dt(98) > 0.001 and O.go_dt(99) == 0.001
    assert O.go_dt(119) == 0.001
    assert all(O.go_dt(n + 1) <= O.go_dt(n) for n in range(130))


def test_go_descends_the_exact_energy():
    """With the exact gradient (every S^z = 0 configuration weighted by W^2/Z,
    the estimator pinned against finite differences), GO steps lower
    <psi|H|psi>/<psi|psi> at every step and stay above the ED ground energy
    (variational bound).  2x4, D = 2 (exact contraction), J2 = 0.5."""
    Ly, Lx, D, Dc, J2 = 2, 4, 2, 4, 0.5
    N = Ly * Lx
    A = inputs.make_tensors(Ly, Lx, D, seed=131)
    H, basis = O.hamiltonian_sz0(Ly, Lx, 1.0, J2)
    spins = [[(int(x) >> i) & 1 for i in range(N)] for x in basis]
    e0 = O.ground_energy(Ly, Lx, 1.0, J2)

    def energy(B):
        _, p = O.exact_sz0_wavefunction(B, Ly, Lx)
        return p @ (H @ p) / (p @ p)

    es = [energy(A)]
    for n in range(12):
        evals = [O.evaluate(A, s, Ly, Lx, Dc, 1.0, J2) for s in spins]
        w = np.array([math.exp(2 * ev.logabs) if ev.status == 0 else 0.0 for ev in evals])
        _, g, _, _ = O.gradient(evals, spins, N, D, weights=w)
        A = O.go_step(A, g, 0.003, seed=17, step=n)
        es.append(energy(A))
    assert all(b < a for a, b in zip(es, es[1:])), es
    assert es[-1] > e0


def test_exact_gradient_go_driver_descends():
    """oracle/go_exact.py on 2x2 (3 steps): energies fall and stay above ED."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "oracle.go_exact", "--L", "2", "--steps", "3", "--workers", "1"],
                       cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x.split() for x in r.stdout.splitlines() if x and not x.startswith("#")]
    e = [float(x[2]) for x in lines]
    assert len(e) == 3 and e[0] > e[1] > e[2] > -0.5


def test_go_step_rejects_non_finite_derivatives():
    """A NaN or infinite derivative has no sign to step against: the update
    raises instead of moving (the GPU path refuses it with EINVAL)."""
    A = inputs.make_tensors(3, 3, 2, seed=5)
    g = np.ones((9, 2, 16))
    for bad in (np.nan, np.inf, -np.inf):
        gb = g.copy()
        gb[4, 1, 3] = bad
        with pytest.raises(ValueError):
            O.go_step(A, gb, 0.004, 1, 0)
