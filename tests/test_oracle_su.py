"""Pins of the simple-update oracle (Sec. III, the SU initialiser): its gate
against the matrix exponential, one bond update against the exact action of
the gate where nothing is truncated, its truncation against the best
rank-D approximation, and the imaginary-time evolution against the
variational bound and the paper's SU energy (Table I)."""
import math

import numpy as np
import pytest

from oracle import peps_oracle as O
from oracle import simple_update as SU
from paper_1611_09467_gb300 import inputs


def test_gate_is_the_exponential_of_the_heisenberg_pair():
    """S_i.S_j has the eigenvalues 1/4 (three times) and -3/4 (the singlet);
    the gate equals scipy's expm(-dtau J S.S)."""
    sl = pytest.importorskip("scipy.linalg")
    h = SU.heisenberg_pair()
    assert np.allclose(np.sort(np.linalg.eigvalsh(h)), [-0.75, 0.25, 0.25, 0.25])
    for J, dt in ((1.0, 0.01), (0.5, 0.001), (1.0, 0.7)):
        assert np.abs(SU.gate(J, dt) - sl.expm(-dt * J * h)).max() < 1e-14
    assert np.allclose(SU.SWAP @ SU.SWAP, np.eye(4))


def _vector(A, Ly, Lx):
    """All 2^N amplitudes of the PEPS (exact contraction), index sum_i s_i 2^(N-1-i)."""
    N = Ly * Lx
    out = np.zeros(2 ** N)
    for x in range(2 ** N):
        spins = [(x >> (N - 1 - i)) & 1 for i in range(N)]
        out[x] = O.contract_exact(O.project(A, spins, Ly, Lx), Ly, Lx)
    return out


def _apply_pair(G, psi, i, j, N):
    """G (basis 2 s_i + s_j) applied to sites i, j of a 2^N vector."""
    t = psi.reshape([2] * N)
    t = np.moveaxis(t, [i, j], [0, 1])
    t = np.tensordot(G.reshape(2, 2, 2, 2), t, axes=([2, 3], [0, 1]))
    return np.moveaxis(t, [0, 1], [i, j]).reshape(-1)


@pytest.mark.parametrize("bond", [(0, 1), (1, 3), (2, 3), (0, 2)])
def test_bond_update_on_a_product_state_is_the_gate(bond):
    """From a product state (every bond of dimension one), a gate on one bond
    needs bond dimension <= 2 = D: nothing is cut, so the updated PEPS is
    exactly G|psi> up to normalisation, on a horizontal or vertical bond."""
    Ly = Lx = 2
    D = 2
    rng = np.random.default_rng(3)
    Gam = np.zeros((4, 2, D, D, D, D))
    Gam[:, :, 0, 0, 0, 0] = rng.standard_normal((4, 2))
    lam = {b: np.array([1.0, 0.0]) for b in [(0, 1), (2, 3), (0, 2), (1, 3)]}
    psi0 = _vector(SU.to_peps(Gam, lam, Ly, Lx), Ly, Lx)
    G = SU.gate(1.0, 0.3)
    SU.bond_update(Gam, lam, bond[0], bond[1], G, Ly, Lx, D)
    psi1 = _vector(SU.to_peps(Gam, lam, Ly, Lx), Ly, Lx)
    ref = _apply_pair(G, psi0, bond[0], bond[1], 4)
    cos = abs(psi1 @ ref) / (np.linalg.norm(psi1) * np.linalg.norm(ref))
    assert cos > 1 - 1e-13
    assert abs(np.linalg.norm(lam[bond]) - 1.0) < 1e-14


def test_truncation_keeps_the_largest_singular_values():
    """An entangling gate on a bond of dimension D = 1 keeps the largest
    Schmidt value only: the two-site state becomes the best product (rank-1)
    approximation of G|psi>, whose overlap is sigma_1 / |G psi|."""
    Ly = Lx = 2
    D = 1
    rng = np.random.default_rng(4)
    Gam = rng.standard_normal((4, 2, 1, 1, 1, 1))
    lam = {b: np.array([1.0]) for b in [(0, 1), (2, 3), (0, 2), (1, 3)]}
    psi0 = _vector(SU.to_peps(Gam, lam, Ly, Lx), Ly, Lx)
    G = SU.gate(1.0, 1.0)
    SU.bond_update(Gam, lam, 0, 1, G, Ly, Lx, D)
    psi1 = _vector(SU.to_peps(Gam, lam, Ly, Lx), Ly, Lx)
    ref = _apply_pair(G, psi0, 0, 1, 4)
    # Schmidt values of ref across site 0 | sites 1, 2, 3 (sites 2, 3 are a product with the pair)
    sv = np.linalg.svd(ref.reshape(2, 8), compute_uv=False)
    ov = abs(psi1 @ ref) / (np.linalg.norm(psi1) * np.linalg.norm(ref))
    assert abs(ov - sv[0] / np.linalg.norm(sv)) < 1e-12


def test_imaginary_time_evolution_descends_to_the_su_energy():
    """4x4, J2 = 0, D = 2 from the seeded random tensors, dtau = 0.01: the exact
    energy of the SU state falls, stays above ED, and after 500 Trotter
    steps lies within 0.01 of the paper's SU value for D = 2 (Table I,
    -0.54557; the paper's runs start from other tensors and read the energy
    by sampling)."""
    L, D = 4, 2
    H, _ = O.hamiltonian_sz0(L, L, 1.0, 0.0)

    def energy(A):
        _, psi = O.exact_sz0_wavefunction(A, L, L)
        return float(psi @ (H @ psi) / (psi @ psi)) / (L * L)

    Gam, lam = SU.init_state(L, L, D, 301)
    e = [energy(SU.to_peps(Gam, lam, L, L))]
    for _ in range(5):
        SU.evolve(Gam, lam, L, L, 1.0, 0.0, D, 0.01, 100)
        e.append(energy(SU.to_peps(Gam, lam, L, L)))
    ed = O.ground_energy(L, L, 1.0, 0.0) / (L * L)
    print(" ".join("%.5f" % x for x in e))
    assert all(b < a + 1e-6 for a, b in zip(e, e[1:]))
    assert e[-1] > ed
    assert abs(e[-1] - (-0.54557)) < 0.01


def test_next_nearest_routes_cover_each_pair_once():
    """Every NNN pair of the lattice appears in exactly one route (i, j, k) with
    i, j nearest neighbours and j, k nearest neighbours; no two routes of a
    group share a site."""
    Ly, Lx = 4, 5
    d1, d2 = O.nnn_bonds(Ly, Lx)
    want = {tuple(sorted(p)) for p in d1 + d2}
    got = []
    nn = {tuple(sorted(p)) for grp in O.nn_bonds(Ly, Lx) for p in grp}
    for group in SU.nnn_routes(Ly, Lx):
        sites = [s for r in group for s in r]
        assert len(sites) == len(set(sites))
        for i, j, k in group:
            assert tuple(sorted((i, j))) in nn and tuple(sorted((j, k))) in nn
            got.append(tuple(sorted((i, k))))
    assert sorted(got) == sorted(want)
