"""Pins of the correlation-function oracle (Sec. IV): exchange ratios against
exact contraction, the sampled estimator against <psi|S_i.S_j|psi> over the
full S^z = 0 basis, product-state closed forms, agreement with E(S)'s
horizontal ratios where both estimators coincide, and the Neel value of M^2."""
import math

import numpy as np
import pytest

from oracle import correlations as C
from oracle import peps_oracle as O
from paper_1611_09467_gb300 import inputs


def test_exchange_ratios_equal_exact_contraction_when_nothing_is_cut():
    """4x4 D=2 Dc=4 (exact regime): every pair's ratio equals
    psi(S^{ij}) / psi(S) from the exact contraction (Eq. 1)."""
    Ly = Lx = 4
    A = inputs.make_tensors(Ly, Lx, 2, 401)
    sites = list(range(16))
    for s in inputs.random_sz0(3, 16, 402):
        rat = C.exchange_ratios(A, s, Ly, Lx, 4, sites)
        w = O.contract_exact(O.project(A, s, Ly, Lx), Ly, Lx)
        anti = [(p, q) for p in range(16) for q in range(p + 1, 16) if s[p] != s[q]]
        assert sorted(rat) == anti
        for (p, q), x in rat.items():
            t = s.copy()
            t[p], t[q] = t[q], t[p]
            ref = O.contract_exact(O.project(A, t, Ly, Lx), Ly, Lx) / w
            assert abs(x - ref) < 1e-10 * (1 + abs(ref)), (p, q, x, ref)


def _apply_SS(psi, basis, i, j):
    """(S_i.S_j) psi on the S^z = 0 basis (S = sigma / 2)."""
    bi = (basis >> i) & 1
    bj = (basis >> j) & 1
    out = np.where(bi == bj, 0.25, -0.25) * psi
    anti = np.nonzero(bi != bj)[0]
    tgt = np.searchsorted(basis, basis[anti] ^ ((1 << i) | (1 << j)))
    np.add.at(out, tgt, 0.5 * psi[anti])
    return out


@pytest.mark.parametrize("Ly,Lx", [(2, 4), (3, 4)])
def test_sampled_estimator_is_the_expectation_over_the_basis(Ly, Lx):
    """Over every S^z = 0 configuration weighted by W(S)^2 / Z, the mean of
    (S_i.S_j)_loc equals <psi|S_i.S_j|psi> / <psi|psi> of the projected state
    (exact regime, D = 2, Dc = 4), for every pair, and the mean of the local
    M^2 equals the staggered sum of those expectations."""
    N = Ly * Lx
    A = inputs.make_tensors(Ly, Lx, 2, 403)
    basis, psi = O.exact_sz0_wavefunction(A, Ly, Lx)
    Z = psi @ psi
    sites = list(range(N))
    acc = np.zeros((N, N))
    m2 = 0.0
    for x, w in zip(basis, psi):
        s = [(int(x) >> i) & 1 for i in range(N)]
        acc += w * w * C.correlations(A, s, Ly, Lx, 4, sites)
        m2 += w * w * C.staggered_m2(A, s, Ly, Lx, 4, sites)
    acc /= Z
    m2 /= Z
    ref = np.eye(N) * 0.75
    for i in range(N):
        for j in range(N):
            if i != j:
                ref[i, j] = psi @ _apply_SS(psi, basis, i, j) / Z
    assert np.abs(acc - ref).max() < 1e-11
    eps = np.array([C.staggered_sign(i, Lx) for i in sites])
    assert abs(m2 - eps @ ref @ eps / N ** 2) < 1e-11


def test_product_state_closed_form():
    """D = 1 (a product state, any Dc): W(S^{ij}) / W(S) =
    t_i(s_j) t_j(s_i) / (t_i(s_i) t_j(s_j)) for every pair, at any distance."""
    Ly, Lx = 4, 6
    rng = np.random.default_rng(404)
    t = rng.uniform(0.3, 1.0, size=(Ly * Lx, 2)) * rng.choice([-1.0, 1.0], size=(Ly * Lx, 2))
    A = t.reshape(Ly * Lx, 2, 1, 1, 1, 1)
    s = inputs.random_sz0(1, Ly * Lx, 405)[0]
    sites = C.central_sites(Ly, Lx, 1)
    rat = C.exchange_ratios(A, s, Ly, Lx, 2, sites)
    for (p, q), x in rat.items():
        i, j = sites[p], sites[q]
        ref = t[i, s[j]] * t[j, s[i]] / (t[i, s[i]] * t[j, s[j]])
        assert abs(x - ref) < 1e-13 * abs(ref)


def test_same_row_neighbours_match_the_local_energy_ratios():
    """Truncated regime (6x6 D=3 Dc=4): for horizontal nearest neighbours both
    estimators use the same single-row sandwich, so the exchange ratio equals
    E(S)'s horizontal ratio (Sec. II) to rounding."""
    Ly = Lx = 6
    A = inputs.make_tensors(Ly, Lx, 3, 406)
    s = inputs.random_sz0(1, 36, 407)[0]
    sites = list(range(36))
    rat = C.exchange_ratios(A, s, Ly, Lx, 4, sites)
    ev = O.evaluate(A, s, Ly, Lx, 4, 1.0, 0.0, want_O=False)
    n = 0
    for (i, j), x in ev.ratios.items():
        if j == i + 1:
            assert abs(rat[(i, j)] - x) < 1e-10 * (1 + abs(x))
            n += 1
    assert n > 5


def test_neel_state_m2():
    """The Neel product state (only the staggered configuration has weight):
    no exchange contributes, so M^2 = (1/n^2)(n/2 + (n/2)^2) = 1/4 + 1/(2n)
    on n central sites."""
    Ly = Lx = 6
    N = Ly * Lx
    neel = np.array([(i // Lx + i % Lx) % 2 for i in range(N)])
    A = np.zeros((N, 2, 1, 1, 1, 1))
    A[np.arange(N), neel] = 1.0
    A[np.arange(N), 1 - neel] = 0.0
    sites = C.central_sites(Ly, Lx, 1)
    n = len(sites)
    m2 = C.staggered_m2(A, neel, Ly, Lx, 2, sites)
    assert abs(m2 - (0.25 + 0.5 / n)) < 1e-14
