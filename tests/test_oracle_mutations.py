"""Mutation check of the oracle's pins.

Each plausible mistake below (a dropped term, a wrong sign, an index or an
operand mixed up, an off-by-one) is planted in the oracle, on the CPU,
through monkeypatch; the pins of test_oracle.py that should catch it must
then fail.  This shows that the pins constrain each part of what the oracle
computes, rather than only that the oracle passes them.
"""
import numpy as np
import pytest

import test_oracle as P
import test_oracle_go as G
from oracle import peps_oracle as O

PINS = {
    "bonds": P.test_bond_counts_and_codec,
    "ed_2x2": P.test_ed_2x2_closed_form,
    "ed_4x4": P.test_ed_4x4_table1,
    "bruteforce": lambda: P.test_exact_contraction_vs_bruteforce(2, 3, 2),
    "exact_regime": lambda: P.test_boundary_mps_exact_regime(4, 4, 2, 4),
    "converges": P.test_boundary_mps_truncates_and_converges_with_dc,
    "linearity": P.test_linearity_in_each_tensor,
    "product": P.test_product_state_closed_forms,
    "H_psi": lambda: P.test_local_energy_equals_H_psi_over_psi(3, 4, 2, 4, 0.5),
    "fd": P.test_log_derivative_vs_finite_differences,
    "euler": P.test_euler_identity_truncated,
    "gradient": P.test_gradient_estimator_equals_energy_derivative,
    "splitmix": P.test_sampler_uniform_is_splitmix64,
    "chi2": P.test_sampler_stationary_distribution_chi_square,
    "go_move": G.test_go_step_moves_against_the_sign_by_less_than_dt,
    "go_descends": G.test_go_descends_the_exact_energy,
}


def drop_nnn(mp):
    """J2 bonds left out of the bond list."""
    mp.setattr(O, "nnn_bonds", lambda Ly, Lx: ([], []))


def antidiagonal_as_diagonal(mp):
    """The anti-diagonal pairs (r,c+1)-(r+1,c) replaced by the diagonal ones."""
    orig = O.nnn_bonds
    mp.setattr(O, "nnn_bonds", lambda Ly, Lx: (orig(Ly, Lx)[0], orig(Ly, Lx)[0]))


def exchange_sign(mp):
    """Wrong sign of the spin-exchange part (S+S- + S-S+)/2 of H."""
    import scipy.sparse as sp
    orig = O.hamiltonian_sz0

    def h(Ly, Lx, J1, J2):
        H, basis = orig(Ly, Lx, J1, J2)
        d = sp.diags(H.diagonal())
        return (2 * d - H).tocsr(), basis
    mp.setattr(O, "hamiltonian_sz0", h)


def truncation_off_by_one(mp):
    """One singular vector fewer kept at every cut (K = Dc - 1)."""
    orig = O.absorb_row
    mp.setattr(O, "absorb_row", lambda mps, Trow, Dc, left_to_right, perturb=None:
               orig(mps, Trow, max(1, Dc - 1), left_to_right, perturb))


def _reassemble_eloc(ev, spins, Ly, Lx, J1, J2):
    e = 0.0
    for i, j, J, _ in O.all_bonds(Ly, Lx, J1, J2):
        e += 0.25 * J if spins[i] == spins[j] else -0.25 * J + 0.5 * J * ev.ratios[(i, j)]
    ev.eloc = e


def ratio_inverted(mp):
    """E_loc built from W(S)/W(S') instead of W(S')/W(S)."""
    orig = O.evaluate

    def ev(A, spins, Ly, Lx, Dc, J1, J2, want_O=True, perturb=None):
        e = orig(A, spins, Ly, Lx, Dc, J1, J2, want_O, perturb)
        if e.status == 0:
            e.ratios = {k: 1.0 / v for k, v in e.ratios.items()}
            _reassemble_eloc(e, np.asarray(spins), Ly, Lx, J1, J2)
        return e
    mp.setattr(O, "evaluate", ev)


def delta_not_divided(mp):
    """Delta = B instead of B / W (the division by the sandwich left out)."""
    orig = O.evaluate

    def ev(A, spins, Ly, Lx, Dc, J1, J2, want_O=True, perturb=None):
        e = orig(A, spins, Ly, Lx, Dc, J1, J2, want_O, perturb)
        if e.status == 0 and e.O is not None:
            for i in range(Ly * Lx):
                e.O[i] *= e.W_row[i // Lx]
        return e
    mp.setattr(O, "evaluate", ev)


def wrong_spin_block(mp):
    """Site 0 projected on the other spin block."""
    orig = O.project
    mp.setattr(O, "project", lambda A, spins, Ly, Lx:
               orig(A, [1 - int(spins[0])] + [int(x) for x in spins[1:]], Ly, Lx))


def gradient_without_mean_term(mp):
    """g = 2<E O>: the -2<E><O> term dropped."""
    orig = O.gradient

    def g(evals, spins_batch, N, D, d=2, weights=None):
        e_site, grad, cov, n = orig(evals, spins_batch, N, D, d, weights)
        ok = [k for k, ev in enumerate(evals) if ev.status == 0]
        w = np.ones(len(evals)) if weights is None else np.asarray(weights, dtype=np.float64)
        obar = np.zeros((N, d, D ** 4))
        for k in ok:
            for i in range(N):
                obar[i, int(spins_batch[k][i])] += w[k] * evals[k].O[i].reshape(-1)
        obar /= sum(w[k] for k in ok)
        grad = grad + 2.0 * (e_site * N) * obar
        return e_site, grad, grad / 2, n
    mp.setattr(O, "gradient", g)


def acceptance_abs_ratio(mp):
    """Metropolis with |W(S')/W(S)| instead of its square (u^2 < r^2 iff u < |r|)."""
    orig = O.sampler_uniform
    mp.setattr(O, "sampler_uniform", lambda *a: orig(*a) ** 2)


def go_along_the_sign(mp):
    """GO update with the wrong sign: A + p dt sign(dE/dA)."""
    orig = O.go_step
    mp.setattr(O, "go_step", lambda A, grad, dt, seed, step: 2 * A - orig(A, grad, dt, seed, step))


def go_uses_the_value(mp):
    """GO update with the derivative's value instead of its sign."""
    mp.setattr(O, "go_step", lambda A, grad, dt, seed, step:
               A - O.go_uniform(seed, step, A.size).reshape(A.shape) * dt * np.reshape(grad, A.shape))


# each planted mistake and the pins that must catch it
EXPECTED = [
    (drop_nnn, ["bonds", "ed_2x2"]),
    (antidiagonal_as_diagonal, ["bonds"]),
    (exchange_sign, ["ed_2x2", "H_psi", "gradient"]),
    (truncation_off_by_one, ["exact_regime", "converges", "H_psi", "fd"]),
    (ratio_inverted, ["product", "H_psi", "gradient"]),
    (delta_not_divided, ["product", "fd", "euler", "gradient"]),
    (wrong_spin_block, ["product", "H_psi", "fd", "euler", "gradient", "chi2"]),
    (gradient_without_mean_term, ["gradient"]),
    (acceptance_abs_ratio, ["splitmix", "chi2"]),
    (go_along_the_sign, ["go_move", "go_descends"]),
    (go_uses_the_value, ["go_move"]),
]


@pytest.mark.parametrize("plant,pins", EXPECTED, ids=[m.__name__ for m, _ in EXPECTED])
def test_pins_catch_planted_mistake(plant, pins, monkeypatch):
    plant(monkeypatch)
    missed = []
    for name in pins:
        try:
            PINS[name]()
        except AssertionError:
            continue
        missed.append(name)
    assert not missed, f"{plant.__name__} passes {missed}"
