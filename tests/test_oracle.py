"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the pin it implements; none compares the oracle with itself
by retyping one of its formulas.
"""
import math
import os

import numpy as np
import pytest

from oracle import peps_oracle as O
from paper_1611_09467_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_exact_energies.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                Ly, Lx, J2, e = line.split()
                rows.append((int(Ly), int(Lx), float(J2), float(e)))
    return rows


# ------------------------------------------------------------ codec / lattice

def test_bond_counts_and_codec():
    """Bond counts 2L(L-1) NN and 2(L-1)^2 NNN; pack/unpack round trip; popcount N/2."""
    for L in (2, 3, 4, 6, 8, 16):
        h, v = O.nn_bonds(L, L)
        d1, d2 = O.nnn_bonds(L, L)
        assert len(h) + len(v) == 2 * L * (L - 1)
        assert len(d1) + len(d2) == 2 * (L - 1) ** 2
        # NN pairs are at distance 1, NNN at distance sqrt(2), no duplicates
        for i, j in h + v:
            (ri, ci), (rj, cj) = divmod(i, L), divmod(j, L)
            assert abs(ri - rj) + abs(ci - cj) == 1
        for i, j in d1 + d2:
            (ri, ci), (rj, cj) = divmod(i, L), divmod(j, L)
            assert abs(ri - rj) == 1 and abs(ci - cj) == 1
        assert len(set(map(frozenset, h + v + d1 + d2))) == len(h + v + d1 + d2)
    sp = inputs.random_sz0(50, 100, seed=5)
    assert (sp.sum(axis=1) == 50).all()
    packed = inputs.pack_spins(sp)
    assert packed.shape == (50, 2)
    assert (inputs.unpack_spins(packed, 100) == sp).all()
    pc = [sum(bin(int(w)).count("1") for w in row) for row in packed]
    assert pc == [50] * 50


def test_tensor_generator_layout():
    """Edge bonds have dimension one (Eq. 1 text); unit Frobenius norm per site."""
    A = inputs.make_tensors(3, 4, 3, seed=9)
    N = 12
    assert A.shape == (N, 2, 3, 3, 3, 3)
    norms = np.sqrt((A.reshape(N, -1) ** 2).sum(axis=1))
    assert np.allclose(norms, 1.0, atol=1e-14)
    # corner (0,0): only l=0 and u=0 may be non-zero
    assert np.all(A[0, :, 1:] == 0) and np.all(A[0, :, :, :, 1:] == 0)
    # bottom-right corner: r = 0 and d = 0 only
    assert np.all(A[N - 1, :, :, 1:] == 0) and np.all(A[N - 1, :, :, :, :, 1:] == 0)
    # The bias adds 1.0 to A_i[s=0][0][0][0][0] before normalisation.  With
    # raw = unnormalised draws, A = raw/|raw| and Ab = (raw + e0)/|raw + e0|:
    # Ab/A = c elsewhere, Ab0/c - A0 = 1/|raw| and c^2 |raw + e0|^2 = |raw|^2.
    Ab = inputs.make_tensors(3, 4, 3, seed=9, bias_zero_index=True)
    for i in range(N):
        a, b = A[i].reshape(-1), Ab[i].reshape(-1)
        nz = a != 0
        nz[0] = False
        c = b[nz] / a[nz]
        assert np.allclose(c, c[0], rtol=1e-12)
        c = c[0]
        raw_norm = 1.0 / (b[0] / c - a[0])
        assert raw_norm > 0
        assert abs(c * c * (raw_norm ** 2 + 2 * a[0] * raw_norm + 1) - raw_norm ** 2) < 1e-10 * raw_norm ** 2


def test_near_product_generator():
    """Near-product tensors: edge bonds of dimension one, unit norm per site,
    deterministic; the all-zero-bond entries of the two spin components are
    in the ratio sin t : cos t with t in [pi/8, 3pi/8] up to the noise (whose
    expected norm equals the product part's), and the noise is the same keyed
    draw as the i.i.d. recipe scaled by eta / sqrt(d D^4)."""
    Ly, Lx, D = 3, 4, 3
    A = inputs.near_product_tensors(Ly, Lx, D, seed=9)
    N = Ly * Lx
    assert A.shape == (N, 2, D, D, D, D)
    assert np.array_equal(A, inputs.near_product_tensors(Ly, Lx, D, seed=9))
    assert np.allclose(np.sqrt((A.reshape(N, -1) ** 2).sum(axis=1)), 1.0, atol=1e-14)
    assert np.all(A[0, :, 1:] == 0) and np.all(A[0, :, :, :, 1:] == 0)
    assert np.all(A[N - 1, :, :, 1:] == 0) and np.all(A[N - 1, :, :, :, :, 1:] == 0)
    # without noise the tensors are exactly the product state
    P = inputs.near_product_tensors(Ly, Lx, D, seed=9, eta=0.0)
    t = np.arctan2(P[:, 1, 0, 0, 0, 0], P[:, 0, 0, 0, 0, 0])
    assert np.all((t >= np.pi / 8 - 1e-12) & (t <= 3 * np.pi / 8 + 1e-12))
    assert np.allclose(P[:, 0, 0, 0, 0, 0] ** 2 + P[:, 1, 0, 0, 0, 0] ** 2, 1.0)
    rest = P.copy()
    rest[:, :, 0, 0, 0, 0] = 0
    assert np.all(rest == 0)
    # the noise is the keyed i.i.d. draw, scaled (compare before normalisation)
    eta = 0.7
    B = inputs.near_product_tensors(Ly, Lx, D, seed=9, eta=eta)
    G = inputs.make_tensors(Ly, Lx, D, seed=9)   # i.i.d. draw, normalised per site
    for i in range(N):
        b, g = B[i].reshape(-1).copy(), G[i].reshape(-1).copy()
        b[0] = g[0] = 0.0
        b[D ** 4] = g[D ** 4] = 0.0              # the all-zero-bond entry of s = 1
        nz = g != 0
        r = b[nz] / g[nz]
        assert np.allclose(r, r[0], rtol=1e-12)


# ------------------------------------------------------------- P-a: ED pins

def test_ed_2x2_closed_form():
    """2x2 open square: E0 = -2 J1 + J2/2 for J2 <= J1 (textbook)."""
    for J2 in (0.0, 0.25, 0.5):
        e = O.ground_energy(2, 2, 1.0, J2)
        assert abs(e - (-2.0 + J2 / 2)) < 1e-12


def test_ed_4x4_table1():
    """Table I 'Exact' column: 4x4, J2 = 0, -0.57432544 per site."""
    for Ly, Lx, J2, e in _table1():
        if (Ly, Lx) == (4, 4):
            got = O.ground_energy(Ly, Lx, 1.0, J2) / (Ly * Lx)
            assert abs(got - e) < 6e-9


@pytest.mark.slow
def test_ed_4x6_frustrated_table1():
    """Table I: 4x6, J2 = 0.5 (pins the NNN bonds and their coupling), -0.47437906 per site."""
    for Ly, Lx, J2, e in _table1():
        if (Ly, Lx, J2) == (4, 6, 0.5):
            got = O.ground_energy(Ly, Lx, 1.0, J2) / (Ly * Lx)
            assert abs(got - e) < 6e-9


# ------------------------------------------- P-b / P-c: contraction pins

@pytest.mark.parametrize("Ly,Lx,D", [(2, 2, 2), (2, 3, 2), (3, 3, 2), (2, 2, 3)])
def test_exact_contraction_vs_bruteforce(Ly, Lx, D):
    """Transfer-vector contraction equals the explicit sum over all virtual indices (Eq. 1)."""
    A = inputs.make_tensors(Ly, Lx, D, seed=21)
    for k in range(3):
        sp = inputs.random_sz0(1, Ly * Lx, seed=22, first=k)[0] if Ly * Lx % 2 == 0 \
            else np.arange(Ly * Lx) % 2
        T = O.project(A, sp, Ly, Lx)
        a, b = O.contract_exact(T, Ly, Lx), O.contract_bruteforce(T, Ly, Lx)
        assert abs(a - b) <= 1e-13 * max(abs(b), 1e-300) + 1e-300


@pytest.mark.parametrize("Ly,Lx,D,Dc", [(4, 4, 2, 4), (3, 4, 2, 4), (4, 3, 3, 9), (5, 4, 2, 4)])
def test_boundary_mps_exact_regime(Ly, Lx, D, Dc):
    """Dc >= D^floor(Lx/2): boundary MPS equals exact contraction, top-down and bottom-up."""
    A = inputs.make_tensors(Ly, Lx, D, seed=31)
    sp = inputs.random_sz0(6, Ly * Lx, seed=32)
    for s in sp:
        T = O.project(A, s, Ly, Lx)
        w = O.contract_exact(T, Ly, Lx)
        la, sg = O.amplitude(A, s, Ly, Lx, Dc)
        assert sg == np.sign(w)
        assert abs(la - math.log(abs(w))) < 1e-12
        mps, ls = O.bottom_envs(T, Ly, Lx, Dc)[0]
        v = O.close_chain(mps) * math.exp(ls)
        assert abs(v - w) <= 1e-12 * abs(w)


def test_boundary_mps_truncates_and_converges_with_dc():
    """P-l: |psi_Dc - psi_exact| shrinks as Dc grows on 6x6 D=2 (cf. the Dc study, Appendix)."""
    Ly = Lx = 6
    A = inputs.make_tensors(Ly, Lx, 2, seed=41)
    sp = inputs.random_sz0(8, 36, seed=42)
    errs = {Dc: [] for Dc in (2, 3, 4, 8)}
    for s in sp:
        w = O.contract_exact(O.project(A, s, Ly, Lx), Ly, Lx)
        for Dc in errs:
            la, sg = O.amplitude(A, s, Ly, Lx, Dc)
            errs[Dc].append(abs(sg * math.exp(la) - w) / abs(w))
    med = {Dc: float(np.median(v)) for Dc, v in errs.items()}
    assert med[2] > med[3] > med[4]
    assert med[8] < 1e-12          # 8 = D^3: exact
    assert med[2] > 1e-6           # truncation really happens


def test_linearity_in_each_tensor():
    """P-e: psi(c * A_i) = c * psi(A), exact and truncated (SVD truncation is scale-free)."""
    Ly, Lx, D = 6, 6, 3
    A = inputs.make_tensors(Ly, Lx, D, seed=51)
    s = inputs.random_sz0(1, 36, seed=52)[0]
    for Dc in (4, 9):
        la, sg = O.amplitude(A, s, Ly, Lx, Dc)
        for i, c in ((0, 3.0), (14, -0.5), (35, 7.25)):
            B = A.copy()
            B[i] *= c
            lb, sb = O.amplitude(B, s, Ly, Lx, Dc)
            assert sb == sg * np.sign(c)
            assert abs(lb - la - math.log(abs(c))) < 1e-11


def _random_orthogonal(n, rng):
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    return q * np.sign(np.diag(r))


def _gauge(A, Ly, Lx, D, rng, orthogonal=True):
    """Insert G G^-1 on every internal bond (horizontal and vertical)."""
    B = A.copy()
    for r in range(Ly):
        for c in range(Lx):
            i = r * Lx + c
            if c + 1 < Lx:
                G = _random_orthogonal(D, rng) if orthogonal else rng.standard_normal((D, D)) + 2 * np.eye(D)
                Gi = np.linalg.inv(G)
                B[i] = np.einsum("slrud,rx->slxud", B[i], G)
                B[i + 1] = np.einsum("xl,slrud->sxrud", Gi, B[i + 1])
            if r + 1 < Ly:
                G = _random_orthogonal(D, rng) if orthogonal else rng.standard_normal((D, D)) + 2 * np.eye(D)
                Gi = np.linalg.inv(G)
                B[i] = np.einsum("slrud,dx->slrux", B[i], G)
                B[i + Lx] = np.einsum("xu,slrud->slrxd", Gi, B[i + Lx])
    return B


def test_gauge_invariance():
    """P-e: G G^-1 on every bond leaves exact psi unchanged; orthogonal G leaves the
    truncated boundary-MPS psi and E_loc unchanged too (the kept subspaces rotate with G)."""
    rng = np.random.default_rng(61)
    Ly = Lx = 5
    D = 3
    A = inputs.make_tensors(Ly, Lx, D, seed=62)
    A = A * inputs.edge_mask(Ly, Lx, D)
    s = np.append(inputs.random_sz0(1, 24, seed=63)[0], 0)   # 25 sites, amplitude only
    Bn = _gauge(A, Ly, Lx, D, rng, orthogonal=False)
    we = O.contract_exact(O.project(A, s, Ly, Lx), Ly, Lx)
    wg = O.contract_exact(O.project(Bn, s, Ly, Lx), Ly, Lx)
    assert abs(we - wg) < 1e-11 * abs(we)
    Bo = _gauge(A, Ly, Lx, D, rng, orthogonal=True)
    for Dc in (3, 5):
        la, sa = O.amplitude(A, s, Ly, Lx, Dc)
        lb, sb = O.amplitude(Bo, s, Ly, Lx, Dc)
        assert sa == sb and abs(la - lb) < 1e-10
    Ly = Lx = 4
    A = inputs.make_tensors(Ly, Lx, 2, seed=64)
    Bo = _gauge(A, Ly, Lx, 2, rng, orthogonal=True)
    s = inputs.random_sz0(1, 16, seed=65)[0]
    ea = O.evaluate(A, s, Ly, Lx, 3, 1.0, 0.5)
    eb = O.evaluate(Bo, s, Ly, Lx, 3, 1.0, 0.5)
    assert abs(ea.eloc - eb.eloc) < 1e-9 * max(1.0, abs(ea.eloc))


# -------------------------------------------------- P-f: product state

def test_product_state_closed_forms():
    """P-f: D = 1: psi = prod t_i(s_i), O_i = 1/t_i(s_i), ratio = t_i(s_j) t_j(s_i) / (t_i(s_i) t_j(s_j))."""
    Ly, Lx = 4, 4
    N = 16
    rng = np.random.default_rng(71)
    t = rng.uniform(0.3, 1.5, size=(N, 2)) * rng.choice([-1, 1], size=(N, 2))
    A = t.reshape(N, 2, 1, 1, 1, 1)
    J1, J2 = 1.0, 0.5
    for s in inputs.random_sz0(4, N, seed=72):
        ev = O.evaluate(A, s, Ly, Lx, 2, J1, J2)
        psi = np.prod([t[i, s[i]] for i in range(N)])
        assert abs(ev.logabs - math.log(abs(psi))) < 1e-12 and ev.sign == np.sign(psi)
        e = 0.0
        for i, j, J, _ in O.all_bonds(Ly, Lx, J1, J2):
            if s[i] == s[j]:
                e += J / 4
            else:
                e += -J / 4 + J / 2 * t[i, s[j]] * t[j, s[i]] / (t[i, s[i]] * t[j, s[j]])
        assert abs(ev.eloc - e) < 1e-12 * max(1, abs(e))
        for i in range(N):
            assert abs(ev.O[i].reshape(-1)[0] - 1.0 / t[i, s[i]]) < 1e-12 / abs(t[i, s[i]])


# -------------------------------- P-d: E_loc against the exact wavefunction

@pytest.mark.parametrize("Ly,Lx,D,Dc,J2", [(4, 4, 2, 4, 0.5), (3, 4, 2, 4, 0.5), (4, 3, 2, 8, 0.0)])
def test_local_energy_equals_H_psi_over_psi(Ly, Lx, D, Dc, J2):
    """P-d: in the exact regime E_loc(S) = (H psi)(S) / psi(S) with psi the exact
    Sz=0 wavefunction and H the sparse ED Hamiltonian (pinned by Table I); the
    energy expectation is above the ED ground energy (variational bound)."""
    A = inputs.make_tensors(Ly, Lx, D, seed=81)
    basis, psi = O.exact_sz0_wavefunction(A, Ly, Lx)
    H, hb = O.hamiltonian_sz0(Ly, Lx, 1.0, J2)
    assert (hb == basis).all()
    Hpsi = H @ psi
    N = Ly * Lx
    rng = np.random.default_rng(82)
    for k in rng.choice(len(basis), size=6, replace=False):
        s = [(int(basis[k]) >> i) & 1 for i in range(N)]
        ev = O.evaluate(A, s, Ly, Lx, Dc, 1.0, J2, want_O=False)
        assert abs(ev.eloc - Hpsi[k] / psi[k]) < 1e-9 * max(1.0, abs(ev.eloc))
    e_var = psi @ Hpsi / (psi @ psi)
    assert e_var >= O.ground_energy(Ly, Lx, 1.0, J2) - 1e-10


# ----------------------------------- P-g / P-h: log-derivatives

def test_log_derivative_vs_finite_differences():
    """P-g: exact regime, Delta = B/W equals the central difference of ln|psi|."""
    Ly, Lx, D, Dc = 4, 4, 2, 4
    A = inputs.make_tensors(Ly, Lx, D, seed=91)
    s = inputs.random_sz0(1, 16, seed=92)[0]
    ev = O.evaluate(A, s, Ly, Lx, Dc, 1.0, 0.5)
    rng = np.random.default_rng(93)
    h = 1e-5
    mask = inputs.edge_mask(Ly, Lx, D)[:, 0]
    for _ in range(12):
        i = int(rng.integers(16))
        idx = tuple(int(x) for x in np.argwhere(mask[i])[rng.integers(mask[i].sum())])
        Ap, Am = A.copy(), A.copy()
        Ap[(i, s[i]) + idx] += h
        Am[(i, s[i]) + idx] -= h
        fd = (O.amplitude_exact(Ap, s, Ly, Lx)[0] - O.amplitude_exact(Am, s, Ly, Lx)[0]) / (2 * h)
        assert abs(ev.O[(i,) + idx] - fd) < 1e-6 * max(1.0, abs(fd))
        # the other spin block does not enter psi(S)
        Ap = A.copy()
        Ap[(i, 1 - s[i]) + idx] += 0.3
        assert O.amplitude_exact(Ap, s, Ly, Lx)[0] == O.amplitude_exact(A, s, Ly, Lx)[0]


def test_euler_identity_truncated():
    """P-h: psi is linear in T_i, so sum_lrud T_i * Delta_i = 1 per site, in any regime."""
    Ly, Lx, D, Dc = 6, 6, 3, 4
    A = inputs.make_tensors(Ly, Lx, D, seed=101)
    s = inputs.random_sz0(1, 36, seed=102)[0]
    ev = O.evaluate(A, s, Ly, Lx, Dc, 1.0, 0.5)
    for i in range(36):
        assert abs(np.sum(A[i, s[i]] * ev.O[i]) - 1.0) < 1e-10


# -------------------------------------------- P-i: gradient estimator

def test_gradient_estimator_equals_energy_derivative():
    """P-i: with every Sz=0 configuration weighted by W^2/Z, 2(<E O> - <E><O>) equals the
    finite-difference derivative of <psi|H|psi>/<psi|psi> (pins the 2 and the covariance form)."""
    Ly, Lx, D, Dc, J2 = 2, 4, 2, 4, 0.5
    N = Ly * Lx
    A = inputs.make_tensors(Ly, Lx, D, seed=111)
    basis, _ = O.exact_sz0_wavefunction(A, Ly, Lx)
    H, _ = O.hamiltonian_sz0(Ly, Lx, 1.0, J2)
    spins = [[(int(x) >> i) & 1 for i in range(N)] for x in basis]
    evals = [O.evaluate(A, s, Ly, Lx, Dc, 1.0, J2) for s in spins]
    w = np.array([math.exp(2 * ev.logabs) for ev in evals])
    e_site, g, cov, n = O.gradient(evals, spins, N, D, weights=w)
    assert n == len(basis)

    def energy(B):
        _, p = O.exact_sz0_wavefunction(B, Ly, Lx)
        return p @ (H @ p) / (p @ p)

    assert abs(e_site * N - energy(A)) < 1e-10
    mask = inputs.edge_mask(Ly, Lx, D)[:, 0].reshape(N, -1)
    rng = np.random.default_rng(112)
    h = 1e-5
    for _ in range(8):
        i = int(rng.integers(N))
        sblk = int(rng.integers(2))
        p = int(rng.choice(np.nonzero(mask[i])[0]))
        Ap, Am = A.copy(), A.copy()
        Ap.reshape(N, 2, -1)[i, sblk, p] += h
        Am.reshape(N, 2, -1)[i, sblk, p] -= h
        fd = (energy(Ap) - energy(Am)) / (2 * h)
        assert abs(g[i, sblk, p] - fd) < 1e-6 * max(1.0, abs(fd))
    assert np.allclose(cov, g / 2)


# ------------------------------------------------- P-k: Metropolis sampler

def test_sampler_uniform_is_splitmix64():
    """The sampler's keyed uniform is SplitMix64's published output function.

    Known value: SplitMix64 seeded with 0 first returns 0xE220A8397B1DCDAF
    (state 0 + golden gamma, then the output mix)."""
    assert O._mix64(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF
    u = [O.sampler_uniform(1, c, 0, 0) for c in range(2000)]
    assert 0.0 <= min(u) and max(u) < 1.0
    assert abs(np.mean(u) - 0.5) < 0.03


def test_sampler_stationary_distribution_chi_square():
    """P-k: in the exact regime the sweep samples |P0 psi|^2 / Z (chi-square on 2x3)."""
    Ly, Lx, D, Dc = 2, 3, 2, 4
    N = 6
    A = inputs.make_tensors(Ly, Lx, D, seed=121)
    basis, psi = O.exact_sz0_wavefunction(A, Ly, Lx)
    p = psi ** 2 / np.sum(psi ** 2)
    nchains, nsweeps = 600, 6
    starts = inputs.random_sz0(nchains, N, seed=122)
    counts = np.zeros(len(basis))
    index = {int(x): k for k, x in enumerate(basis)}
    acc = 0
    for ch in range(nchains):
        s = starts[ch]
        for sw in range(nsweeps):
            s, a = O.mc_sweep(A, s, Ly, Lx, Dc, seed=7, chain=ch, sweep=sw)
            acc += a
        assert s.sum() == N // 2
        counts[index[sum(int(s[i]) << i for i in range(N))]] += 1
    assert acc > 0
    exp = p * nchains
    keep = exp > 5
    chi2 = float(np.sum((counts[keep] - exp[keep]) ** 2 / exp[keep]))
    dof = int(keep.sum()) - 1
    # 99.9% quantile of chi-square with dof <= 19 is below 44
    assert chi2 < 44.0, (chi2, dof)
