"""FP64 oracle of the simple-update initialiser (Sec. III, computational details).

TEST INFRASTRUCTURE ONLY, like peps_oracle: only the tests, the smoke entry
point and bench.py's CPU legs may import it; it shares no code with the CUDA
path.

The paper starts its gradient optimisation from tensors found by imaginary
time evolution with the simple update (SU): the Hamiltonian is split into
groups of mutually commuting bond terms, exp(-dtau H) is Trotter-expanded
into two-site gates, and each gate is applied to its bond and the bond is
cut back to D by an SVD, with QR decompositions isolating the bond so the
cost is O(D^5).  dtau = 0.01 until the tensors stop changing (relative change
below 1e-6), then dtau = 0.001.

Readings of what the paper leaves open (each in the design notes):
* State: site tensors Gamma_i[s][l][r][u][d] and a bond weight vector lam_b
  (diagonal, length D) on every bond; the PEPS of Eq. 1 is
  A_i = Gamma_i times sqrt(lam) on each of its bonds.
* A gate on bond (i, j): the weights of i's and j's other bonds are absorbed
  into Gamma_i and Gamma_j, and the bond's own weight into Gamma_i; each
  tensor is split by a thin QR into Q (its outer legs) and R (spin and bond);
  Theta = gate applied to R_i R_j; SVD of Theta; the D largest singular
  values (normalised to unit 2-norm) become the new weight, U and V^T the new
  R's; the outer weights are divided out again (zero weights leave zero).
* One Trotter step: horizontal bonds at even columns, horizontal at odd
  columns, vertical at even rows, vertical at odd rows (each group has no
  shared site), first order.  With J2 != 0 the next-nearest gates follow:
  a diagonal pair (i, k) sharing neighbour j is done as SWAP(i, j), the gate
  on (j, k), SWAP(i, j), with a truncation after each two-site update.
* Entries past an open edge are set back to zero after every update.
* Gate: exp(-dtau J S_i.S_j) = e^{-dtau J/4} P_triplet + e^{3 dtau J/4} P_singlet
  (S.S is 1/4 on the triplet and -3/4 on the singlet).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import peps_oracle as O

# spin basis of a pair: index 2 s_i + s_j, s = 0 is S^z = +1/2
_SINGLET = np.array([0.0, 1.0, -1.0, 0.0]) / math.sqrt(2.0)
SWAP = np.eye(4)[[0, 2, 1, 3]]


def heisenberg_pair():
    """S_i.S_j on two spins 1/2 in the basis 2 s_i + s_j (S = sigma / 2)."""
    h = np.zeros((4, 4))
    for a in range(4):
        si, sj = a >> 1, a & 1
        h[a, a] = 0.25 if si == sj else -0.25
        if si != sj:
            h[(sj << 1) | si, a] = 0.5
    return h


def gate(J, dtau):
    """exp(-dtau J S_i.S_j) in the basis 2 s_i + s_j, from the two projectors."""
    Ps = np.outer(_SINGLET, _SINGLET)
    Pt = np.eye(4) - Ps
    return math.exp(-dtau * J / 4.0) * Pt + math.exp(3.0 * dtau * J / 4.0) * Ps


def init_state(Ly, Lx, D, seed):
    """Gamma = the seeded tensors (padded [N][2][D^4]), every weight = 1 on its
    true dimension (D inside the lattice)."""
    from paper_1611_09467_gb300 import inputs
    Gam = inputs.make_tensors(Ly, Lx, D, seed).copy()
    h, v = O.nn_bonds(Ly, Lx)
    lam = {b: np.ones(D) for b in h + v}
    return Gam, lam


def _bonds_of(i, Ly, Lx):
    """{leg: bond} of site i: leg 0 l, 1 r, 2 u, 3 d; bonds as sorted (a, b) pairs."""
    r, c = divmod(i, Lx)
    out = {}
    if c > 0:
        out[0] = (i - 1, i)
    if c < Lx - 1:
        out[1] = (i, i + 1)
    if r > 0:
        out[2] = (i - Lx, i)
    if r < Ly - 1:
        out[3] = (i, i + Lx)
    return out


def _scale_leg(T, leg, w):
    """T[s, l, r, u, d] times w on leg `leg` (0..3)."""
    shape = [1, 1, 1, 1, 1]
    shape[1 + leg] = len(w)
    return T * w.reshape(shape)


def bond_update(Gam, lam, i, j, G, Ly, Lx, D):
    """Apply the two-site gate G (basis 2 s_i + s_j) to bond (i, j), i the left
    or upper site, and cut the bond back to D (in place on Gam and lam)."""
    bi, bj = _bonds_of(i, Ly, Lx), _bonds_of(j, Ly, Lx)
    horizontal = j == i + 1
    li, lj = (1, 0) if horizontal else (3, 2)        # the shared legs of i and j
    bond = (i, j)
    Ti, Tj = Gam[i].copy(), Gam[j].copy()            # [s, l, r, u, d]
    for leg, b in bi.items():
        if leg != li:
            Ti = _scale_leg(Ti, leg, lam[b])
    for leg, b in bj.items():
        if leg != lj:
            Tj = _scale_leg(Tj, leg, lam[b])
    Ti = _scale_leg(Ti, li, lam[bond])
    # outer legs first, then (s, shared leg)
    oi = [1 + x for x in range(4) if x != li]
    oj = [1 + x for x in range(4) if x != lj]
    Mi = Ti.transpose(oi + [0, 1 + li])              # [o1, o2, o3, s, x]
    Mj = Tj.transpose(oj + [0, 1 + lj])
    osh_i, osh_j = Mi.shape[:3], Mj.shape[:3]
    Qi, Ri = np.linalg.qr(Mi.reshape(-1, 2 * D))     # Ri [ki, (s, x)]
    Qj, Rj = np.linalg.qr(Mj.reshape(-1, 2 * D))
    ki, kj = Ri.shape[0], Rj.shape[0]
    Ri = Ri.reshape(ki, 2, D)
    Rj = Rj.reshape(kj, 2, D)
    # Theta[ki, s_i', s_j', kj] = sum G[s_i' s_j', s_i s_j] Ri[ki, s_i, x] Rj[kj, s_j, x]
    P = np.einsum("aix,bjx->aibj", Ri, Rj)                     # [ki, s_i, kj, s_j]
    G4 = G.reshape(2, 2, 2, 2)                                 # [s_i', s_j', s_i, s_j]
    Th = np.einsum("pqij,aibj->apqb", G4, P)                   # [ki, s_i', s_j', kj]
    U, sv, Vt = np.linalg.svd(Th.reshape(ki * 2, 2 * kj), full_matrices=False)
    K = min(D, len(sv))
    s = sv[:K]
    nrm = np.linalg.norm(s)
    new = np.zeros(D)
    new[:K] = s / nrm if nrm > 0 else s
    lam[bond] = new
    Ri2 = np.zeros((ki, 2, D))
    Ri2[:, :, :K] = U[:, :K].reshape(ki, 2, K)
    Rj2 = np.zeros((kj, 2, D))
    Rj2[:, :, :K] = Vt[:K].reshape(K, 2, kj).transpose(2, 1, 0)
    Ni = (Qi @ Ri2.reshape(ki, 2 * D)).reshape(*osh_i, 2, D)
    Nj = (Qj @ Rj2.reshape(kj, 2 * D)).reshape(*osh_j, 2, D)
    # back to [s, l, r, u, d]
    inv_i = np.argsort(oi + [0, 1 + li])
    inv_j = np.argsort(oj + [0, 1 + lj])
    Ti, Tj = Ni.transpose(inv_i), Nj.transpose(inv_j)
    for leg, b in bi.items():
        if leg != li:
            Ti = _scale_leg(Ti, leg, _inv(lam[b]))
    for leg, b in bj.items():
        if leg != lj:
            Tj = _scale_leg(Tj, leg, _inv(lam[b]))
    # entries past an open edge stay zero (a rank-deficient split may leave
    # rounding-sized values there)
    from paper_1611_09467_gb300 import inputs
    mask = inputs.edge_mask(Ly, Lx, D)
    Gam[i], Gam[j] = Ti * mask[i], Tj * mask[j]


def _inv(w):
    out = np.zeros_like(w)
    nz = w != 0
    out[nz] = 1.0 / w[nz]
    return out


def bond_groups(Ly, Lx):
    """The four groups of nearest-neighbour bonds without a shared site, in
    the Trotter order: horizontal at even / odd columns, vertical at even /
    odd rows."""
    h, v = O.nn_bonds(Ly, Lx)
    he = [(i, j) for i, j in h if (i % Lx) % 2 == 0]
    ho = [(i, j) for i, j in h if (i % Lx) % 2 == 1]
    ve = [(i, j) for i, j in v if (i // Lx) % 2 == 0]
    vo = [(i, j) for i, j in v if (i // Lx) % 2 == 1]
    return [he, ho, ve, vo]


def nnn_routes(Ly, Lx):
    """Next-nearest pairs as (i, j, k): SWAP on (i, j) brings s_i next to k.
    Diagonal (r,c)-(r+1,c+1) goes through (r,c+1); anti-diagonal
    (r,c+1)-(r+1,c) through (r,c).  Each route's swap is a horizontal bond
    (i, j) with i < j or a vertical one; grouped so no two routes of a group
    share a site: one group per (kind, column parity, row parity)."""
    groups = {}
    for r in range(Ly - 1):
        for c in range(Lx - 1):
            a = r * Lx + c
            groups.setdefault(("d1", c % 2, r % 2), []).append((a, a + 1, a + 1 + Lx))    # (r,c) -> (r,c+1) -> (r+1,c+1)
            groups.setdefault(("d2", c % 2, r % 2), []).append((a + 1, a, a + Lx))        # (r,c+1) -> (r,c) -> (r+1,c)
    return [groups[k] for k in sorted(groups)]


def _ordered(a, b):
    return (a, b) if a < b else (b, a)


def _update(Gam, lam, a, b, G, Ly, Lx, D):
    """bond_update on the pair {a, b} in either order (G in the basis 2 s_a + s_b)."""
    if a < b:
        bond_update(Gam, lam, a, b, G, Ly, Lx, D)
    else:
        Gs = SWAP @ G @ SWAP                      # the same gate in the basis 2 s_b + s_a
        bond_update(Gam, lam, b, a, Gs, Ly, Lx, D)


def trotter_step(Gam, lam, Ly, Lx, J1, J2, dtau, D):
    """One first-order Trotter step of exp(-dtau H) by simple updates."""
    G1 = gate(J1, dtau)
    for group in bond_groups(Ly, Lx):
        for i, j in group:
            bond_update(Gam, lam, i, j, G1, Ly, Lx, D)
    if J2 != 0.0:
        G2 = gate(J2, dtau)
        for group in nnn_routes(Ly, Lx):
            for i, j, k in group:
                _update(Gam, lam, i, j, SWAP, Ly, Lx, D)
                _update(Gam, lam, j, k, G2, Ly, Lx, D)
                _update(Gam, lam, i, j, SWAP, Ly, Lx, D)


def to_peps(Gam, lam, Ly, Lx):
    """A_i = Gamma_i times sqrt(lam) on each bond (Eq. 1 tensors), each site
    scaled to unit Frobenius norm."""
    A = Gam.copy()
    for i in range(Ly * Lx):
        for leg, b in _bonds_of(i, Ly, Lx).items():
            A[i] = _scale_leg(A[i], leg, np.sqrt(lam[b]))
        n = np.linalg.norm(A[i])
        if n > 0:
            A[i] /= n
    return A


def evolve(Gam, lam, Ly, Lx, J1, J2, D, dtau, steps):
    """`steps` Trotter steps at time step dtau; returns the largest relative
    change of A over the last step (the paper's convergence measure)."""
    change = math.inf
    for _ in range(steps):
        A0 = to_peps(Gam, lam, Ly, Lx)
        trotter_step(Gam, lam, Ly, Lx, J1, J2, dtau, D)
        A1 = to_peps(Gam, lam, Ly, Lx)
        change = float(np.max(np.abs(A1 - A0)) / max(np.max(np.abs(A0)), 1e-300))
    return change
