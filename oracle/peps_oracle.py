"""FP64 CPU oracle of the PEPS sampling hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  It
shares no code with the CUDA path; its only input dependency is the seeded
generator module, which holds none of the method's arithmetic.

Everything here is plain numpy in float64, written for a reader to check it
against the paper (Liu, Dong, Han, Guo, He, "Gradient optimization of finite
projected entangled pair states", arXiv:1611.09467):

* Eq. 1 (Sec. II): psi(S) = W(S) = Tr prod_i A_i^{s_i}, single-layer network
  at fixed S (Fig. 1c), virtual bonds D, open edges of dimension one.
* Fig. 1(d) and Sec. II: boundary-MPS contraction with cut-off Dc.  The paper
  does not name its truncation scheme; this oracle uses the alternating
  zip-up with SVD truncation described in ``absorb_row``.
* Sec. II energy estimator: E = (1/Z) sum_S W^2(S) E(S) with
  E(S) = sum_S' W(S')/W(S) <S'|H|S>.
* Sec. IV Hamiltonian: H = J1 sum_<ij> S_i.S_j + J2 sum_<<ij>> S_i.S_j, spin 1/2.
* Sec. II gradient: dE/dA = 2<Delta E> - 2<Delta><E>, Delta = B/W, B the
  environment of site m.
* Sec. III gradient optimisation: A(n+1) = A(n) - p dt(n) sign(dE/dA), p
  uniform in [0, 1) per element.

Readings of points the paper leaves open (each listed in the design notes):
zip-up truncation, alternating absorption direction, ratios and Delta taken
with the same sandwich's W, NNN bonds = both plaquette diagonals, canonical
bond order, S^z = 0 sector, plain sample means, Metropolis move set.
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------- lattice

def site(r: int, c: int, Lx: int) -> int:
    return r * Lx + c


def nn_bonds(Ly: int, Lx: int):
    """Nearest-neighbour pairs (Sec. IV, <i,j>): horizontal row-major, then vertical row-major."""
    h = [(site(r, c, Lx), site(r, c + 1, Lx)) for r in range(Ly) for c in range(Lx - 1)]
    v = [(site(r, c, Lx), site(r + 1, c, Lx)) for r in range(Ly - 1) for c in range(Lx)]
    return h, v


def nnn_bonds(Ly: int, Lx: int):
    """Next-nearest-neighbour pairs (Sec. IV, <<i,j>>) on the open lattice.

    Both diagonals of every plaquette, each pair once, no wrap-around:
    first (r,c)-(r+1,c+1) row-major, then (r,c+1)-(r+1,c) row-major.
    """
    d1 = [(site(r, c, Lx), site(r + 1, c + 1, Lx)) for r in range(Ly - 1) for c in range(Lx - 1)]
    d2 = [(site(r, c + 1, Lx), site(r + 1, c, Lx)) for r in range(Ly - 1) for c in range(Lx - 1)]
    return d1, d2


def all_bonds(Ly: int, Lx: int, J1: float, J2: float):
    """Canonical bond list [(i, j, J, kind)], kind in {'h', 'v', 'd1', 'd2'}."""
    h, v = nn_bonds(Ly, Lx)
    d1, d2 = nnn_bonds(Ly, Lx)
    out = [(i, j, J1, "h") for i, j in h] + [(i, j, J1, "v") for i, j in v]
    out += [(i, j, J2, "d1") for i, j in d1] + [(i, j, J2, "d2") for i, j in d2]
    return out


def site_dims(Ly: int, Lx: int, D: int):
    """True (l, r, u, d) dimensions per site: D inside, 1 on open edges (Eq. 1 text)."""
    dims = []
    for r in range(Ly):
        for c in range(Lx):
            dims.append((1 if c == 0 else D, 1 if c == Lx - 1 else D,
                         1 if r == 0 else D, 1 if r == Ly - 1 else D))
    return dims


def project(A: np.ndarray, spins, Ly: int, Lx: int):
    """Single-layer network at fixed S (Fig. 1c): T_i = A_i^{s_i}, true dims, index order (l, r, u, d).

    A is the padded array [N][d][D][D][D][D]; the oracle slices it to the true
    dimensions instead of carrying the zero padding.
    """
    D = A.shape[2]
    dims = site_dims(Ly, Lx, D)
    T = []
    for i in range(Ly * Lx):
        dl, dr, du, dd = dims[i]
        T.append(np.array(A[i, int(spins[i]), :dl, :dr, :du, :dd], dtype=np.float64))
    return T


def rows_of(T, Ly: int, Lx: int):
    return [T[r * Lx:(r + 1) * Lx] for r in range(Ly)]


# ------------------------------------------------- exact contraction (pins)

def contract_exact(T, Ly: int, Lx: int) -> float:
    """Exact W(S) (Eq. 1 'Tr'): a transfer vector over the down bonds, row by row, no truncation."""
    v = np.ones((1,) * Lx)
    for r in range(Ly):
        # W axes: new down bonds of columns < c, horizontal bond h, old up bonds of columns >= c
        W = v.reshape((1,) + v.shape)
        for c in range(Lx):
            Tc = T[r * Lx + c]                       # [l, r, u, d]
            W = np.tensordot(W, Tc, axes=([c, c + 1], [0, 2]))
            # remaining: new_0..new_{c-1}, old_{c+1}.., then (r', d)
            W = np.moveaxis(W, [-1, -2], [c, c + 1])  # d -> position c, r' -> c+1
        v = W.reshape(W.shape[:Lx])
    return float(v.reshape(-1)[0])


def contract_bruteforce(T, Ly: int, Lx: int) -> float:
    """Eq. 1 summed explicitly over every assignment of every virtual bond (tiny lattices only)."""
    import itertools
    bonds = []   # (site_a, axis_a, site_b, axis_b, dim)
    for r in range(Ly):
        for c in range(Lx):
            i = r * Lx + c
            if c + 1 < Lx:
                bonds.append((i, 1, i + 1, 0, T[i].shape[1]))
            if r + 1 < Ly:
                bonds.append((i, 3, i + Lx, 2, T[i].shape[3]))
    total = 0.0
    for assign in itertools.product(*[range(b[4]) for b in bonds]):
        idx = [[0, 0, 0, 0] for _ in range(Ly * Lx)]
        for (ia, xa, ib, xb, _), val in zip(bonds, assign):
            idx[ia][xa] = val
            idx[ib][xb] = val
        term = 1.0
        for i in range(Ly * Lx):
            term *= T[i][tuple(idx[i])]
        total += term
    return total


# -------------------------------------------- boundary MPS (Fig. 1d, Dc)

def absorb_row(mps, Trow, Dc: int, left_to_right: bool, perturb=None):
    """Absorb one row of the single-layer network into a boundary MPS, truncating to Dc.

    ``mps[c]`` is [a, p, b] (left bond, physical index facing the row, right
    bond); ``Trow[c]`` is [l, r, in, out] where ``in`` contracts with p.
    Zip-up: a carry tensor moves along the row; at every column the
    two-column block X is split by an SVD and only the K = min(Dc, rows,
    cols) largest singular values are kept (zero ones included).
    Left-to-right keeps the left singular vectors as the new tensor (a left
    isometry) and carries diag(s) V^T; right-to-left mirrors this.  The
    last tensor takes the rest; it is divided by its Frobenius norm n (the
    norm of the whole MPS, since the others are isometries) and ln n is
    returned.  Returns (new_mps, ln n); n == 0 gives ln n = -inf.

    ``perturb`` (diagnostic, default None) is a callable applied to each block
    X before its SVD; the tests use it to measure how strongly the truncated
    result reacts to rounding-sized changes of X (conditioning of the cut).
    """
    L = len(Trow)
    out = [None] * L
    if left_to_right:
        C = np.ones((1, 1, 1))                        # [k, a, l]
        for c in range(L):
            Y = np.tensordot(C, mps[c], axes=([1], [0]))          # [k, l, i, b]
            X = np.tensordot(Y, Trow[c], axes=([1, 2], [0, 2]))   # [k, b, r, o]
            X = X.transpose(0, 3, 1, 2)                           # [k, o, b, r]
            k, o, b, rr = X.shape
            if perturb is not None:
                X = perturb(X)
            if c < L - 1:
                U, s, Vt = np.linalg.svd(X.reshape(k * o, b * rr), full_matrices=False)
                K = min(Dc, k * o, b * rr)
                out[c] = U[:, :K].reshape(k, o, K)
                C = (s[:K, None] * Vt[:K]).reshape(K, b, rr)
            else:
                out[c] = X.reshape(k, o, b * rr)
        last = L - 1
    else:
        C = np.ones((1, 1, 1))                        # [b, r, k]
        for c in reversed(range(L)):
            Y = np.tensordot(mps[c], C, axes=([2], [0]))          # [a, i, r, k]
            X = np.tensordot(Y, Trow[c], axes=([1, 2], [2, 1]))   # [a, k, l, o]
            X = X.transpose(0, 2, 3, 1)                           # [a, l, o, k]
            a, l, o, k = X.shape
            if perturb is not None:
                X = perturb(X)
            if c > 0:
                U, s, Vt = np.linalg.svd(X.reshape(a * l, o * k), full_matrices=False)
                K = min(Dc, a * l, o * k)
                out[c] = Vt[:K].reshape(K, o, k)
                C = (U[:, :K] * s[None, :K]).reshape(a, l, K)
            else:
                out[c] = X.reshape(a * l, o, k)
        last = 0
    n = float(np.linalg.norm(out[last]))
    if n == 0.0:
        return out, -math.inf
    out[last] = out[last] / n
    return out, math.log(n)


def fit_site(F, Mu, T, G):
    """P[a', d, b'] = sum F[a,l,a'] Mu[a,u,b] T[l,r,u,d] G[b,r,b']: the
    derivative of <P|Mu T> with respect to the candidate tensor at one column
    (its environment in the overlap network)."""
    X = np.tensordot(F, Mu, axes=([0], [0]))            # [l, a', u, b]
    X = np.tensordot(X, T, axes=([0, 2], [0, 2]))       # [a', b, r, d]
    return np.tensordot(X, G, axes=([1, 2], [0, 1]))   # [a', d, b']


def absorb_row_fit(mps, Trow, Dc, left_to_right, sweeps):
    """Absorb one row with the variational-fit truncation (the boundary-MPS
    method of Sec. II by variational compression): start from the zip-up
    result of `absorb_row`, then `sweeps` one-site ALS sweeps that maximise
    <P|Phi> over the candidate MPS P at fixed bond dimensions, Phi = the row
    applied to `mps`.  The zip-up leaves P in mixed canonical form with the
    centre at the last column it visited; each sweep runs from that end to
    the other and back, every column set to its environment in the overlap
    (fit_site) and re-orthonormalised by a QR (left-isometric, moving right)
    or an LQ (right-isometric, moving left), the triangular factor dropped
    (the next column is recomputed from its environment).  The centre's
    Frobenius norm n is divided out and ln n returned, as absorb_row.
    ``Trow[c]`` is [l, r, in, out] as in absorb_row."""
    P, ln0 = absorb_row(mps, Trow, Dc, left_to_right)
    if ln0 == -math.inf or sweeps == 0:
        return P, ln0
    L = len(Trow)
    # the zip-up divided the norm out of its last tensor; restore it so the
    # centre carries the scale while sweeping
    last = L - 1 if left_to_right else 0
    P[last] = P[last] * math.exp(ln0)
    Tz = [t.transpose(0, 1, 2, 3) for t in Trow]           # [l, r, in, out]

    def left_env(c):          # F_{c-1}[a, l, a'] of columns < c
        F = np.ones((1, 1, 1))
        for k in range(c):
            F = col1_left(F, mps[k], Tz[k], P[k])
        return F

    def right_env(c):         # G_{c+1}[b, r, b'] of columns > c
        G = np.ones((1, 1, 1))
        for k in reversed(range(c + 1, L)):
            G = col1_right(G, mps[k], Tz[k], P[k])
        return G

    order_rl = list(reversed(range(L)))
    order_lr = list(range(L))
    passes = []
    for _ in range(sweeps):
        passes += [order_rl, order_lr] if left_to_right else [order_lr, order_rl]
    centre = last
    for cols in passes:
        moving_left = cols[0] > cols[-1]
        for idx, c in enumerate(cols):
            X = fit_site(left_env(c), mps[c], Tz[c], right_env(c))      # [a', d, b']
            a, d, b = X.shape
            last_of_pass = idx == len(cols) - 1
            if last_of_pass:
                P[c] = X
                centre = c
            elif moving_left:
                Q, _ = np.linalg.qr(X.reshape(a, d * b).T)           # X^T = Q R -> X = R^T Q^T
                k = Q.shape[1]
                Pn = np.zeros((a, d * b))
                Pn[:k] = Q.T
                P[c] = Pn.reshape(a, d, b)
            else:
                Q, _ = np.linalg.qr(X.reshape(a * d, b))
                k = Q.shape[1]
                Pn = np.zeros((a * d, b))
                Pn[:, :k] = Q
                P[c] = Pn.reshape(a, d, b)
    n = float(np.linalg.norm(P[centre]))
    if n == 0.0:
        return P, -math.inf
    P[centre] = P[centre] / n
    return P, math.log(n)


def trivial_mps(L: int):
    return [np.ones((1, 1, 1)) for _ in range(L)]


def _absorb(mps, Trow, Dc, left_to_right, perturb, fit_sweeps):
    if fit_sweeps:
        return absorb_row_fit(mps, Trow, Dc, left_to_right, fit_sweeps)
    return absorb_row(mps, Trow, Dc, left_to_right, perturb=perturb)


def top_envs(T, Ly: int, Lx: int, Dc: int, perturb=None, fit_sweeps=0):
    """Upper environments U_r (rows 0..r absorbed), r = -1..Ly-1, as a list indexed r+1.

    Row r is absorbed left-to-right when r is even, right-to-left when odd.
    Each entry is (mps, log_scale) with log_scale = sum of ln n over the
    absorbed rows; the physical index is the down bond of row r.
    """
    rows = rows_of(T, Ly, Lx)
    envs = [(trivial_mps(Lx), 0.0)]
    mps, ls = envs[0]
    for r in range(Ly):
        mps, ln = _absorb(mps, rows[r], Dc, r % 2 == 0, perturb, fit_sweeps)
        ls += ln
        envs.append((mps, ls))
        if ln == -math.inf:
            for _ in range(r + 1, Ly):
                envs.append((mps, -math.inf))
            break
    return envs


def bottom_envs(T, Ly: int, Lx: int, Dc: int, perturb=None, fit_sweeps=0):
    """Lower environments L_r (rows r..Ly-1 absorbed), r = Ly..0, as a list indexed r.

    Built from the bottom: the j-th absorbed row (j = Ly-1-r) goes
    left-to-right when j is even.  Rows enter with up and down exchanged, so
    the physical index is the up bond of row r.
    """
    rows = rows_of(T, Ly, Lx)
    envs = [None] * (Ly + 1)
    envs[Ly] = (trivial_mps(Lx), 0.0)
    mps, ls = envs[Ly]
    for r in reversed(range(Ly)):
        j = Ly - 1 - r
        flipped = [t.transpose(0, 1, 3, 2) for t in rows[r]]
        mps, ln = _absorb(mps, flipped, Dc, j % 2 == 0, perturb, fit_sweeps)
        ls += ln
        envs[r] = (mps, ls)
        if ln == -math.inf:
            for rr in range(r):
                envs[rr] = (mps, -math.inf)
            break
    return envs


def close_chain(mps) -> float:
    """Value of an MPS whose physical dimensions are all one."""
    v = np.ones((1,))
    for M in mps:
        v = v @ M[:, 0, :]
    return float(v[0])


def amplitude(A, spins, Ly, Lx, Dc, fit_sweeps=0):
    """(ln|psi|, sign psi) from the top-down boundary-MPS sweep (Fig. 1d);
    fit_sweeps > 0 takes the variational-fit truncation (absorb_row_fit)."""
    T = project(A, spins, Ly, Lx)
    mps, ls = top_envs(T, Ly, Lx, Dc, fit_sweeps=fit_sweeps)[Ly]
    if ls == -math.inf:
        return -math.inf, 0
    v = close_chain(mps)
    if v == 0.0:
        return -math.inf, 0
    return ls + math.log(abs(v)), (1 if v > 0 else -1)


def amplitude_exact(A, spins, Ly, Lx):
    T = project(A, spins, Ly, Lx)
    w = contract_exact(T, Ly, Lx)
    if w == 0.0:
        return -math.inf, 0
    return math.log(abs(w)), (1 if w > 0 else -1)


# ------------------------------------------------------------- sandwiches

def col1_left(F, Mu, T, Md):
    """F_c[b, r, b'] = sum F_{c-1}[a, l, a'] Mu[a, u, b] T[l, r, u, d] Md[a', d, b']."""
    P = np.tensordot(F, Mu, axes=([0], [0]))            # [l, a', u, b]
    Q = np.tensordot(P, T, axes=([0, 2], [0, 2]))       # [a', b, r, d]
    return np.tensordot(Q, Md, axes=([0, 3], [0, 1]))   # [b, r, b']


def col1_right(G, Mu, T, Md):
    """G_c[a, l, a'] = sum Mu[a, u, b] T[l, r, u, d] Md[a', d, b'] G_{c+1}[b, r, b']."""
    P = np.tensordot(Mu, G, axes=([2], [0]))            # [a, u, r, b']
    Q = np.tensordot(P, T, axes=([1, 2], [2, 1]))       # [a, b', l, d]
    return np.tensordot(Q, Md, axes=([1, 3], [2, 1]))   # [a, l, a']


def site_env(F, Mu, Md, G):
    """B[l, r, u, d] = sum F[a, l, a'] Mu[a, u, b] Md[a', d, b'] G[b, r, b'] (the B of Delta = B/W)."""
    P = np.tensordot(F, Mu, axes=([0], [0]))            # [l, a', u, b]
    Q = np.tensordot(P, Md, axes=([1], [0]))            # [l, u, b, d, b']
    R = np.tensordot(Q, G, axes=([2, 4], [0, 2]))       # [l, u, d, r]
    return R.transpose(0, 3, 1, 2)


def col2_left(E, Mu, T1, T2, Md):
    """E_c[b, r1, r2, b'] from E_{c-1}[a, l1, l2, a'] through one column of two rows."""
    P = np.tensordot(E, Mu, axes=([0], [0]))            # [l1, l2, a', u1, b]
    P = np.tensordot(P, T1, axes=([0, 3], [0, 2]))      # [l2, a', b, r1, m]
    P = np.tensordot(P, T2, axes=([0, 4], [0, 2]))      # [a', b, r1, r2, d2]
    return np.tensordot(P, Md, axes=([0, 4], [0, 1]))   # [b, r1, r2, b']


def col2_right(H, Mu, T1, T2, Md):
    """H_c[a, l1, l2, a'] from H_{c+1}[b, r1, r2, b'] through one column of two rows."""
    P = np.tensordot(Mu, H, axes=([2], [0]))            # [a, u1, r1, r2, b']
    P = np.tensordot(P, T1, axes=([1, 2], [2, 1]))      # [a, r2, b', l1, m]
    P = np.tensordot(P, T2, axes=([1, 4], [1, 2]))      # [a, b', l1, l2, d2]
    return np.tensordot(P, Md, axes=([1, 4], [2, 1]))   # [a, l1, l2, a']


class Evaluation:
    """All per-configuration outputs of the hot path for one S."""

    def __init__(self):
        self.logabs = -math.inf
        self.sign = 0
        self.eloc = math.nan
        self.O = None            # [N][D][D][D][D] padded, block of s_i
        self.W_row = None        # raw single-row sandwich values
        self.ratios = {}         # (i, j) -> W_x(S')/W_x(S)
        self.status = 0


PEPS_OK, PEPS_EINVAL, PEPS_ENUMERIC = 0, 1, 5


def evaluate(A, spins, Ly, Lx, Dc, J1, J2, want_O=True, perturb=None, fit_sweeps=0):
    """ln|psi|, sign, E_loc (Sec. II, E(S)) and Delta = B/W (Sec. II) for one configuration.

    Ratios W(S')/W(S) and Delta reuse the environments of S: a pair inside
    row r uses <U_{r-1}| row r |L_{r+1}>, a pair across rows r, r+1 (vertical
    or diagonal) uses <U_{r-1}| rows r, r+1 |L_{r+2}>; each ratio and each
    Delta is divided by the W of the same sandwich.  fit_sweeps > 0 builds
    the environments with the variational-fit truncation (absorb_row_fit).
    """
    ev = Evaluation()
    N = Ly * Lx
    spins = np.asarray(spins).astype(np.int64)
    if N % 2 == 0 and int(spins.sum()) != N // 2:
        ev.status = PEPS_EINVAL
        return ev
    D = A.shape[2]
    T = project(A, spins, Ly, Lx)
    up = top_envs(T, Ly, Lx, Dc, perturb, fit_sweeps)
    dn = bottom_envs(T, Ly, Lx, Dc, perturb, fit_sweeps)
    mps, ls = up[Ly]
    v = close_chain(mps) if ls != -math.inf else 0.0
    if v == 0.0:
        ev.status = PEPS_ENUMERIC
        return ev
    ev.logabs = ls + math.log(abs(v))
    ev.sign = 1 if v > 0 else -1

    def flipT(i):
        r, c = divmod(i, Lx)
        dims = T[i].shape
        return A[i, 1 - spins[i], :dims[0], :dims[1], :dims[2], :dims[3]]

    # ---- single-row sandwiches: W_r, horizontal ratios, Delta
    ev.W_row = np.zeros(Ly)
    O = np.zeros((N, D, D, D, D)) if want_O else None
    hratio = {}
    for r in range(Ly):
        Mu = up[r][0]              # U_{r-1}
        Md = dn[r + 1][0]          # L_{r+1}
        Trow = T[r * Lx:(r + 1) * Lx]
        F = [np.ones((1, 1, 1))]
        for c in range(Lx):
            F.append(col1_left(F[-1], Mu[c], Trow[c], Md[c]))   # F[c+1] = F_c
        G = [None] * (Lx + 1)
        G[Lx] = np.ones((1, 1, 1))
        for c in reversed(range(Lx)):
            G[c] = col1_right(G[c + 1], Mu[c], Trow[c], Md[c])  # G[c] = G_c
        W = float(F[Lx].reshape(-1)[0])
        ev.W_row[r] = W
        if W == 0.0:
            ev.status = PEPS_ENUMERIC
            return ev
        for c in range(Lx - 1):
            i, j = r * Lx + c, r * Lx + c + 1
            if spins[i] != spins[j]:
                X = col1_left(F[c], Mu[c], flipT(i), Md[c])
                X = col1_left(X, Mu[c + 1], flipT(j), Md[c + 1])
                hratio[(i, j)] = float(np.sum(X * G[c + 2])) / W
        if want_O:
            for c in range(Lx):
                B = site_env(F[c], Mu[c], Md[c], G[c + 1])
                i = r * Lx + c
                dl, dr, du, dd = B.shape
                O[i, :dl, :dr, :du, :dd] = B / W

    # ---- two-row sandwiches: vertical and diagonal ratios
    vratio = {}
    for r in range(Ly - 1):
        Mu = up[r][0]              # U_{r-1}
        Md = dn[r + 2][0]          # L_{r+2}
        T1 = T[r * Lx:(r + 1) * Lx]
        T2 = T[(r + 1) * Lx:(r + 2) * Lx]
        E = [np.ones((1, 1, 1, 1))]
        for c in range(Lx):
            E.append(col2_left(E[-1], Mu[c], T1[c], T2[c], Md[c]))
        H = [None] * (Lx + 1)
        H[Lx] = np.ones((1, 1, 1, 1))
        for c in reversed(range(Lx)):
            H[c] = col2_right(H[c + 1], Mu[c], T1[c], T2[c], Md[c])
        W2 = float(E[Lx].reshape(-1)[0])
        if W2 == 0.0:
            ev.status = PEPS_ENUMERIC
            return ev
        for c in range(Lx):
            i, j = r * Lx + c, (r + 1) * Lx + c
            if spins[i] != spins[j]:
                X = col2_left(E[c], Mu[c], flipT(i), flipT(j), Md[c])
                vratio[(i, j)] = float(np.sum(X * H[c + 1])) / W2
        for c in range(Lx - 1):
            a, b = r * Lx + c, (r + 1) * Lx + c + 1          # diagonal (r,c)-(r+1,c+1)
            if spins[a] != spins[b]:
                X = col2_left(E[c], Mu[c], flipT(a), T2[c], Md[c])
                X = col2_left(X, Mu[c + 1], T1[c + 1], flipT(b), Md[c + 1])
                vratio[(a, b)] = float(np.sum(X * H[c + 2])) / W2
            a, b = r * Lx + c + 1, (r + 1) * Lx + c          # anti-diagonal (r,c+1)-(r+1,c)
            if spins[a] != spins[b]:
                X = col2_left(E[c], Mu[c], T1[c], flipT(b), Md[c])
                X = col2_left(X, Mu[c + 1], flipT(a), T2[c + 1], Md[c + 1])
                vratio[(a, b)] = float(np.sum(X * H[c + 2])) / W2

    # ---- E(S) = sum_S' W(S')/W(S) <S'|H|S>, spin 1/2 (S = sigma/2)
    ev.ratios = {**hratio, **vratio}
    e = 0.0
    for i, j, J, kind in all_bonds(Ly, Lx, J1, J2):
        if spins[i] == spins[j]:
            e += 0.25 * J
        else:
            e += -0.25 * J + 0.5 * J * ev.ratios[(i, j)]
    ev.eloc = e
    ev.O = O
    return ev


def gradient(evals, spins_batch, N, D, d=2, weights=None):
    """Energy per site and g = 2(<E O> - <E><O>) (Sec. II gradient).

    <...> is the plain sample mean over the given configurations, or the
    weighted mean with ``weights`` (normalised here), e.g. W^2 over a full
    enumeration.  O is the full log-derivative over both spin blocks: zero
    in the block not selected by s_i.  Configurations with a non-zero status
    are left out.  Returns (energy_per_site, grad [N][d][D^4], cov = grad/2,
    count).
    """
    ok = [k for k, ev in enumerate(evals) if ev.status == 0]
    w = np.ones(len(evals)) if weights is None else np.asarray(weights, dtype=np.float64)
    wsum = float(sum(w[k] for k in ok))
    Ebar = sum(w[k] * evals[k].eloc for k in ok) / wsum
    Obar = np.zeros((N, d, D ** 4))
    EO = np.zeros((N, d, D ** 4))
    for k in ok:
        ev = evals[k]
        for i in range(N):
            s = int(spins_batch[k][i])
            o = ev.O[i].reshape(-1)
            Obar[i, s] += w[k] * o
            EO[i, s] += w[k] * ev.eloc * o
    Obar /= wsum
    EO /= wsum
    cov = EO - Ebar * Obar
    return Ebar / N, 2.0 * cov, cov, len(ok)


# ------------------------------------------------------- Metropolis sweep

_GOLD = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1


def _mix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood 2014)."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def sampler_uniform(seed: int, chain: int, sweep: int, bond: int) -> float:
    """u in [0,1) for one Metropolis decision, keyed by (seed, chain, sweep, bond index)."""
    h = seed & _MASK
    for c in (chain, sweep, bond):
        h = _mix64((h + _GOLD * (1 + c)) & _MASK)
    return (h >> 11) * 2.0 ** -53


def mc_sweep(A, spins, Ly, Lx, Dc, seed, chain, sweep, decisions=None):
    """One Metropolis sweep over the nearest-neighbour bonds; returns (spins, accepted).

    The move exchanges the two spins of an antiparallel NN pair (this keeps
    S^z = 0); it is accepted when u < (W(S')/W(S))^2 (sampling with weight
    W^2, Sec. II).  Bonds are visited in the canonical order: horizontal
    row-major, then vertical row-major; u is keyed by the bond's index in
    that order.  Ratios use the environments of the current S:
    horizontal pass: lower environments from the S at the start of the
    pass; the upper environment grows row by row from the updated rows.
    Vertical pass: the same, recomputed at its start, with the two-row
    sandwich <U_{r-1}| rows r, r+1 |L_{r+2}>.

    ``decisions`` (diagnostic, default None): a list that receives
    (bond index, (W(S')/W(S))^2, u) for every decision taken, so that a test
    can tell which decisions sat close to their threshold.
    """
    spins = np.array(spins, dtype=np.int64)
    h_bonds, v_bonds = nn_bonds(Ly, Lx)
    accepted = 0

    def T_of(i, s):
        dims = site_dims(Ly, Lx, A.shape[2])[i]
        return A[i, s, :dims[0], :dims[1], :dims[2], :dims[3]]

    # horizontal pass
    T = project(A, spins, Ly, Lx)
    dn = bottom_envs(T, Ly, Lx, Dc)
    mps_up = trivial_mps(Lx)
    for r in range(Ly):
        Md = dn[r + 1][0]
        for c in range(Lx - 1):
            b = r * (Lx - 1) + c
            i, j = r * Lx + c, r * Lx + c + 1
            if spins[i] == spins[j]:
                continue
            Trow = [T_of(r * Lx + cc, spins[r * Lx + cc]) for cc in range(Lx)]
            Fw = np.ones((1, 1, 1))
            for cc in range(Lx):
                Fw = col1_left(Fw, mps_up[cc], Trow[cc], Md[cc])
            Trow2 = list(Trow)
            Trow2[c] = T_of(i, spins[j])
            Trow2[c + 1] = T_of(j, spins[i])
            Fp = np.ones((1, 1, 1))
            for cc in range(Lx):
                Fp = col1_left(Fp, mps_up[cc], Trow2[cc], Md[cc])
            w, wp = float(Fw.reshape(-1)[0]), float(Fp.reshape(-1)[0])
            ratio2 = (wp / w) ** 2 if w != 0.0 else math.inf
            u = sampler_uniform(seed, chain, sweep, b)
            if decisions is not None:
                decisions.append((b, ratio2, u))
            if u < ratio2:
                spins[i], spins[j] = spins[j], spins[i]
                accepted += 1
        if r < Ly - 1:
            Trow = [T_of(r * Lx + cc, spins[r * Lx + cc]) for cc in range(Lx)]
            mps_up, _ = absorb_row(mps_up, Trow, Dc, left_to_right=(r % 2 == 0))

    # vertical pass
    T = project(A, spins, Ly, Lx)
    dn = bottom_envs(T, Ly, Lx, Dc)
    mps_up = trivial_mps(Lx)
    nh = len(h_bonds)
    for r in range(Ly - 1):
        Md = dn[r + 2][0]
        for c in range(Lx):
            b = nh + r * Lx + c
            i, j = r * Lx + c, (r + 1) * Lx + c
            if spins[i] == spins[j]:
                continue
            T1 = [T_of(r * Lx + cc, spins[r * Lx + cc]) for cc in range(Lx)]
            T2 = [T_of((r + 1) * Lx + cc, spins[(r + 1) * Lx + cc]) for cc in range(Lx)]
            Ew = np.ones((1, 1, 1, 1))
            for cc in range(Lx):
                Ew = col2_left(Ew, mps_up[cc], T1[cc], T2[cc], Md[cc])
            T1p, T2p = list(T1), list(T2)
            T1p[c] = T_of(i, spins[j])
            T2p[c] = T_of(j, spins[i])
            Ep = np.ones((1, 1, 1, 1))
            for cc in range(Lx):
                Ep = col2_left(Ep, mps_up[cc], T1p[cc], T2p[cc], Md[cc])
            w, wp = float(Ew.reshape(-1)[0]), float(Ep.reshape(-1)[0])
            ratio2 = (wp / w) ** 2 if w != 0.0 else math.inf
            u = sampler_uniform(seed, chain, sweep, b)
            if decisions is not None:
                decisions.append((b, ratio2, u))
            if u < ratio2:
                spins[i], spins[j] = spins[j], spins[i]
                accepted += 1
        Trow = [T_of(r * Lx + cc, spins[r * Lx + cc]) for cc in range(Lx)]
        mps_up, _ = absorb_row(mps_up, Trow, Dc, left_to_right=(r % 2 == 0))
    return spins, accepted


# ------------------------------------------------------- GO update (Sec. III)

def _mix64_vec(z):
    """SplitMix64 output function on a numpy uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def go_uniform(seed: int, step: int, n: int) -> np.ndarray:
    """p in [0, 1) for the n tensor elements of GO step `step`: one SplitMix64
    draw keyed by (seed, step, element index), top 53 bits times 2^-53."""
    gold = np.uint64(_GOLD)
    with np.errstate(over="ignore"):
        h = _mix64_vec(np.uint64(seed & _MASK) + gold * np.uint64(1 + step))
        h = _mix64_vec(h + gold * (np.uint64(1) + np.arange(n, dtype=np.uint64)))
    return (h >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def go_step(A, grad, dt: float, seed: int, step: int):
    """One gradient-optimisation update (Sec. III):

        A_lrud^s(n+1) = A_lrud^s(n) - p * dt(n) * sign(dE/dA_lrud^s),

    p uniform in [0, 1), drawn per element.  Only the sign of the derivative
    enters.  ``grad`` is dE/dA, [N][2][D^4] or A's shape (the estimator of
    `gradient`).  Entries whose derivative is zero do not move: padding past
    an open edge, or blocks that no sampled configuration selects.  A NaN or
    infinite derivative has no sign, so such a gradient is rejected
    (ValueError) and nothing moves.
    """
    g = np.asarray(grad, dtype=np.float64).reshape(A.shape)
    if not np.isfinite(g).all():
        # the rule moves an entry against the sign of its derivative; NaN has no sign
        raise ValueError("dE/dA holds NaN or infinite entries")
    p = go_uniform(seed, step, A.size).reshape(A.shape)
    return A - p * dt * np.sign(g)


def go_dt(n: int, dt0: float = 0.005, dt1: float = 0.001, n_hold: int = 50, factor: float = 0.968) -> float:
    """Step length dt(n) of the paper's 10x10 GO run (Sec. III, Fig. 4): dt0 for
    the first n_hold steps, then dt(n+1) = factor * dt(n) down to dt1, then dt1."""
    if n < n_hold:
        return dt0
    return max(dt1, dt0 * factor ** (n - n_hold + 1))


# ------------------------------------------------- exact diagonalisation

def sz0_basis(N: int) -> np.ndarray:
    """All N-bit integers with N/2 set bits (bit i = s_i), ascending."""
    from itertools import combinations
    out = []
    for ones in combinations(range(N), N // 2):
        x = 0
        for i in ones:
            x |= 1 << i
        out.append(x)
    return np.array(sorted(out), dtype=np.int64)


def hamiltonian_sz0(Ly, Lx, J1, J2):
    """Sparse H (Sec. IV) in the S^z = 0 sector; S_i.S_j = Sz Sz + (S+S- + S-S+)/2, S = sigma/2."""
    import scipy.sparse as sp
    N = Ly * Lx
    basis = sz0_basis(N)
    dim = len(basis)
    diag = np.zeros(dim)
    rows, cols, vals = [], [], []
    for i, j, J, _ in all_bonds(Ly, Lx, J1, J2):
        if J == 0.0:
            continue
        bi = (basis >> i) & 1
        bj = (basis >> j) & 1
        par = bi == bj
        diag += np.where(par, 0.25 * J, -0.25 * J)
        anti = np.nonzero(~par)[0]
        flipped = basis[anti] ^ ((1 << i) | (1 << j))
        target = np.searchsorted(basis, flipped)
        rows.append(target)
        cols.append(anti)
        vals.append(np.full(len(anti), 0.5 * J))
    rows = np.concatenate(rows + [np.arange(dim)])
    cols = np.concatenate(cols + [np.arange(dim)])
    vals = np.concatenate(vals + [diag])
    return sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim)), basis


def ground_energy(Ly, Lx, J1, J2) -> float:
    """Lowest eigenvalue of H in the S^z = 0 sector (Lanczos via ARPACK, FP64)."""
    import scipy.sparse.linalg as sla
    H, _ = hamiltonian_sz0(Ly, Lx, J1, J2)
    if H.shape[0] <= 64:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    w = sla.eigsh(H, k=1, which="SA", tol=1e-12, v0=np.ones(H.shape[0]))[0]
    return float(w[0])


def exact_sz0_wavefunction(A, Ly, Lx):
    """(basis, psi) for every S^z = 0 configuration by exact contraction (small lattices)."""
    N = Ly * Lx
    basis = sz0_basis(N)
    psi = np.empty(len(basis))
    for k, x in enumerate(basis):
        spins = [(int(x) >> i) & 1 for i in range(N)]
        psi[k] = contract_exact(project(A, spins, Ly, Lx), Ly, Lx)
    return basis, psi
