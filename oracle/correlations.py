"""FP64 oracle of the sampled spin-spin correlations and the staggered
magnetisation (Sec. IV).

TEST INFRASTRUCTURE ONLY, like peps_oracle: only the tests, the smoke entry
point and bench.py's CPU legs may import it; it shares no code with the CUDA
path.

The paper measures m_s^2(k) = (1/N^2) sum_{i,j} <S_i.S_j> e^{i k.(r_i - r_j)}
at k = (pi, pi), M^2, over the central (L-2)^2 or (L-4)^2 sites, from the
sampled PEPS.  With configurations S drawn with weight W(S)^2 (Sec. II) an
operator's expectation is the mean of its local value
sum_S' <S|O|S'> W(S')/W(S).  For S_i.S_j = S^z_i S^z_j + (S+_i S-_j + S-_i S+_j)/2
and i != j that is

    (S_i.S_j)_loc(S) = S^z_i S^z_j + [s_i != s_j] (1/2) W(S^{ij}) / W(S),

S^{ij} the configuration with s_i and s_j exchanged, and 3/4 for i = j.

Reading of how W(S^{ij}) / W(S) is contracted (the paper gives E(S)'s ratios
only for nearest and next-nearest pairs): for i in row r_i and j in row
r_j >= r_i (site order i < j), the upper environment U_{r_i - 1} of S
absorbs row r_i with s_i flipped and then rows r_i + 1 .. r_j - 1, each by
the same zip-up truncation as Fig. 1(d); the result meets row r_j with s_j
flipped and the lower environment L_{r_j + 1} of S in a single-row sandwich.
The denominator is the same single-row sandwich of S, <U_{r_j-1}| row r_j
|L_{r_j+1}>, and the ratio carries the difference of the per-row norms the
two sweeps divided out.  With no truncation this is exactly
psi(S^{ij}) / psi(S).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import peps_oracle as O


def central_sites(Ly, Lx, margin):
    """Sites of the central region: rows and columns margin .. L-1-margin."""
    return [r * Lx + c for r in range(margin, Ly - margin) for c in range(margin, Lx - margin)]


def staggered_sign(i, Lx):
    r, c = divmod(i, Lx)
    return 1.0 if (r + c) % 2 == 0 else -1.0


def _row_sandwich_envs(Mu, Md, Trow):
    """Left transfers F[0..Lx] and right transfers G[0..Lx] of one row (Sec. II)."""
    Lx = len(Trow)
    F = [np.ones((1, 1, 1))]
    for c in range(Lx):
        F.append(O.col1_left(F[-1], Mu[c], Trow[c], Md[c]))
    G = [None] * (Lx + 1)
    G[Lx] = np.ones((1, 1, 1))
    for c in reversed(range(Lx)):
        G[c] = O.col1_right(G[c + 1], Mu[c], Trow[c], Md[c])
    return F, G


def exchange_ratios(A, spins, Ly, Lx, Dc, sites):
    """{(p, q): W(S^{ij}) / W(S)} for every antiparallel pair i = sites[p],
    j = sites[q] with i < j, by the contraction described in the module
    docstring."""
    spins = np.asarray(spins).astype(np.int64)
    D = A.shape[2]
    dims = O.site_dims(Ly, Lx, D)
    T = O.project(A, spins, Ly, Lx)
    up = O.top_envs(T, Ly, Lx, Dc)           # up[r + 1] = (U_r, log scale through row r)
    dn = O.bottom_envs(T, Ly, Lx, Dc)        # dn[r] = (L_r, log scale)
    rows = O.rows_of(T, Ly, Lx)

    def flipT(i):
        dl, dr, du, dd = dims[i]
        return A[i, 1 - spins[i], :dl, :dr, :du, :dd]

    # single-row sandwiches of S: W_r
    Wrow = []
    for r in range(Ly):
        F, _ = _row_sandwich_envs(up[r][0], dn[r + 1][0], rows[r])
        Wrow.append(float(F[Lx].reshape(-1)[0]))
    # per-row log norms of S's top-down sweep: ln n_r = ls(U_r) - ls(U_{r-1})
    lnU = [up[r + 1][1] - up[r][1] for r in range(Ly)]
    pos = {s: p for p, s in enumerate(sites)}
    out = {}
    for p, i in enumerate(sites):
        ri, ci = divmod(i, Lx)
        Ti = list(T)
        Ti[i] = flipT(i)
        mods = O.rows_of(Ti, Ly, Lx)
        mps = up[ri][0]                      # U_{r_i - 1} of S
        lsdiff = 0.0
        for r in range(ri, Ly):
            F, G = _row_sandwich_envs(mps, dn[r + 1][0], mods[r])
            for c in range(Lx):
                j = r * Lx + c
                if j <= i or j not in pos or spins[j] == spins[i]:
                    continue
                B = O.site_env(F[c], mps[c], dn[r + 1][0][c], G[c + 1])
                w = float(np.sum(B * flipT(j)))
                out[(p, pos[j])] = w / Wrow[r] * math.exp(lsdiff)
            if r < Ly - 1:
                mps, ln = O.absorb_row(mps, mods[r], Dc, left_to_right=(r % 2 == 0))
                lsdiff += ln - lnU[r]
    return out


def correlations(A, spins, Ly, Lx, Dc, sites):
    """C[p][q] = (S_i.S_j)_loc(S) for i = sites[p], j = sites[q] (Sec. IV)."""
    spins = np.asarray(spins).astype(np.int64)
    nc = len(sites)
    ratios = exchange_ratios(A, spins, Ly, Lx, Dc, sites)
    sz = np.array([0.5 - spins[i] for i in sites])      # s = 0 is S^z = +1/2
    C = np.outer(sz, sz)
    for (p, q), x in ratios.items():
        C[p, q] += 0.5 * x
        C[q, p] += 0.5 * x
    np.fill_diagonal(C, 0.75)
    return C


def staggered_m2(A, spins, Ly, Lx, Dc, sites):
    """M^2 local value: (1/nc^2) sum_{p,q} eps_p eps_q (S_p.S_q)_loc, eps the
    staggered sign (-1)^(r+c) (k = (pi, pi), Sec. IV)."""
    C = correlations(A, spins, Ly, Lx, Dc, sites)
    eps = np.array([staggered_sign(i, Lx) for i in sites])
    return float(eps @ C @ eps) / len(sites) ** 2
