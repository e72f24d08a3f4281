"""Algorithmic work of the sampling path, counted with the true bond dimensions.

The counts are what the scheme itself needs: every contraction step at the
actual (unpadded) dimensions of the lattice edges and of the boundary MPS
after each truncation, and one ratio contraction per antiparallel pair.  The
kernels work on padded tiles, so they execute more; the roofline divides
these algorithmic counts by measured time.

A multiply-add counts as two flops.
"""
from __future__ import annotations

import numpy as np


def bond_dims(Lx, Ly, D, Dc):
    """bd[dir][j][c], c = 0..Lx: bonds of the boundary MPS after absorbing j+1 rows.

    dir 0 is the top-down sweep, dir 1 the bottom-up sweep; rows alternate
    direction and each cut keeps K = min(Dc, rows, cols) singular values.
    """
    bd = np.ones((2, Ly, Lx + 1), dtype=np.int64)
    for dr in range(2):
        b = [1] * (Lx + 1)
        for j in range(Ly):
            r = j if dr == 0 else Ly - 1 - j
            o = (1 if r == Ly - 1 else D) if dr == 0 else (1 if r == 0 else D)
            nb = [1] * (Lx + 1)
            k = 1
            if j % 2 == 0:
                for c in range(Lx - 1):
                    K = min(Dc, k * o, b[c + 1] * D)
                    nb[c + 1] = K
                    k = K
            else:
                for c in range(Lx - 1, 0, -1):
                    K = min(Dc, o * k, b[c] * D)
                    nb[c] = K
                    k = K
            bd[dr, j] = nb
            b = nb
    return bd


class Work:
    def __init__(self, Lx, Ly, D, Dc):
        self.Lx, self.Ly, self.D, self.Dc = Lx, Ly, D, Dc
        self.bd = bond_dims(Lx, Ly, D, Dc)

    def tdim(self, r, c):
        D, Lx, Ly = self.D, self.Lx, self.Ly
        return (1 if c == 0 else D, 1 if c == Lx - 1 else D, 1 if r == 0 else D, 1 if r == Ly - 1 else D)

    def env_up(self, r):
        """(bonds[c], phys) of U_{r-1} (trivial for r = 0)."""
        if r == 0:
            return [1] * (self.Lx + 1), 1
        return list(self.bd[0, r - 1]), self.tdim(r - 1, 0)[3]

    def env_dn(self, r):
        """(bonds, phys) of L_{r+1} seen from row r, i.e. rows r+1.. absorbed (trivial past the bottom)."""
        if r + 1 > self.Ly - 1:
            return [1] * (self.Lx + 1), 1
        j = self.Ly - 1 - (r + 1)
        return list(self.bd[1, j]), self.tdim(r + 1, 0)[2]

    # --- one column of the two-row transfer (left direction; right is the same count)
    def col2(self, r, c, ub, up, db, dp):
        a, b = ub[c], ub[c + 1]
        ap, bp = db[c], db[c + 1]
        l1, r1, u1, m = self.tdim(r, c)
        l2, r2, _, d2 = self.tdim(r + 1, c)
        u1 = up
        d2 = dp
        return 2 * (l1 * l2 * ap * a * u1 * b + l2 * ap * b * l1 * u1 * r1 * m + ap * b * r1 * l2 * m * r2 * d2
                    + b * r1 * r2 * ap * d2 * bp)

    def col1(self, r, c, ub, up, db, dp):
        a, b = ub[c], ub[c + 1]
        ap, bp = db[c], db[c + 1]
        l, rr, _, _ = self.tdim(r, c)
        return 2 * (l * ap * up * b * a + ap * b * rr * dp * l * up + b * rr * bp * ap * dp)

    def site_env(self, r, c, ub, up, db, dp):
        """B = (F Mu) (Md G): pair each boundary with its neighbour, then one
        contraction over (a', b)."""
        a, b = ub[c], ub[c + 1]
        ap, bp = db[c], db[c + 1]
        l, rr, _, _ = self.tdim(r, c)
        return 2 * (ap * l * up * b * a + ap * dp * b * rr * bp + l * up * dp * rr * ap * b)

    def pair_flops(self, spins=None, J2=0.5):
        """Two-row sandwiches of one configuration: transfers both ways plus flip ratios."""
        Lx, Ly = self.Lx, self.Ly
        total = 0
        for r in range(Ly - 1):
            ub, up = self.env_up(r)
            db, dp = self.env_dn(r + 1)
            cols = [self.col2(r, c, ub, up, db, dp) for c in range(Lx)]
            total += sum(cols) + sum(cols[:-1])
            if spins is not None:
                s = np.asarray(spins).reshape(Ly, Lx)
                for c in range(Lx):
                    if s[r, c] != s[r + 1, c]:
                        total += cols[c]
                    if c < Lx - 1 and J2 != 0.0:
                        if s[r, c] != s[r + 1, c + 1]:
                            total += cols[c] + cols[c + 1]
                        if s[r, c + 1] != s[r + 1, c]:
                            total += cols[c] + cols[c + 1]
        return total

    def row_flops(self, spins=None, with_O=True):
        Lx, Ly = self.Lx, self.Ly
        total = 0
        for r in range(Ly):
            ub, up = self.env_up(r)
            db, dp = self.env_dn(r)
            cols = [self.col1(r, c, ub, up, db, dp) for c in range(Lx)]
            total += sum(cols) + sum(cols[:-1])
            if with_O:
                total += sum(self.site_env(r, c, ub, up, db, dp) for c in range(Lx))
            if spins is not None:
                s = np.asarray(spins).reshape(Ly, Lx)
                for c in range(Lx - 1):
                    if s[r, c] != s[r, c + 1]:
                        total += cols[c] + cols[c + 1]
        return total


def truncation_flops(m, n, K):
    """Flops of the kept-subspace computation of an m x n block (the kernel's
    algorithm): Householder bidiagonalisation 4 P Q^2 - 4 Q^3 / 3 (P = max,
    Q = min), back-transformation of K vectors ~ 4 P Q K, and C' = U_K^T X
    2 K m n.  Nothing is computed when K == m (no cut)."""
    if K >= m:
        return 0
    P, Q = max(m, n), min(m, n)
    return 4 * P * Q * Q - 4 * Q ** 3 // 3 + 4 * P * Q * K + 2 * K * m * n


def boundary_flops(Lx, Ly, D, Dc, truncation=True):
    """One configuration's boundary sweeps: top-down over all rows and
    bottom-up over rows Ly-1..1 (zip-up contractions + truncations, true
    bond dimensions; the zip-up contractions alone with truncation=False)."""
    bd = bond_dims(Lx, Ly, D, Dc)
    total = 0
    for dr in range(2):
        rows = Ly if dr == 0 else Ly - 1
        b = [1] * (Lx + 1)
        for j in range(rows):
            r = j if dr == 0 else Ly - 1 - j
            o = (1 if r == Ly - 1 else D) if dr == 0 else (1 if r == 0 else D)
            i_phys = 1 if j == 0 else D
            k = 1
            cols = range(Lx) if j % 2 == 0 else range(Lx - 1, -1, -1)
            for c in cols:
                l = 1 if c == 0 else D
                rr = 1 if c == Lx - 1 else D
                a_, b_ = b[c], b[c + 1]
                if j % 2 == 0:
                    total += 2 * (k * l * i_phys * b_ * a_ + k * b_ * rr * o * l * i_phys)
                    m, n = k * o, b_ * rr
                    last = c == Lx - 1
                else:
                    total += 2 * (a_ * i_phys * rr * k * b_ + a_ * k * l * o * i_phys * rr)
                    m, n = o * k, a_ * l
                    last = c == 0
                if not last:
                    K = min(Dc, m, n)
                    if truncation:
                        total += truncation_flops(m, n, K)
                    k = K
            b = list(bd[dr, j])
    return total


def pair_flops_batch(Lx, Ly, D, Dc, spins, J2=0.5):
    w = Work(Lx, Ly, D, Dc)
    return sum(w.pair_flops(s, J2) for s in spins)


def row_flops_batch(Lx, Ly, D, Dc, spins, with_O=True):
    w = Work(Lx, Ly, D, Dc)
    return sum(w.row_flops(s, with_O) for s in spins)
