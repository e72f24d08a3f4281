"""Float32 emulation of the oracle's evaluation (test infrastructure).

The FP32 and mixed GPU paths are float32 evaluations of the algorithm the
oracle runs in float64 (Fig. 1d boundary sweeps with SVD truncation, the
single- and two-row sandwiches of Sec. II).  This module runs the same steps
in float32 with numpy: every contraction is a float32 ``tensordot`` (sgemm,
float32 accumulation), every truncation a float32 SVD (LAPACK sgesdd).  It
keeps in float64 what the GPU path keeps in float64: the per-row norm and the
log scale, the ratios W(S')/W(S) once both sandwiches are formed, and the sum
E(S).  Sandwich transfers are renormalised by exact powers of two, as on the
GPU, so nothing underflows.  With ``tf32=True`` the operands of every two-row
transfer are rounded to TF32 (10 explicit mantissa bits, to nearest, ties
away from zero) before each contraction, as the tensor-core step rounds its
inputs and intermediates.

Its error against the FP64 oracle is what float32 arithmetic does to this
algorithm on this input, so the parity tests hold the GPU paths to a stated
multiple of it instead of a hand-set constant.  It imports the oracle only
for the bond list, the lattice geometry and the gradient formula (plain
definitions, not the float32 arithmetic under test).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import peps_oracle as O

F32 = np.float32


def tf32_round(x):
    """Round float32 values to TF32: keep 10 explicit mantissa bits, to nearest,
    ties away from zero (the rounding of cvt.rna.tf32.f32)."""
    b = np.ascontiguousarray(x, dtype=F32).view(np.uint32)
    finite = (b & np.uint32(0x7F800000)) != np.uint32(0x7F800000)
    r = np.where(finite, (b + np.uint32(0x1000)) & np.uint32(0xFFFFE000), b)
    return r.astype(np.uint32).view(F32).reshape(np.shape(x))


def _pow2_renorm(X):
    """X scaled by 2^-e with e the binary exponent of max|X| (exact); returns (X, e)."""
    m = float(np.max(np.abs(X))) if X.size else 0.0
    if m == 0.0 or not math.isfinite(m):
        return X, 0
    e = math.frexp(m)[1]
    return (X * F32(2.0 ** -e)).astype(F32), e


def project32(A, spins, Ly, Lx):
    D = A.shape[2]
    dims = O.site_dims(Ly, Lx, D)
    T = []
    for i in range(Ly * Lx):
        dl, dr, du, dd = dims[i]
        T.append(np.array(A[i, int(spins[i]), :dl, :dr, :du, :dd], dtype=F32))
    return T


def absorb_row32(mps, Trow, Dc, left_to_right):
    """oracle.absorb_row in float32 (norm of the last tensor in float64)."""
    L = len(Trow)
    out = [None] * L
    if left_to_right:
        C = np.ones((1, 1, 1), dtype=F32)
        for c in range(L):
            Y = np.tensordot(C, mps[c], axes=([1], [0]))
            X = np.tensordot(Y, Trow[c], axes=([1, 2], [0, 2])).transpose(0, 3, 1, 2)
            k, o, b, rr = X.shape
            if c < L - 1:
                U, s, Vt = np.linalg.svd(np.ascontiguousarray(X.reshape(k * o, b * rr)), full_matrices=False)
                K = min(Dc, k * o, b * rr)
                out[c] = U[:, :K].reshape(k, o, K).astype(F32)
                C = (s[:K, None] * Vt[:K]).reshape(K, b, rr).astype(F32)
            else:
                out[c] = X.reshape(k, o, b * rr).astype(F32)
        last = L - 1
    else:
        C = np.ones((1, 1, 1), dtype=F32)
        for c in reversed(range(L)):
            Y = np.tensordot(mps[c], C, axes=([2], [0]))
            X = np.tensordot(Y, Trow[c], axes=([1, 2], [2, 1])).transpose(0, 2, 3, 1)
            a, l, o, k = X.shape
            if c > 0:
                U, s, Vt = np.linalg.svd(np.ascontiguousarray(X.reshape(a * l, o * k)), full_matrices=False)
                K = min(Dc, a * l, o * k)
                out[c] = Vt[:K].reshape(K, o, k).astype(F32)
                C = (U[:, :K] * s[None, :K]).reshape(a, l, K).astype(F32)
            else:
                out[c] = X.reshape(a * l, o, k).astype(F32)
        last = 0
    n = float(np.linalg.norm(out[last].astype(np.float64)))
    if n == 0.0:
        return out, -math.inf
    out[last] = (out[last] / F32(n)).astype(F32)
    return out, math.log(n)


def _envs32(T, Ly, Lx, Dc):
    rows = O.rows_of(T, Ly, Lx)
    triv = [np.ones((1, 1, 1), dtype=F32) for _ in range(Lx)]
    up = [(triv, 0.0)]
    mps, ls = triv, 0.0
    for r in range(Ly):
        mps, ln = absorb_row32(mps, rows[r], Dc, r % 2 == 0)
        ls += ln
        up.append((mps, ls))
    dn = [None] * (Ly + 1)
    dn[Ly] = (triv, 0.0)
    mps, ls = triv, 0.0
    for r in reversed(range(Ly)):
        j = Ly - 1 - r
        mps, ln = absorb_row32(mps, [t.transpose(0, 1, 3, 2) for t in rows[r]], Dc, j % 2 == 0)
        ls += ln
        dn[r] = (mps, ls)
    return up, dn


def _td(a, b, axes, tf32):
    if tf32:
        a, b = tf32_round(a), tf32_round(b)
    return np.tensordot(a, b, axes=axes).astype(F32)


def col1_left(F, Mu, T, Md):
    P = np.tensordot(F, Mu, axes=([0], [0]))
    Q = np.tensordot(P, T, axes=([0, 2], [0, 2]))
    return np.tensordot(Q, Md, axes=([0, 3], [0, 1])).astype(F32)


def col1_right(G, Mu, T, Md):
    P = np.tensordot(Mu, G, axes=([2], [0]))
    Q = np.tensordot(P, T, axes=([1, 2], [2, 1]))
    return np.tensordot(Q, Md, axes=([1, 3], [2, 1])).astype(F32)


def site_env(F, Mu, Md, G):
    P = np.tensordot(F, Mu, axes=([0], [0]))
    Q = np.tensordot(P, Md, axes=([1], [0]))
    R = np.tensordot(Q, G, axes=([2, 4], [0, 2]))
    return R.transpose(0, 3, 1, 2).astype(F32)


def col2_left(E, Mu, T1, T2, Md, tf32):
    P = _td(E, Mu, ([0], [0]), tf32)
    P = _td(P, T1, ([0, 3], [0, 2]), tf32)
    P = _td(P, T2, ([0, 4], [0, 2]), tf32)
    return _td(P, Md, ([0, 4], [0, 1]), tf32)


def col2_right(H, Mu, T1, T2, Md, tf32):
    P = _td(Mu, H, ([2], [0]), tf32)
    P = _td(P, T1, ([1, 2], [2, 1]), tf32)
    P = _td(P, T2, ([1, 4], [1, 2]), tf32)
    return _td(P, Md, ([1, 4], [2, 1]), tf32)


class Eval32:
    def __init__(self):
        self.logabs, self.sign, self.eloc, self.O, self.status = -math.inf, 0, math.nan, None, 0


def evaluate32(A, spins, Ly, Lx, Dc, J1, J2, tf32=False, want_O=True):
    """ln|psi|, sign, E(S) and Delta as oracle.evaluate computes them, in float32."""
    ev = Eval32()
    N = Ly * Lx
    spins = np.asarray(spins).astype(np.int64)
    D = A.shape[2]
    A32 = np.asarray(A, dtype=F32)
    T = project32(A32, spins, Ly, Lx)
    up, dn = _envs32(T, Ly, Lx, Dc)
    mps, ls = up[Ly]
    v = np.ones((1,), dtype=F32)
    for M in mps:
        v = (v @ M[:, 0, :]).astype(F32)
    v = float(v[0])
    if v == 0.0 or ls == -math.inf:
        ev.status = O.PEPS_ENUMERIC
        return ev
    ev.logabs = ls + math.log(abs(v))
    ev.sign = 1 if v > 0 else -1

    def flipT(i):
        dims = T[i].shape
        return A32[i, 1 - spins[i], :dims[0], :dims[1], :dims[2], :dims[3]]

    ratios = {}
    Ob = np.zeros((N, D, D, D, D), dtype=F32) if want_O else None
    for r in range(Ly):
        Mu, Md = up[r][0], dn[r + 1][0]
        Trow = T[r * Lx:(r + 1) * Lx]
        F, eF = [np.ones((1, 1, 1), dtype=F32)], [0]
        for c in range(Lx):
            X, e = _pow2_renorm(col1_left(F[-1], Mu[c], Trow[c], Md[c]))
            F.append(X)
            eF.append(eF[-1] + e)
        G, eG = [None] * (Lx + 1), [0] * (Lx + 1)
        G[Lx] = np.ones((1, 1, 1), dtype=F32)
        for c in reversed(range(Lx)):
            X, e = _pow2_renorm(col1_right(G[c + 1], Mu[c], Trow[c], Md[c]))
            G[c], eG[c] = X, eG[c + 1] + e
        W, eW = float(F[Lx].reshape(-1)[0]), eF[Lx]
        if W == 0.0:
            ev.status = O.PEPS_ENUMERIC
            return ev
        for c in range(Lx - 1):
            i, j = r * Lx + c, r * Lx + c + 1
            if spins[i] != spins[j]:
                X, e1 = _pow2_renorm(col1_left(F[c], Mu[c], flipT(i), Md[c]))
                X = col1_left(X, Mu[c + 1], flipT(j), Md[c + 1])
                wp = float(np.sum(X * G[c + 2], dtype=F32))
                ratios[(i, j)] = math.ldexp(wp / W, eF[c] + e1 + eG[c + 2] - eW)
        if want_O:
            for c in range(Lx):
                B = site_env(F[c], Mu[c], Md[c], G[c + 1]).astype(np.float64)
                i = r * Lx + c
                dl, dr, du, dd = B.shape
                Ob[i, :dl, :dr, :du, :dd] = (B / W * 2.0 ** (eF[c] + eG[c + 1] - eW)).astype(F32)
    for r in range(Ly - 1):
        Mu, Md = up[r][0], dn[r + 2][0]
        T1, T2 = T[r * Lx:(r + 1) * Lx], T[(r + 1) * Lx:(r + 2) * Lx]
        E, eE = [np.ones((1, 1, 1, 1), dtype=F32)], [0]
        for c in range(Lx):
            X, e = _pow2_renorm(col2_left(E[-1], Mu[c], T1[c], T2[c], Md[c], tf32))
            E.append(X)
            eE.append(eE[-1] + e)
        H, eH = [None] * (Lx + 1), [0] * (Lx + 1)
        H[Lx] = np.ones((1, 1, 1, 1), dtype=F32)
        for c in reversed(range(Lx)):
            X, e = _pow2_renorm(col2_right(H[c + 1], Mu[c], T1[c], T2[c], Md[c], tf32))
            H[c], eH[c] = X, eH[c + 1] + e
        W2, eW2 = float(E[Lx].reshape(-1)[0]), eE[Lx]
        if W2 == 0.0:
            ev.status = O.PEPS_ENUMERIC
            return ev

        def ratio(X, eX, c_next):
            wp = float(np.sum(X * H[c_next], dtype=F32))
            return math.ldexp(wp / W2, eX + eH[c_next] - eW2)

        for c in range(Lx):
            i, j = r * Lx + c, (r + 1) * Lx + c
            if spins[i] != spins[j]:
                ratios[(i, j)] = ratio(col2_left(E[c], Mu[c], flipT(i), flipT(j), Md[c], tf32), eE[c], c + 1)
        for c in range(Lx - 1):
            a, b = r * Lx + c, (r + 1) * Lx + c + 1
            if spins[a] != spins[b]:
                X, e1 = _pow2_renorm(col2_left(E[c], Mu[c], flipT(a), T2[c], Md[c], tf32))
                X = col2_left(X, Mu[c + 1], T1[c + 1], flipT(b), Md[c + 1], tf32)
                ratios[(a, b)] = ratio(X, eE[c] + e1, c + 2)
            a, b = r * Lx + c + 1, (r + 1) * Lx + c
            if spins[a] != spins[b]:
                X, e1 = _pow2_renorm(col2_left(E[c], Mu[c], T1[c], flipT(b), Md[c], tf32))
                X = col2_left(X, Mu[c + 1], flipT(a), T2[c + 1], Md[c + 1], tf32)
                ratios[(a, b)] = ratio(X, eE[c] + e1, c + 2)
    e = 0.0
    for i, j, J, _ in O.all_bonds(Ly, Lx, J1, J2):
        e += 0.25 * J if spins[i] == spins[j] else -0.25 * J + 0.5 * J * ratios[(i, j)]
    ev.eloc = e
    ev.O = Ob.astype(np.float64) if want_O else None
    ev.ratios = ratios
    return ev


def float32_error(A, spins, Ly, Lx, Dc, J2, ref, tf32=False, draws=3, seed=0, want_O=True):
    """Largest error of float32 evaluations against the FP64 oracle result `ref`.

    Draw 0 evaluates A as given; draws 1.. evaluate A with every entry moved
    by one float32 unit roundoff (factor 1 +- 2^-24, random sign), standing in
    for the other rounding orders a float32 evaluation may take.  Returns
    (max |d ln|psi||, max |d E|, max |d Delta|, the evaluations)."""
    rng = np.random.default_rng(seed)
    u = 2.0 ** -24
    dl = de = do = 0.0
    evs = []
    for k in range(draws):
        Ak = A if k == 0 else A * (1.0 + u * rng.choice([-1.0, 1.0], size=A.shape))
        ev = evaluate32(Ak, spins, Ly, Lx, Dc, 1.0, J2, tf32=tf32, want_O=want_O)
        evs.append(ev)
        dl = max(dl, abs(ev.logabs - ref.logabs))
        de = max(de, abs(ev.eloc - ref.eloc))
        if want_O:
            do = max(do, float(np.abs(ev.O.reshape(Ly * Lx, -1) - ref.O.reshape(Ly * Lx, -1)).max()))
    return dl, de, do, evs
