"""Pins of the oracle's variational-fit truncation mode (absorb_row_fit, the
boundary-MPS method by variational compression, Sec. II): exactness when
nothing is cut, the variational property (the fitted row's overlap with the
uncut row is at least the zip-up's and never falls from one sweep to the
next), the stationarity of the converged fit, and the structural pins of
the hot path (Euler identity) in the fit mode."""
import math

import numpy as np
import pytest

from oracle import peps_oracle as O
from paper_1611_09467_gb300 import inputs


def mps_vector(mps):
    """Full vector of an MPS [a][p][b] with boundary bonds of dimension one."""
    v = np.ones((1, 1))
    for M in mps:
        v = np.tensordot(v, M, axes=([1], [0])).reshape(-1, M.shape[2])
    return v.reshape(-1)


def row_target(mps, Trow):
    """The uncut row applied to the MPS, as a vector over the out legs."""
    L = len(Trow)
    W = None
    for c in range(L):
        X = np.tensordot(mps[c], Trow[c], axes=([1], [2]))   # [a, b, l, r, o]
        X = X.transpose(0, 2, 4, 1, 3)                       # [a, l, o, b, r]
        a, l, o, b, r = X.shape
        X = X.reshape(a * l, o, b * r)
        W = X if W is None else np.tensordot(W, X, axes=([-1], [0]))
    return W.reshape(-1)


def fidelity(P, target, ln):
    v = mps_vector(P) * math.exp(ln)
    return abs(v @ target) / (np.linalg.norm(v) * np.linalg.norm(target))


@pytest.mark.parametrize("sweeps", [1, 3])
def test_fit_is_exact_when_nothing_is_cut(sweeps):
    """4x4 D=2 Dc=4: the fit-mode amplitude equals exact contraction."""
    A = inputs.make_tensors(4, 4, 2, 601)
    for s in inputs.random_sz0(4, 16, 602):
        la, sg = O.amplitude(A, s, 4, 4, 4, fit_sweeps=sweeps)
        le, se = O.amplitude_exact(A, s, 4, 4)
        assert sg == se and abs(la - le) < 1e-12


@pytest.mark.parametrize("lr", [True, False])
def test_fit_overlap_is_variational(lr):
    """One truncated row (6 columns, D = 3, Dc = 4, an MPS of bond 3 above):
    the fitted MPS's fidelity with the uncut row is at least the zip-up's,
    and does not decrease with the number of sweeps."""
    rng = np.random.default_rng(605)
    L, D, chi, Dc = 6, 3, 3, 4
    mps = [rng.standard_normal((1 if c == 0 else chi, D, 1 if c == L - 1 else chi)) for c in range(L)]
    Trow = [rng.standard_normal((1 if c == 0 else D, 1 if c == L - 1 else D, D, D)) for c in range(L)]
    target = row_target(mps, Trow)
    Pz, lz = O.absorb_row(mps, Trow, Dc, lr)
    f = [fidelity(Pz, target, lz)]
    for sw in (1, 2, 4, 8):
        P, ln = O.absorb_row_fit(mps, Trow, Dc, lr, sw)
        f.append(fidelity(P, target, ln))
    print(" ".join("%.8f" % x for x in f))
    assert all(b >= a - 1e-12 for a, b in zip(f, f[1:]))
    assert f[-1] > f[0]


def test_converged_fit_is_stationary():
    """After many sweeps each column of the fit is parallel to its
    environment in the overlap (the ALS fixed point): the column's
    environment, projected out of the column, vanishes."""
    rng = np.random.default_rng(606)
    L, D, chi, Dc = 5, 2, 3, 3
    mps = [rng.standard_normal((1 if c == 0 else chi, D, 1 if c == L - 1 else chi)) for c in range(L)]
    Trow = [rng.standard_normal((1 if c == 0 else D, 1 if c == L - 1 else D, D, D)) for c in range(L)]
    P, ln = O.absorb_row_fit(mps, Trow, Dc, True, 60)
    P[-1] = P[-1] * math.exp(ln)            # centre at the last column
    F = np.ones((1, 1, 1))
    for k in range(L - 1):
        F = O.col1_left(F, mps[k], Trow[k], P[k])
    X = O.fit_site(F, mps[-1], Trow[-1], np.ones((1, 1, 1)))
    x, p = X.ravel(), P[-1].ravel()
    resid = np.linalg.norm(x - (x @ p) / (p @ p) * p) / np.linalg.norm(x)
    assert resid < 1e-8, resid


def test_fit_mode_keeps_the_euler_identity():
    """6x6 D=3 Dc=4 in the fit mode (2 sweeps): sum over each site of T_i Delta_i
    is 1, as in the zip-up mode (Delta is divided by the same sandwich's W)."""
    Ly = Lx = 6
    A = inputs.make_tensors(Ly, Lx, 3, 607)
    s = inputs.random_sz0(1, 36, 608)[0]
    ev = O.evaluate(A, s, Ly, Lx, 4, 1.0, 0.5, fit_sweeps=2)
    T = O.project(A, s, Ly, Lx)
    for i in range(36):
        dl, dr, du, dd = T[i].shape
        assert abs(np.sum(T[i] * ev.O[i, :dl, :dr, :du, :dd]) - 1.0) < 1e-10
    ez = O.evaluate(A, s, Ly, Lx, 4, 1.0, 0.5)
    assert abs(ev.logabs - ez.logabs) > 1e-6      # a different truncation, not the zip-up's
