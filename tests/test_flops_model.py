"""The roofline's algorithmic work model (flops.py) against the contractions
the oracle performs: multiply-adds are counted on every np.tensordot the
oracle calls, at the true bond dimensions of its truncated boundary MPS."""
import numpy as np
import pytest

from oracle import peps_oracle as O
from paper_1611_09467_gb300 import flops, inputs


def _count_tensordot(monkeypatch):
    """Counts 2 * (free A) * (contracted) * (free B) flops per np.tensordot."""
    count = [0]
    orig = np.tensordot

    def td(a, b, axes=2):
        a, b = np.asarray(a), np.asarray(b)
        ia, ib = axes
        free_b = int(np.prod([b.shape[j] for j in range(b.ndim) if j not in ib]))
        count[0] += 2 * a.size * free_b
        return orig(a, b, axes)
    monkeypatch.setattr(np, "tensordot", td)
    return count


@pytest.mark.parametrize("Ly,Lx,D,Dc", [(4, 4, 2, 3), (5, 4, 3, 4), (4, 6, 2, 4), (6, 5, 3, 6)])
def test_zip_up_work_equals_the_oracles_contractions(Ly, Lx, D, Dc, monkeypatch):
    """Zip-up contractions of the top-down sweep and of the bottom-up sweep
    over rows Ly-1..1 (the rows the lower environments need)."""
    count = _count_tensordot(monkeypatch)
    per_row = []
    orig = O.absorb_row

    def absorb(*a, **k):
        before = count[0]
        out = orig(*a, **k)
        per_row.append(count[0] - before)
        return out
    monkeypatch.setattr(O, "absorb_row", absorb)
    A = inputs.make_tensors(Ly, Lx, D, seed=151)
    s = inputs.random_sz0(1, Ly * Lx, 152)[0]
    T = O.project(A, s, Ly, Lx)
    O.top_envs(T, Ly, Lx, Dc)
    top = sum(per_row)
    per_row.clear()
    O.bottom_envs(T, Ly, Lx, Dc)
    bottom = sum(per_row[:Ly - 1])
    assert top + bottom == flops.boundary_flops(Lx, Ly, D, Dc, truncation=False)


@pytest.mark.parametrize("Ly,Lx,D,Dc", [(5, 4, 3, 4), (6, 6, 2, 3), (4, 5, 4, 8)])
def test_transfer_columns_equal_the_oracles_contractions(Ly, Lx, D, Dc, monkeypatch):
    """Per column, the single- and two-row transfer costs of the model equal the
    multiply-adds of the oracle's col1_left / col2_left at the same dimensions."""
    count = _count_tensordot(monkeypatch)
    w = flops.Work(Lx, Ly, D, Dc)
    rng = np.random.default_rng(153)
    for r in range(Ly):
        ub, up = w.env_up(r)
        db, dp = w.env_dn(r)
        for c in range(Lx):
            a, b, ap, bp = ub[c], ub[c + 1], db[c], db[c + 1]
            l, rr, _, _ = w.tdim(r, c)
            F = rng.standard_normal((a, l, ap))
            Mu = rng.standard_normal((a, up, b))
            T = rng.standard_normal((l, rr, up, dp))
            Md = rng.standard_normal((ap, dp, bp))
            count[0] = 0
            O.col1_left(F, Mu, T, Md)
            assert count[0] == w.col1(r, c, ub, up, db, dp), (r, c)
    for r in range(Ly - 1):
        ub, up = w.env_up(r)
        db, dp = w.env_dn(r + 1)
        for c in range(Lx):
            a, b, ap, bp = ub[c], ub[c + 1], db[c], db[c + 1]
            l1, r1, _, m = w.tdim(r, c)
            l2, r2, _, _ = w.tdim(r + 1, c)
            E = rng.standard_normal((a, l1, l2, ap))
            Mu = rng.standard_normal((a, up, b))
            T1 = rng.standard_normal((l1, r1, up, m))
            T2 = rng.standard_normal((l2, r2, m, dp))
            Md = rng.standard_normal((ap, dp, bp))
            count[0] = 0
            O.col2_left(E, Mu, T1, T2, Md)
            assert count[0] == w.col2(r, c, ub, up, db, dp), (r, c)
