"""Checks of the float32 emulation the FP32 and mixed parity tests measure
their tolerances with: it is the oracle's algorithm in float32, so on a well
conditioned lattice it must agree with the FP64 oracle to float32 accuracy,
its TF32 rounding must be the hardware's rule, and it must stay in float32."""
import math

import numpy as np

from oracle import peps_oracle as O
from paper_1611_09467_gb300 import inputs
import f32_sweep as E


def test_tf32_rounding_rule():
    """10 explicit mantissa bits, to nearest, ties away from zero."""
    one = np.float32(1.0)
    ulp = 2.0 ** -10
    x = np.array([1.0, 1.0 + 2.0 ** -12, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -12, -(1.0 + 2.0 ** -11),
                  1.0 + ulp, 3.0e-39, np.inf, -np.inf], dtype=np.float32)
    r = E.tf32_round(x)
    assert r[0] == one
    assert r[1] == one                                  # below half an ulp: down
    assert r[2] == np.float32(1.0 + ulp)                # exactly half: away from zero
    assert r[3] == np.float32(1.0 + ulp)
    assert r[4] == np.float32(-(1.0 + ulp))
    assert r[5] == np.float32(1.0 + ulp)                # representable: unchanged
    assert np.isinf(r[7]) and np.isinf(r[8])
    bits = r[:7].view(np.uint32)
    assert np.all((bits & np.uint32(0x1FFF)) == 0)


def test_emulation_matches_the_oracle_to_float32_accuracy():
    """4x4 D=2 Dc=4 (exact contraction, well conditioned): ln|psi| within
    2e-6, E within 1e-4 of its scale, Delta within 1e-4 of its largest entry;
    with TF32 two-row transfers E stays within 2e-2 of its scale."""
    Ly = Lx = 4
    D, Dc, J2 = 2, 4, 0.5
    A, spins = inputs.workload_inputs("4x4_D2_Dc4", n=6)
    for s in spins:
        ref = O.evaluate(A, s, Ly, Lx, Dc, 1.0, J2)
        ev = E.evaluate32(A, s, Ly, Lx, Dc, 1.0, J2)
        scale = 1.0 + sum(abs(J) / 4 + (abs(J) / 2 * abs(ref.ratios[(i, j)]) if s[i] != s[j] else 0.0)
                          for i, j, J, _ in O.all_bonds(Ly, Lx, 1.0, J2))
        assert ev.sign == ref.sign
        assert abs(ev.logabs - ref.logabs) < 2e-6
        assert abs(ev.eloc - ref.eloc) < 1e-4 * scale
        assert abs(ev.O - ref.O).max() < 1e-4 * abs(ref.O).max()
        assert ev.logabs != ref.logabs                  # it did round
        et = E.evaluate32(A, s, Ly, Lx, Dc, 1.0, J2, tf32=True, want_O=False)
        assert abs(et.eloc - ref.eloc) < 2e-2 * scale


def test_emulation_stays_in_float32():
    """Every truncated boundary tensor is float32 (sgesdd), and a float32
    evaluation of a float64-exact product state shows float32-sized errors."""
    Ly, Lx, D, Dc = 3, 4, 2, 4
    A = inputs.make_tensors(Ly, Lx, D, 7)
    s = inputs.random_sz0(1, Ly * Lx, 7)[0]
    T = E.project32(A, s, Ly, Lx)
    assert all(t.dtype == np.float32 for t in T)
    mps = [np.ones((1, 1, 1), dtype=np.float32) for _ in range(Lx)]
    out, ln = E.absorb_row32(mps, T[:Lx], Dc, True)
    assert all(m.dtype == np.float32 for m in out) and math.isfinite(ln)
    err = E.float32_error(A, s, Ly, Lx, Dc, 0.5, O.evaluate(A, s, Ly, Lx, Dc, 1.0, 0.5), draws=2)
    assert 0.0 < err[0] < 1e-4
