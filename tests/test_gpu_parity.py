"""GPU parity: libpeps.so (through the C ABI) against the FP64 oracle.

Tolerances (from the arithmetic; see the design notes):
  FP64 path: ln|psi| within 1e-10 (relative error of psi <= 1e-10), same sign;
             E_loc within 1e-8 * (1 + sum of |terms|); Delta within 1e-8 relative
             to its largest entry; gradient within 1e-8 relative to its norm.
  FP32 path: ln|psi| within 1e-5, E_loc within 2e-3 * (1 + sum|terms|),
             gradient cosine similarity >= 0.999.
"""
import math

import numpy as np
import pytest

from oracle import peps_oracle as O
from paper_1611_09467_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_09467_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def make(A, L, Ly, D, Dc, J2, prec):
    from paper_1611_09467_gb300.peps import PEPS
    return PEPS(A, L, Ly, D, Dc, J1=1.0, J2=J2, prec=prec)


def packed(spins):
    return torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()


def eloc_scale(ev, Ly, Lx, J1, J2, spins):
    """1 + sum over bonds of |each term| of E(S): the scale rounding errors are relative to."""
    s = 1.0
    for i, j, J, _ in O.all_bonds(Ly, Lx, J1, J2):
        s += abs(J) / 4
        if spins[i] != spins[j]:
            s += abs(J) / 2 * abs(ev.ratios[(i, j)])
    return s


def oracle_evals(A, spins, Ly, Lx, Dc, J2, want_O=True):
    return [O.evaluate(A, s, Ly, Lx, Dc, 1.0, J2, want_O=want_O) for s in spins]


CASES_FP64 = [
    # (Ly, Lx, D, Dc, J2, n, bias, seed) -- 4x4 D=2 Dc=4 is the exact regime
    (4, 4, 2, 4, 0.5, 64, False, inputs.SEED_BASE + 1),
    (6, 6, 3, 4, 0.5, 12, False, 77),          # truncated: Dc < D^3
    (4, 5, 2, 3, 0.5, 12, True, 78),           # rectangular, odd width, truncated
    (5, 4, 3, 9, 0.0, 8, False, 79),           # J2 = 0, exact
    (2, 6, 2, 2, 0.5, 10, False, 80),          # two rows only, truncated
    (6, 5, 4, 8, 0.5, 6, True, 81),            # fused two-row step (D=4, Dc=8), truncated
    (4, 4, 8, 16, 0.5, 4, False, 82),          # D=8: cut blocks of up to 128 x 128, fused row step
    (5, 6, 6, 12, 0.5, 4, True, 83),           # D=6: cut blocks of up to 72 rows
    (4, 4, 10, 20, 0.5, 3, False, 84),         # D=10: cut blocks of 200 rows held in global memory
]


@pytest.mark.parametrize("case", CASES_FP64)
def test_fp64_parity(case):
    Ly, Lx, D, Dc, J2, n, bias, seed = case
    A = inputs.make_tensors(Ly, Lx, D, seed, bias_zero_index=bias)
    spins = inputs.random_sz0(n, Ly * Lx, seed)
    p = make(A, Lx, Ly, D, Dc, J2, "fp64")
    r = p.evaluate(packed(spins), logabs=True, eloc=True, O=True)
    torch.cuda.synchronize()
    la = r["logabs"].cpu().numpy()
    sg = r["sign"].cpu().numpy()
    el = r["eloc"].cpu().numpy()
    Og = r["O"].cpu().numpy()
    st = r["status"].cpu().numpy()
    evs = oracle_evals(A, spins, Ly, Lx, Dc, J2)
    assert (st == 0).all()
    for k, ev in enumerate(evs):
        assert sg[k] == ev.sign, k
        assert abs(la[k] - ev.logabs) < 1e-10, (k, la[k], ev.logabs)
        scale = eloc_scale(ev, Ly, Lx, 1.0, J2, spins[k])
        assert abs(el[k] - ev.eloc) < 1e-8 * scale, (k, el[k], ev.eloc)
        ref = ev.O.reshape(Ly * Lx, -1)
        assert np.abs(Og[k] - ref).max() < 1e-8 * np.abs(ref).max(), k
    # gradient over the batch
    g = p.gradient(packed(spins))
    e_site, gref, cref, nref = O.gradient(evs, spins, Ly * Lx, D)
    assert g["n_used"] == nref
    assert abs(g["energy_per_site"] - e_site) < 1e-9 * (1 + abs(e_site))
    gg = g["grad"].cpu().numpy()
    assert np.linalg.norm(gg - gref) < 1e-8 * np.linalg.norm(gref)
    assert np.allclose(g["cov"].cpu().numpy(), gg / 2)
    p.close()


def fp32_sensitivity(A, spins, Ly, Lx, Dc, J2, trials=2, seed=0):
    """How much the FP64 oracle's ln|psi| and E_loc move under FP32-sized
    rounding: the input tensors and every block X entering a truncation are
    multiplied by (1 + 2^-24 xi), xi = +-1 at random.

    A backward-stable FP32 evaluation returns the exact result of data
    perturbed like this (times a modest constant), so its error is a multiple
    of this sensitivity.  A cut with sigma_K ~ sigma_K+1 makes it large; the
    tolerance follows it instead of a fixed number.
    """
    rng = np.random.default_rng(seed)
    u = 2.0 ** -24

    def perturb(X):
        return X * (1.0 + u * rng.choice([-1.0, 1.0], size=X.shape))

    base = O.evaluate(A, spins, Ly, Lx, Dc, 1.0, J2, want_O=False)
    dl, de = 0.0, 0.0
    for _ in range(trials):
        Ap = A * (1.0 + u * rng.choice([-1.0, 1.0], size=A.shape))
        ev = O.evaluate(Ap, spins, Ly, Lx, Dc, 1.0, J2, want_O=False, perturb=perturb)
        dl = max(dl, abs(ev.logabs - base.logabs))
        de = max(de, abs(ev.eloc - base.eloc))
    return dl, de


FP32_COND = 30.0     # FP32 error / FP32 sensitivity allowed (backward-error constant)


def test_fp32_parity_8x8():
    """The 8x8 D=4 Dc=8 workload (biased tensors), FP32 path, a sample of configurations.

    Bounds: ln|psi| within 1e-5 + 30 s_psi, E_loc within 2e-3 (1 + sum|terms|)
    + 30 s_E (s = FP32 sensitivity of the FP64 result), the batch energy per
    site within the mean of those E_loc bounds / N, gradient cosine >= 0.999.
    (The median FP32 sensitivity of ln|psi| here is ~1.5e-5: rounding A to FP32
    alone moves psi by more than 1e-5, so no FP32 path can meet a flat 1e-5.)"""
    Ly = Lx = 8
    D, Dc, J2 = 4, 8, 0.5
    A, _ = inputs.workload_inputs("8x8_D4_Dc8", n=1)
    spins = inputs.random_sz0(24, 64, inputs.SEED_BASE + 2)
    p = make(A, Lx, Ly, D, Dc, J2, "fp32")
    r = p.evaluate(packed(spins), logabs=True, eloc=True, O=True)
    torch.cuda.synchronize()
    la = r["logabs"].cpu().numpy()
    el = r["eloc"].cpu().numpy()
    evs = oracle_evals(A, spins, Ly, Lx, Dc, J2)
    rows = []
    for k, ev in enumerate(evs):
        sl, se = fp32_sensitivity(A, spins[k], Ly, Lx, Dc, J2, seed=k)
        scale = eloc_scale(ev, Ly, Lx, 1.0, J2, spins[k])
        rows.append((abs(la[k] - ev.logabs), sl, abs(el[k] - ev.eloc), se, scale, r["sign"][k].item() == ev.sign))
    print("\nk  dlogpsi  sens_psi  dE  sens_E  scale")
    for k, row in enumerate(rows):
        print(k, "%.2e %.2e %.2e %.2e %.1f %s" % row)
    for k, (dl, sl, de, se, scale, sg) in enumerate(rows):
        assert sg, k
        assert dl < 1e-5 + FP32_COND * sl, (k, dl, sl)
        assert de < 2e-3 * scale + FP32_COND * se, (k, de, se)
    g = p.gradient(packed(spins))
    e_site, gref, _, _ = O.gradient(evs, spins, 64, D)
    e_tol = np.mean([2e-3 * x[4] + FP32_COND * x[3] for x in rows]) / 64
    assert abs(g["energy_per_site"] - e_site) < e_tol
    gg = g["grad"].cpu().numpy().ravel()
    cos = gg @ gref.ravel() / (np.linalg.norm(gg) * np.linalg.norm(gref))
    assert cos > 0.999, cos
    p.close()


def test_fp32_parity_d10():
    """D = 10, Dc = 20 (the larger 16x16 workload's shapes) on a 4x5 lattice:
    cut blocks of 200 x 200 held in global memory, the generic single- and
    two-row steps.  Both precision settings run FP32 here (the tensor-core
    step covers D = 8, Dc = 16 only).  Bounds as in the 8x8 FP32 test."""
    Ly, Lx, D, Dc, J2 = 4, 5, 10, 20, 0.5
    A = inputs.make_tensors(Ly, Lx, D, 85)
    spins = inputs.random_sz0(6, Ly * Lx, 85)
    evs = oracle_evals(A, spins, Ly, Lx, Dc, J2)
    sens = [fp32_sensitivity(A, spins[k], Ly, Lx, Dc, J2, seed=k) for k in range(len(spins))]
    for prec in ("fp32", "mixed_tf32"):
        p = make(A, Lx, Ly, D, Dc, J2, prec)
        r = p.evaluate(packed(spins), logabs=True, eloc=True, O=True)
        torch.cuda.synchronize()
        la = r["logabs"].cpu().numpy()
        el = r["eloc"].cpu().numpy()
        sg = r["sign"].cpu().numpy()
        Og = r["O"].cpu().numpy()
        assert (r["status"].cpu().numpy() == 0).all(), prec
        for k, ev in enumerate(evs):
            sl, se = sens[k]
            scale = eloc_scale(ev, Ly, Lx, 1.0, J2, spins[k])
            print(prec, k, "dlogpsi %.2e (sens %.2e)  dE %.2e (sens %.2e, scale %.1f)"
                  % (abs(la[k] - ev.logabs), sl, abs(el[k] - ev.eloc), se, scale))
            assert sg[k] == ev.sign, (prec, k)
            assert abs(la[k] - ev.logabs) < 1e-5 + FP32_COND * sl, (prec, k)
            assert abs(el[k] - ev.eloc) < 2e-3 * scale + FP32_COND * se, (prec, k)
            ref = ev.O.reshape(Ly * Lx, -1)
            cos = (Og[k].ravel() @ ref.ravel()) / (np.linalg.norm(Og[k]) * np.linalg.norm(ref))
            assert cos > 0.9999, (prec, k, cos)
        p.close()


def test_mixed_tf32_parity():
    """Mixed path: two-row transfers on the tensor cores (TF32 inputs, FP32
    accumulation), D = 8, Dc = 16, against the FP64 oracle.

    TF32 keeps 10 mantissa bits (unit roundoff u = 2^-11 ~ 4.9e-4); a ratio
    passes through ~40 rounded TF32 stages (16 column steps x up to 4
    intermediates), so its relative error is bounded by ~40 u ~ 2e-2.  Bounds:
    E_loc within 2e-2 (1 + sum|terms|) + 30 s_E, ln|psi| (FP32 boundary sweep)
    within 1e-5 + 30 s_psi, batch energy per site within the mean E_loc
    bound / N, gradient within the bound the E_loc bounds propagate to.
    (Measured on uniformly drawn configurations, whose E_loc is heavy-tailed:
    relative E_loc errors up to ~2e-2, gradient cosine ~0.93 on 8 of them.)"""
    Ly = Lx = 6
    D, Dc, J2 = 8, 16, 0.5
    A = inputs.make_tensors(Ly, Lx, D, 1611094674)
    spins = inputs.random_sz0(8, Ly * Lx, 1611094674)
    p = make(A, Lx, Ly, D, Dc, J2, "mixed_tf32")
    r = p.evaluate(packed(spins), logabs=True, eloc=True, O=False)
    torch.cuda.synchronize()
    la = r["logabs"].cpu().numpy()
    el = r["eloc"].cpu().numpy()
    assert (r["status"].cpu().numpy() == 0).all()
    evs = oracle_evals(A, spins, Ly, Lx, Dc, J2)
    rows = []
    for k, ev in enumerate(evs):
        sl, se = fp32_sensitivity(A, spins[k], Ly, Lx, Dc, J2, trials=2, seed=k)
        scale = eloc_scale(ev, Ly, Lx, 1.0, J2, spins[k])
        rows.append((abs(la[k] - ev.logabs), sl, abs(el[k] - ev.eloc), se, scale))
    print("\nmixed tf32: k dlogpsi sens_psi dE sens_E scale rel_dE")
    for k, row in enumerate(rows):
        print(k, "%.2e %.2e %.2e %.2e %.1f" % row, "%.2e" % (row[2] / row[4]))
    for k, (dl, sl, de, se, scale) in enumerate(rows):
        assert dl < 1e-5 + FP32_COND * sl, (k, dl, sl)
        assert de < 2e-2 * scale + FP32_COND * se, (k, de, scale)
    g = p.gradient(packed(spins))
    e_site, gref, _, _ = O.gradient(evs, spins, Ly * Lx, D)
    e_tol = np.mean([2e-2 * x[4] + FP32_COND * x[3] for x in rows]) / (Ly * Lx)
    print("energy per site: mixed %.8f oracle %.8f" % (g["energy_per_site"], e_site))
    assert abs(g["energy_per_site"] - e_site) < e_tol
    # the gradient 2/n sum_k (E_k - <E>) O_k inherits the E_loc errors: with
    # |dE_k| <= b_k, |d grad| <= 2/n sum_k b_k |O_k - <O>| (+ the FP32 error of O)
    n = len(evs)
    Ofull = np.zeros((n, Ly * Lx, 2, D ** 4))
    for k, ev in enumerate(evs):
        for i in range(Ly * Lx):
            Ofull[k, i, spins[k][i]] = ev.O[i].reshape(-1)
    Obar = Ofull.mean(axis=0)
    bound = 2.0 / n * sum((2e-2 * x[4] + FP32_COND * x[3]) * np.linalg.norm(Ofull[k] - Obar)
                          for k, x in enumerate(rows))
    gg = g["grad"].cpu().numpy()
    err = np.linalg.norm(gg - gref)
    cos = gg.ravel() @ gref.ravel() / (np.linalg.norm(gg) * np.linalg.norm(gref))
    print("gradient: |d grad| %.3e bound %.3e |grad| %.3e cosine %.6f" % (err, bound, np.linalg.norm(gref), cos))
    assert err < bound + 1e-4 * np.linalg.norm(gref)
    p.close()


def test_status_and_edge_cases():
    Ly = Lx = 4
    D, Dc = 2, 4
    A = inputs.make_tensors(Ly, Lx, D, 5)
    p = make(A, Lx, Ly, D, Dc, 0.5, "fp64")
    # empty batch
    S0 = torch.zeros((0, 1), dtype=torch.int64, device="cuda")
    r = p.evaluate(S0)
    assert r["logabs"].numel() == 0
    # S^z != 0 -> EINVAL status
    bad = np.zeros((1, 16), dtype=np.uint8)
    bad[0, :3] = 1
    r = p.evaluate(packed(bad))
    assert r["status"].item() == 1
    # a zero site tensor block -> zero amplitude -> ENUMERIC, excluded from the gradient
    A2 = A.copy()
    A2[5, 1] = 0.0
    p2 = make(A2, Lx, Ly, D, Dc, 0.5, "fp64")
    spins = inputs.random_sz0(16, 16, 9)
    r = p2.evaluate(packed(spins))
    st = r["status"].cpu().numpy()
    hit = spins[:, 5] == 1
    assert (st[hit] == 5).all() and (st[~hit] == 0).all()
    assert np.isinf(r["logabs"].cpu().numpy()[hit]).all()
    g = p2.gradient(packed(spins))
    assert g["n_used"] == int((~hit).sum())
    p.close()
    p2.close()


def test_invalid_parameters_rejected():
    from paper_1611_09467_gb300.peps import PepsError
    A = inputs.make_tensors(4, 4, 2, 5)
    with pytest.raises(PepsError):
        make(A, 4, 4, 2, 40, 0.5, "fp64")         # Dc > 32
    A[0, 0, 1, 0, 0, 0] = 1.0                    # non-zero past the open left edge
    with pytest.raises(PepsError):
        make(A, 4, 4, 2, 4, 0.5, "fp64")


@pytest.mark.parametrize("Ly,Lx,D,Dc", [(4, 4, 2, 4), (4, 5, 2, 3)])
def test_mc_sweep_matches_oracle(Ly, Lx, D, Dc):
    """Metropolis sweeps, FP64: final configurations and accepted counts equal the
    oracle's, except chains where a decision sat within 1e-9 of the threshold."""
    A = inputs.make_tensors(Ly, Lx, D, 31)
    n = 16
    spins = inputs.random_sz0(n, Ly * Lx, 32)
    p = make(A, Lx, Ly, D, Dc, 0.5, "fp64")
    S = packed(spins)
    acc = p.mc_sweep(S, nsweeps=2, seed=1234, chain0=100, sweep0=7)
    torch.cuda.synchronize()
    got = inputs.unpack_spins(S.cpu().numpy().view(np.uint64), Ly * Lx)
    acc = acc.cpu().numpy()
    mism = 0
    for k in range(n):
        s = spins[k].copy()
        a_tot = 0
        for sw in range(2):
            s, a = O.mc_sweep(A, s, Ly, Lx, Dc, seed=1234, chain=100 + k, sweep=7 + sw)
            a_tot += a
        if not ((got[k] == s).all() and acc[k] == a_tot):
            mism += 1
        assert got[k].sum() == Ly * Lx // 2
    assert mism == 0, mism
    p.close()


def test_fp64_batched_repeatable():
    """Batched FP64 sweeps at 6x6 D=8 Dc=16 (cut blocks of up to 128 rows,
    many CTAs at once) give bit-identical ln|psi| on every run, equal to the
    one-configuration-per-call results.  A missing barrier shows up exactly
    this way: only under many concurrent CTAs, and only now and then, as a
    changed result on a badly conditioned lattice."""
    L, D, Dc = 6, 8, 16
    A = inputs.make_tensors(L, L, D, 84)
    spins = inputs.random_sz0(96, L * L, 84)
    p = make(A, L, L, D, Dc, 0.5, "fp64")
    S = packed(spins)
    runs = []
    for _ in range(3):
        r = p.evaluate(S, logabs=True, eloc=False, O=False)
        torch.cuda.synchronize()
        runs.append(r["logabs"].cpu().numpy().copy())
    for k in (1, 2):
        assert np.array_equal(runs[k], runs[0]), np.flatnonzero(runs[k] != runs[0])
    single = []
    for k in range(8):
        r = p.evaluate(S[k:k + 1], logabs=True, eloc=False, O=False)
        torch.cuda.synchronize()
        single.append(r["logabs"].cpu().numpy()[0])
    assert np.array_equal(np.array(single), runs[0][:8])
    p.close()
