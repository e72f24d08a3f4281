"""Batching: CUDA-graph replay, the autotuner and packed multi-lattice
launches, each against the plain per-context path."""
import numpy as np
import pytest

from paper_1611_09467_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_09467_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def packed(spins):
    return torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()


def model(L, D, Dc, J2, prec, seed):
    from paper_1611_09467_gb300.peps import PEPS
    return PEPS(inputs.make_tensors(L, L, D, seed), L, L, D, Dc, J1=1.0, J2=J2, prec=prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed_tf32"])
def test_graph_replay_is_bit_identical(prec):
    """evaluate and gradient replayed from captured CUDA graphs (first call
    captures, later calls replay) equal the same calls without graphs bit for
    bit, also after the tensors change between replays (the graph reads
    them), and a larger batch (new workspace) recaptures."""
    L, D, Dc = (6, 8, 16) if prec == "mixed_tf32" else (6, 3, 6)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = model(L, D, Dc, 0.5, prec, 71)
        q = model(L, D, Dc, 0.5, prec, 71)
        q.set_graphs(True)
        S = packed(inputs.random_sz0(48, L * L, 72))
        ref = p.gradient(S, per_config=True)
        got = None
        for _ in range(3):
            got = q.gradient(S, per_config=True, out=got)
            for k in ("logabs", "sign", "eloc", "status", "grad", "cov"):
                assert torch.equal(got[k], ref[k]), k
            assert got["energy_per_site"] == ref["energy_per_site"]
        st = q.graph_stats()
        assert st["captures"] == 1 and st["replays"] == 2, st
        r1 = p.evaluate(S, logabs=True, eloc=True)
        for _ in range(2):
            r2 = q.evaluate(S, logabs=True, eloc=True)
            for k in ("logabs", "sign", "eloc", "status"):
                assert torch.equal(r1[k], r2[k]), k
        g = torch.from_numpy(np.random.default_rng(73).standard_normal((L * L, 2, D ** 4))).cuda()
        p.go_step(g, 0.003, seed=1, step=0, copy_back=False)
        q.go_step(g, 0.003, seed=1, step=0, copy_back=False)
        a, b = p.gradient(S, per_config=True), q.gradient(S, per_config=True, out=got)
        for k in ("logabs", "eloc", "grad"):
            assert torch.equal(a[k], b[k]), k
        assert q.graph_stats()["replays"] >= 3
        S2 = packed(inputs.random_sz0(200, L * L, 74))
        a, b = p.gradient(S2), q.gradient(S2)
        assert torch.equal(a["grad"], b["grad"])
        s.synchronize()
        p.close()
        q.close()


def test_autotune_chooses_and_keeps_results():
    """The tuner reports every trial and a choice for each setting; after it
    the context's results stay within rounding of the defaults (FP64: the
    variants compute the same quantities), and a new context of the same
    shape starts with the tuned settings."""
    L, D, Dc = 6, 4, 8
    p = model(L, D, Dc, 0.5, "fp64", 75)
    S = packed(inputs.random_sz0(64, L * L, 76))
    ref = p.gradient(S, per_config=True)
    rep = p.autotune(S)
    print("\n" + rep)
    assert "two-row kernel:" in rep and "single-row kernel:" in rep and "boundary grid:" in rep
    cfg = p.tuned_config()
    print(cfg)
    got = p.gradient(S, per_config=True)
    assert (got["logabs"] - ref["logabs"]).abs().max().item() < 1e-12
    assert (got["eloc"] - ref["eloc"]).abs().max().item() < 1e-10 * (1 + ref["eloc"].abs().max().item())
    q = model(L, D, Dc, 0.5, "fp64", 77)
    assert q.tuned_config()["two_row_kernel"] == cfg["two_row_kernel"]
    assert q.tuned_config()["single_row_kernel"] == cfg["single_row_kernel"]
    p.close()
    q.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_packed_launch_equals_per_lattice_results(prec):
    """Requests of four models (6x6 D=3, 8x8 D=4, 4x4 D=2 with J2 = 0, and
    10x10 D=6 in FP32 or 4x4 D=8 in FP64), their boundary sweeps in one
    launch: ln|psi|, sign, E, Delta and status equal each model's own
    evaluate bit for bit; an amplitude-only request rides along."""
    from paper_1611_09467_gb300.peps import Packer
    big = (10, 6, 12) if prec == "fp32" else (4, 8, 16)
    shapes = [(6, 3, 6, 0.5), (8, 4, 8, 0.5), (4, 2, 4, 0.0), (big[0], big[1], big[2], 0.5)]
    models = [model(L, D, Dc, J2, prec, 80 + k) for k, (L, D, Dc, J2) in enumerate(shapes)]
    reqs = [(m, packed(inputs.random_sz0(17 + 9 * k, m.N, 90 + k))) for k, m in enumerate(models)]
    pk = Packer()
    outs = pk.evaluate(reqs, eloc=True, O=True)
    torch.cuda.synchronize()
    for (m, S), o in zip(reqs, outs):
        ref = m.evaluate(S, logabs=True, eloc=True, O=True)
        torch.cuda.synchronize()
        for k in ("logabs", "sign", "eloc", "status", "O"):
            assert torch.equal(o[k], ref[k]), (m.Lx, m.D, k)
    amp = pk.evaluate([(models[1], reqs[1][1]), (models[0], reqs[0][1])], eloc=False, O=False)
    torch.cuda.synchronize()
    la, sg, st = models[1].amplitudes(reqs[1][1])
    assert torch.equal(amp[0]["logabs"], la) and torch.equal(amp[0]["sign"], sg)
    pk.close()
    for m in models:
        m.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed_tf32"])
def test_env_cache_keeps_results_and_skips_sweeps(prec):
    """With the environment cache on, amplitudes -> E_loc and Delta ->
    gradient on one batch, then a Metropolis sweep (some chains move) and
    the same again, give bit-identical results to a context without the
    cache.  The batch spans several waves of the boundary kernel, so its
    time follows the sweeps it runs: amplitudes sweep top-down, the next
    call only bottom-up, the gradient none."""
    L, D, Dc = (6, 8, 16) if prec == "mixed_tf32" else (6, 4, 8)
    p = model(L, D, Dc, 0.5, prec, 78)
    q = model(L, D, Dc, 0.5, prec, 78)
    p.set_env_cache(True)
    S = packed(inputs.random_sz0(2048, L * L, 79))
    S2 = S.clone()
    p.profile(True)
    for rnd in range(2):
        a1, b1 = p.amplitudes(S), q.amplitudes(S2)
        first = p.profile_read()["boundary"][0]
        a2 = p.evaluate(S, logabs=True, eloc=True, O=True)
        b2 = q.evaluate(S2, logabs=True, eloc=True, O=True)
        second = p.profile_read()["boundary"][0]
        a3, b3 = p.gradient(S, per_config=True), q.gradient(S2, per_config=True)
        third = p.profile_read()["boundary"][0]
        torch.cuda.synchronize()
        for x, y in zip(a1, b1):
            assert torch.equal(x, y)
        for k in ("logabs", "sign", "eloc", "O", "status"):
            assert torch.equal(a2[k], b2[k]), k
        for k in ("logabs", "eloc", "grad", "status"):
            assert torch.equal(a3[k], b3[k]), k
        print(f"{prec} round {rnd}: boundary ms amplitudes {first:.2f}, evaluate {second:.2f}, gradient {third:.2f}")
        if rnd == 0:
            assert third < 0.2 * min(first, second)
        acc_p = p.mc_sweep(S, nsweeps=1, seed=5, chain0=0, sweep0=rnd)
        acc_q = q.mc_sweep(S2, nsweeps=1, seed=5, chain0=0, sweep0=rnd)
        assert torch.equal(S, S2) and torch.equal(acc_p, acc_q)
    p.close()
    q.close()
