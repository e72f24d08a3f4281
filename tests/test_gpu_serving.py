"""Serving loop: requests of several models overlap on the GPU, are admitted
by HBM footprint, and each result equals the same evaluation run alone."""
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


def test_results_alone_equal_results_in_the_mix():
    from paper_1611_09467_gb300.peps import PEPS
    from paper_1611_09467_gb300.serve import Server
    models = {
        "6x6_D3_Dc4_fp64": PEPS(inputs.make_tensors(6, 6, 3, 201), 6, 6, 3, 4, J1=1.0, J2=0.5, prec="fp64"),
        "8x8_D4_Dc8_fp32": PEPS(inputs.make_tensors(8, 8, 4, 202, bias_zero_index=True), 8, 8, 4, 8, J1=1.0,
                                J2=0.5, prec="fp32"),
        "4x6_D2_Dc4_fp32": PEPS(inputs.make_tensors(4, 6, 2, 203), 6, 4, 2, 4, J1=1.0, J2=0.0, prec="fp32"),
    }
    names = list(models)
    rng = np.random.default_rng(204)
    reqs = []
    for k in range(12):
        name = names[k % 3]
        m = models[name]
        n = int(rng.integers(8, 48))
        spins = inputs.random_sz0(n, m.N, 205 + k)
        S = torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()
        reqs.append((name, S, k % 4 == 0))
    alone = []
    for name, S, wantO in reqs:
        r = models[name].evaluate(S, logabs=True, eloc=True, O=wantO)
        torch.cuda.synchronize()
        alone.append({k: (v.clone() if v is not None else None) for k, v in r.items()})
    # small budget: some requests must queue until others finish
    srv = Server(nlanes=3, hbm_budget_gb=0.35)
    ids = [srv.submit(models[name], S, O=wantO) for name, S, wantO in reqs]
    done = srv.drain()
    assert sorted(i for i, _ in done) == sorted(ids)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0
    assert st["hbm_peak_gb"] <= 0.35 + 1e-9
    for rid, ref in zip(ids, alone):
        got = srv.result(rid)
        for key in ("logabs", "sign", "eloc", "status", "O"):
            if ref[key] is None:
                continue
            a, b = got[key].cpu(), ref[key].cpu()
            assert torch.equal(a, b) or torch.allclose(a, b, rtol=0, atol=0, equal_nan=True), key
    srv.close()
    for m in models.values():
        m.close()


@pytest.mark.parametrize("policy", ["fifo", "expected"])
def test_mix_with_packing_chains_and_a_tensor_core_model(policy):
    """A mix of a mixed-TF32 tensor-core model (D=8, Dc=16), FP32 and FP64
    models: small requests co-admitted into packed launches, chain requests
    whose resident configurations take Metropolis sweeps on the server, and
    Delta requested too, under either admission order.  Every result equals
    the same work run alone (chain requests: the same sweeps and evaluation
    on a copy)."""
    from paper_1611_09467_gb300.peps import PEPS
    from paper_1611_09467_gb300.serve import Server
    models = [PEPS(inputs.make_tensors(6, 6, 8, 211), 6, 6, 8, 16, J1=1.0, J2=0.5, prec="mixed_tf32"),
              PEPS(inputs.make_tensors(8, 8, 4, 212), 8, 8, 4, 8, J1=1.0, J2=0.5, prec="fp32"),
              PEPS(inputs.make_tensors(6, 6, 3, 213), 6, 6, 3, 6, J1=1.0, J2=0.0, prec="fp32"),
              PEPS(inputs.make_tensors(4, 6, 3, 214), 6, 4, 3, 6, J1=1.0, J2=0.5, prec="fp64")]
    rng = np.random.default_rng(215)
    srv = Server(nlanes=2, hbm_budget_gb=4.0)
    srv.set_packing(64, 4)
    srv.set_policy(policy)
    plain, chains = [], []
    for k in range(10):
        m = models[k % 4]
        n = int(rng.integers(8, 60))
        S = torch.from_numpy(inputs.pack_spins(inputs.random_sz0(n, m.N, 216 + k)).view(np.int64)).cuda()
        plain.append((m, S, k % 3 == 0))
    for k in range(3):
        m = models[(k + 1) % 4]
        S = torch.from_numpy(inputs.pack_spins(inputs.random_sz0(24, m.N, 230 + k)).view(np.int64)).cuda()
        chains.append((m, S, S.clone()))
    ids = [srv.submit(m, S, O=wantO) for m, S, wantO in plain]
    cids = []
    for rep in range(2):
        for k, (m, S, _) in enumerate(chains):
            cids.append((k, rep, srv.submit_chain(m, S, nsweeps=1, seed=7, chain0=100 * k, sweep0=rep)))
        srv.drain()
    done = srv.drain()
    for (m, S, wantO), rid in zip(plain, ids):
        got = srv.result(rid)
        ref = m.evaluate(S, logabs=True, eloc=True, O=wantO)
        torch.cuda.synchronize()
        for key in ("logabs", "sign", "eloc", "status") + (("O",) if wantO else ()):
            assert torch.equal(got[key], ref[key]), (m.Lx, m.D, key)
    last = {}
    for k, rep, rid in cids:
        last[k] = srv.result(rid)
    for k, (m, S, ref_S) in enumerate(chains):
        for rep in range(2):
            m.mc_sweep(ref_S, nsweeps=1, seed=7, chain0=100 * k, sweep0=rep)
        ref = m.evaluate(ref_S, logabs=True, eloc=True)
        torch.cuda.synchronize()
        assert torch.equal(S, ref_S)
        for key in ("logabs", "sign", "eloc", "status"):
            assert torch.equal(last[k][key], ref[key]), (k, key)
    st = srv.stats()
    assert st["completed"] == len(plain) + len(cids)
    srv.close()
    for m in models:
        m.close()
