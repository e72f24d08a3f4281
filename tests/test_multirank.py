"""The multi-rank (torchrun) path of bench.py, on CPU with gloo, world size 2.

Configurations are independent, so ranks shard them with no data-path
collective (weak scaling): each rank takes its own batch, the time is the
max over ranks, and the value counts every rank's batch.  The reference arm
runs on rank 0 alone; the other ranks exit 0 without work.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2
N_PER_RANK = 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    spins = bench.rank_configurations("16x16_D8_Dc16", N_PER_RANK, rank)
    dist.barrier()
    t = bench.max_over_ranks(5.0 + 3.0 * rank, WORLD, "cpu")
    dist.barrier()
    np.save(os.path.join(out_dir, f"spins{rank}.npy"), spins)
    with open(os.path.join(out_dir, f"t{rank}.json"), "w") as f:
        json.dump({"t": t}, f)
    dist.destroy_process_group()


def test_two_ranks_shard_configurations_and_take_the_max_time(tmp_path):
    port = _free_port()
    ctx = torch.multiprocessing.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, port, str(tmp_path))) for r in range(WORLD)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    assert [p.exitcode for p in procs] == [0] * WORLD
    import bench
    from paper_1611_09467_gb300 import inputs
    shards = [np.load(tmp_path / f"spins{r}.npy") for r in range(WORLD)]
    # together the shards are the first WORLD * n configurations of the stream, in rank order
    whole = inputs.workload_inputs("16x16_D8_Dc16", n=WORLD * N_PER_RANK)[1]
    assert np.array_equal(np.concatenate(shards), whole)
    keys = {row.tobytes() for s in shards for row in s}
    assert len(keys) == WORLD * N_PER_RANK
    for s in shards:
        assert (s.sum(axis=1) == 128).all()          # S^z = 0 on 256 sites
    times = [json.load(open(tmp_path / f"t{r}.json"))["t"] for r in range(WORLD)]
    assert times == [8.0, 8.0]
    # value = every rank's configurations over every timed step / max time
    assert bench.whole_job_rate(N_PER_RANK, WORLD, 3, 8.0) == pytest.approx(N_PER_RANK * WORLD * 3 / 8e-3)


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    """Two ranks under torchrun: one JSON line from rank 0, exit code 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={WORLD}",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", str(WORLD),
           "--steps", "1", "--warmup", "0", "--cpu-seconds", "1", "--workload", "4x4_D2_Dc4"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout
    res = json.loads(lines[0])
    assert res["impl"] == "reference" and res["n_gpus"] == WORLD and res["value"] > 0
    assert res["cpu_baseline"]["kind"] == "oracle" and res["cpu_baseline"]["value"] == res["value"]
    assert res["e2e"] == {"value": res["value"], "unit": res["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def _oracle_sums(A, spins, L, Dc, J2):
    """A rank's gradient sums in the layout of peps_gradient_sums, from the oracle."""
    from oracle import peps_oracle as O
    N, D = L * L, A.shape[2]
    T = N * 2 * D ** 4
    out = np.zeros(4 + 2 * T)
    for s in spins:
        ev = O.evaluate(A, s, L, L, Dc, 1.0, J2)
        if ev.status != 0:
            continue
        o = np.zeros((N, 2, D ** 4))
        for i in range(N):
            o[i, s[i]] = ev.O[i].reshape(-1)
        out[0] += ev.eloc
        out[1] += 1
        out[2] += ev.eloc ** 2
        out[4:4 + T] += o.ravel()
        out[4 + T:] += ev.eloc * o.ravel()
    return out


def _allreduce_rank(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_1611_09467_gb300 import dist as pdist, inputs
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    A, spins = inputs.workload_inputs("4x4_D2_Dc4", n=WORLD * 5)
    mine = spins[rank * 5:(rank + 1) * 5]
    sums = torch.from_numpy(_oracle_sums(A, mine, 4, 4, 0.5))
    np.save(os.path.join(out_dir, f"local{rank}.npy"), sums.numpy().copy())
    pdist.allreduce_sums(sums)
    np.save(os.path.join(out_dir, f"sums{rank}.npy"), sums.numpy())
    dist.destroy_process_group()


def test_allreduce_of_gradient_sums_gives_the_whole_batch_estimator(tmp_path):
    """The exchange step of a multi-rank gradient: two gloo ranks each sum
    their own configurations (layout of peps_gradient_sums), one allreduce
    adds the sums, and the means formed from them equal the single-rank
    estimator 2(<E O> - <E><O>) over the concatenated batch (Sec. II)."""
    port = _free_port()
    ctx = torch.multiprocessing.get_context("spawn")
    procs = [ctx.Process(target=_allreduce_rank, args=(r, port, str(tmp_path))) for r in range(WORLD)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    assert [p.exitcode for p in procs] == [0] * WORLD
    from oracle import peps_oracle as O
    from paper_1611_09467_gb300 import inputs
    got = [np.load(tmp_path / f"sums{r}.npy") for r in range(WORLD)]
    local = [np.load(tmp_path / f"local{r}.npy") for r in range(WORLD)]
    assert np.array_equal(got[0], got[1])                      # every rank holds the same sums
    assert np.allclose(got[0], local[0] + local[1], rtol=0, atol=1e-12 * np.abs(got[0]).max())
    A, spins = inputs.workload_inputs("4x4_D2_Dc4", n=WORLD * 5)
    evs = [O.evaluate(A, s, 4, 4, 4, 1.0, 0.5) for s in spins]
    e_site, gref, _, n = O.gradient(evs, spins, 16, 2)
    s = got[0]
    T = gref.size
    cnt = s[1]
    Ebar = s[0] / cnt
    grad = 2 * (s[4 + T:] / cnt - Ebar * s[4:4 + T] / cnt)
    assert cnt == n
    assert abs(Ebar / 16 - e_site) < 1e-12
    assert np.allclose(grad, gref.ravel(), rtol=0, atol=1e-12 * np.abs(gref).max())
