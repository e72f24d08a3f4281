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
