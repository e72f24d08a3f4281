"""Throughput of the PEPS sampling hot path on GB300.

One step = one pass of the whole path over one batch: for every configuration
ln|psi| and sign (boundary-MPS contraction, Fig. 1d), E_loc (Sec. II with the
J1-J2 Hamiltonian of Sec. IV), Delta = dln psi/dA (Sec. II), and the device
reductions to the energy and the gradient estimator 2(<E Delta> - <E><Delta>).

Default workload: 16x16 open lattice, D = 8, Dc = 16, J2/J1 = 0.5, 16384
configurations per step (per GPU), synthetic tensors and configurations.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun each rank takes its own batch
(weak scaling, no data-path collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1611_09467_gb300 import inputs  # noqa: E402

METRIC = "configs/s (psi+E_loc+dln psi) 16x16 D=8 Dc=16, mixed vs plain FP32; p99 ms"
UNIT = "configs/s"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per configuration
# of a kernel, from one ncu capture of 32 configurations of the same kernel
# build (two launches: two-row tensor-core kernel 1766.7 and 1767.2 MB);
# traffic grows in proportion to the configurations a launch processes.  It
# describes that build only: re-measure it, or drop the entry, when the
# kernel changes.  The boundary kernel has changed since its last capture,
# so it has no entry (its traffic is reported as null).
DRAM_BYTES_PER_CONFIG = {("16x16_D8_Dc16", "float", "pair_sandwich"): 5.52e7}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="16x16_D8_Dc16")
    ap.add_argument("--prec", default="mixed_tf32", choices=["fp32", "fp64", "mixed_tf32"])
    ap.add_argument("--compare-fp32", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the plain FP32 path (1 warm-up, 1 step) on the same configurations")
    ap.add_argument("--n", type=int, default=0, help="batch override (probes only; the metric uses the default)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve", action="store_true",
                    help="serving benchmark: Poisson stream of requests over mixed lattices (continuous batching)")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--serve-policy", choices=("fifo", "expected"), default="fifo",
                    help="admission order of queued requests in --serve")
    ap.add_argument("--lanes", type=int, default=4)
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="pick kernel variants and grids with peps_autotune on a probe batch first")
    ap.add_argument("--graphs", action=argparse.BooleanOptionalAction, default=False,
                    help="replay each timed step from a captured CUDA graph (per-kernel events are then not "
                         "recorded; the default line runs eagerly and measures graph replay on a small batch)")
    ap.add_argument("--workspace-gb", type=float, default=0.0,
                    help="workspace budget (0: sized so one step's batch is one chunk, within half the free HBM)")
    return ap.parse_args()


# ------------------------------------------------------------ CPU oracle arm

def _oracle_worker(args):
    name, k = args
    from oracle import peps_oracle as O
    w = inputs.WORKLOADS[name]
    A, spins = inputs.workload_inputs(name, n=1, first=k)
    t = time.perf_counter()
    O.evaluate(A, spins[0], w["L"], w["L"], w["Dc"], 1.0, w["J2"], want_O=True)
    return time.perf_counter() - t


def cpu_oracle_rate(name, seconds):
    """Oracle configs/s on the host cores: one single-threaded worker per core
    (spawned), each evaluating whole configurations, for about `seconds`."""
    import multiprocessing as mp
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        # probe one configuration per worker, then size the sample to ~seconds
        t0 = time.perf_counter()
        per = pool.map(_oracle_worker, [(name, 10_000 + i) for i in range(cores)])
        t_probe = time.perf_counter() - t0
        per_cfg = statistics.median(per)
        rounds = max(1, int(seconds / max(per_cfg, 1e-3)))
        ncfg = rounds * cores
        t0 = time.perf_counter()
        pool.map(_oracle_worker, [(name, 20_000 + i) for i in range(ncfg)])
        wall = time.perf_counter() - t0
    return dict(value=ncfg / wall, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{ncfg} configurations of the {name} workload, FP64 numpy oracle, "
                       f"{cores} spawned single-threaded workers, {wall:.1f} s (probe {t_probe:.1f} s)")


# ------------------------------------------------------------ ranks (weak scaling)

def rank_configurations(workload, n, rank):
    """Rank `rank`'s own batch: configurations rank*n .. rank*n + n - 1 of the
    workload's keyed stream.  Ranks never share a configuration, and a rank's
    batch does not depend on the world size."""
    w = inputs.WORKLOADS[workload]
    return inputs.random_sz0(n, w["L"] * w["L"], inputs.SEED_BASE + w["cfg"], first=rank * n)


def max_over_ranks(x, world, device):
    """The largest x over the ranks (a time: the job ends with its slowest rank)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_per_rank, world, steps, ms):
    """Configurations per second of the whole job: every rank's batch, every
    timed step, over the max-over-ranks time `ms`."""
    return n_per_rank * world * steps / (ms / 1e3)


# ------------------------------------------------------------- clock sampler

def start_clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def read_clocks(path, dev_index):
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(dev_index):
                continue
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
    except Exception:
        pass
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------- ours

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1611_09467_gb300 import build, flops
    from paper_1611_09467_gb300.dist import distributed_gradient
    from paper_1611_09467_gb300.peps import PEPS

    build.build()
    torch.cuda.set_device(local_rank)
    from paper_1611_09467_gb300.peps import measure_mma_shape, measure_peaks
    peaks = measure_peaks()
    w = inputs.WORKLOADS[args.workload]
    L, D, Dc, J2 = w["L"], w["D"], w["Dc"], w["J2"]
    n = args.n or w["n"]
    A, _ = inputs.workload_inputs(args.workload, n=1)
    # each rank draws its own configurations (weak scaling)
    spins = rank_configurations(args.workload, n, rank)
    S_host = torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).pin_memory()
    # the library's work goes to a stream of its own (graph capture needs one)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    S = S_host.cuda()
    ws_gb = args.workspace_gb
    if ws_gb <= 0:
        # environments + Delta of the whole batch in one chunk where half the free HBM holds them
        per_cfg = (2 * L * L * Dc * D * Dc + L * L * D ** 4) * (8 if args.prec == "fp64" else 4)
        free = torch.cuda.mem_get_info()[0]
        ws_gb = min(per_cfg * n * 1.02, 0.5 * free) / 1e9
    p = PEPS(A, L, L, D, Dc, J1=1.0, J2=J2, prec=args.prec, workspace_gb=ws_gb)
    tune_report = None
    if args.autotune:
        probe = S[: min(n, 608)].clone()
        tune_report = p.autotune(probe)
        del probe
    if args.graphs and world == 1:
        p.set_graphs(True)
    outs = {}

    def step():
        if world > 1:
            # the one exchange of a multi-GPU gradient step: an allreduce of the sums
            return distributed_gradient(p, S)
        outs["g"] = p.gradient(S, out=outs.get("g"))
        return outs["g"]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    p.profile_read(reset=True)
    p.profile(True)
    clk_path = os.path.join(tempfile.gettempdir(), f"peps_bench_clocks_rank{rank}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    sampler, fh = start_clock_sampler(clk_path)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ms = []
    ev0.record(stream)
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = step()
        b.record(stream)
        step_ms.append((a, b))
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    if sampler:
        sampler.terminate()
        sampler.wait()
        fh.close()
    total_ms = ev0.elapsed_time(ev1)
    per_step = [x.elapsed_time(y) for x, y in step_ms]
    prof = p.profile_read(reset=True)
    p.profile(False)
    total_ms = max_over_ranks(total_ms, world, "cuda")
    clocks = read_clocks(clk_path, local_rank)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        la_h = torch.empty(n, dtype=torch.float64).pin_memory()
        el_h = torch.empty(n, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        Sd = torch.empty_like(S)
        o = None
        t0.record(stream)
        for _ in range(args.steps):
            Sd.copy_(S_host, non_blocking=True)
            o = p.gradient(Sd, per_config=True, out=o)
            la_h.copy_(o["logabs"], non_blocking=True)
            el_h.copy_(o["eloc"], non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize()
        e_ms = t0.elapsed_time(t1)
        e_ms = max_over_ranks(e_ms, world, "cuda")
        e2e = {"value": whole_job_rate(n, world, args.steps, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(S_host.numel() * 8),
               "d2h_bytes_per_step": int(2 * n * 8 + 8)}

    # roofline of every kernel with a work model; the dominant one is the line's
    kern = {k: v for k, v in prof.items() if v[1] > 0 and v[0] > 0}
    if not kern:
        raise SystemExit("no per-kernel timings were recorded (graph replay records none; run without --graphs)")
    top = max(kern, key=lambda k: kern[k][0])
    sample = spins[: min(256, n)]
    tc = args.prec == "mixed_tf32" and (D, Dc) == (8, 16)
    # the tensor-core two-row step issues M128 N64 K8 (s1-s3) and M128 N16 K8
    # (s4) instructions; their measured rates bound it below the N256 peak
    mma_rates = {"N64": measure_mma_shape(64), "N16": measure_mma_shape(16)} if tc else None
    fp = "float" if args.prec != "fp64" else "double"

    def roof(kname):
        ms_k, launches_k = kern[kname]
        if kname == "pair_sandwich":
            f_cfg = flops.pair_flops_batch(L, L, D, Dc, sample, J2) / len(sample)
        elif kname == "row_sandwich":
            f_cfg = flops.row_flops_batch(L, L, D, Dc, sample) / len(sample)
        elif kname == "boundary":
            f_cfg = float(flops.boundary_flops(L, L, D, Dc))
        else:
            return None
        achieved = f_cfg * n * args.steps / launches_k / (ms_k / launches_k / 1e3) / 1e12
        if kname == "pair_sandwich" and tc:
            peak, bound, src = peaks["tf32_tcgen05"], "tensor", "measured: dense TF32 tcgen05.mma (peps_measure_peaks)"
        elif args.prec == "fp64":
            peak, bound, src = peaks["fp64_simt"], "alu", "measured: FP64 FMA on the SIMT pipe (peps_measure_peaks)"
        else:
            peak, bound, src = peaks["fp32_simt"], "alu", "measured: FP32 FMA on the SIMT pipe (peps_measure_peaks)"
        bpc = DRAM_BYTES_PER_CONFIG.get((args.workload, fp, kname))
        out = {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
               "frac": achieved / peak, "traffic": bpc * n * args.steps / launches_k if bpc else None,
               "traffic_unit": "bytes per launch (DRAM read + write, ncu)", "peak_source": src,
               "flops_per_config": f_cfg, "launches": launches_k}
        if kname == "pair_sandwich" and tc and mma_rates:
            # per slice: s1 + s2 + s3 at the N64 rate, s4 at the N16 rate
            f64_, f16_ = 2.0 * 128 * 64 * (16 + 64 + 64), 2.0 * 128 * 16 * 8 * 8
            ceil_ = (f64_ + f16_) / (f64_ / mma_rates["N64"] + f16_ / mma_rates["N16"])
            out.update({"mma_shape_rates_tflops": mma_rates, "shape_ceiling_tflops": ceil_,
                        "frac_of_shape_ceiling": achieved / ceil_})
        return out

    roofline = roof(top)
    other_roofs = {k: roof(k) for k in kern if k != top and roof(k) is not None}

    # CUDA-graph replay where launch overhead matters: a small batch (64
    # configurations of a 6x6 D=4 lattice), 50 calls eager and 50 replayed
    graph_cmp = None
    if world == 1:
        from paper_1611_09467_gb300.peps import PEPS as _P
        gs = _P(inputs.make_tensors(6, 6, 4, 99), 6, 6, 4, 8, J1=1.0, J2=0.5, prec="fp32")
        Sg = torch.from_numpy(inputs.pack_spins(inputs.random_sz0(64, 36, 99)).view(np.int64)).cuda()
        og = gs.gradient(Sg, per_config=True)
        times = {}
        for mode in ("eager", "graph"):
            gs.set_graphs(mode == "graph")
            og = gs.gradient(Sg, per_config=True, out=og)
            torch.cuda.synchronize()
            t0g = time.perf_counter()
            for _ in range(50):
                og = gs.gradient(Sg, per_config=True, out=og)
            torch.cuda.synchronize()
            times[mode] = (time.perf_counter() - t0g) / 50 * 1e3
        graph_cmp = {"workload": "6x6 D=4 Dc=8 fp32, 64 configurations, gradient with per-configuration outputs",
                     "eager_ms_per_call": times["eager"], "graph_ms_per_call": times["graph"],
                     "graph_stats": gs.graph_stats()}
        gs.close()
    share = {k: round(v[0] / sum(x[0] for x in kern.values()), 4) for k, v in kern.items()}
    launches = sum(v[1] for v in kern.values())
    value = whole_job_rate(n, world, args.steps, total_ms)
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "mixed_tf32": "tf32/f32"}[args.prec], "data": "synthetic",
        "config": {"workload": args.workload, "lattice": f"{L}x{L}", "D": D, "Dc": Dc, "J2_over_J1": J2,
                   "configs_per_step_per_gpu": n,
                   "precision_path": {"fp32": "plain FP32 SIMT", "fp64": "plain FP64 SIMT",
                                      "mixed_tf32": "two-row transfers on tcgen05 (TF32 in, FP32 accumulate), "
                                                    "rest FP32 SIMT" if (D, Dc) == (8, 16) else
                                                    "FP32 SIMT (the tcgen05 two-row step covers D=8, Dc=16)"}[args.prec],
                   "sampling": "uniform random Sz=0 configurations",
                   "l2": "working set per step (environments, Delta) is tens of GB, far above L2",
                   "parallelism": f"dp{world} (independent configurations"
                                  + ("; one allreduce of the gradient sums per step)" if world > 1 else ")")},
        "whole_step_ms": {"median": statistics.median(per_step), "max": max(per_step),
                          "what": "device time of whole timed steps (one batch each), not request latencies; "
                                  "request latency p50/p99 is the --serve line's"},
        "kernel_share": share, "gpu_launches": launches, "roofline": roofline, "clocks": clocks, "e2e": e2e,
        "energy_per_site": out["energy_per_site"], "roofline_other_kernels": other_roofs,
        "peaks_measured_tflops": peaks, "graph_replay_small_batch": graph_cmp,
    }
    res["config"]["tiles"] = p.tuned_config()
    res["config"]["graphs"] = bool(args.graphs and world == 1)
    if tune_report:
        res["config"]["autotune"] = tune_report
    if args.compare_fp32 and args.prec != "fp32":
        p.close()
        q = PEPS(A, L, L, D, Dc, J1=1.0, J2=J2, prec="fp32", workspace_gb=ws_gb)
        q.gradient(S)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        q.gradient(S)
        c1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(c0.elapsed_time(c1), world, "cuda")
        res["plain_fp32"] = {"value": whole_job_rate(n, world, 1, ms), "unit": UNIT, "ms_per_step": ms, "steps": 1,
                             "warmup": 1}
        q.close()
    return res


# (L, D, Dc, J2/J1, precision): square lattices 6..16, D in {4, 6, 8, 10},
# Dc = 2D, J2/J1 in {0, 0.5}; the D = 8 models take the tensor-core path.
SERVE_MIX = [(6, 4, 8, 0.0, "fp32"), (6, 4, 8, 0.5, "fp32"), (8, 4, 8, 0.5, "fp32"), (8, 6, 12, 0.0, "fp32"),
             (10, 6, 12, 0.5, "fp32"), (8, 8, 16, 0.0, "mixed_tf32"), (12, 8, 16, 0.5, "mixed_tf32"),
             (16, 8, 16, 0.5, "mixed_tf32"), (6, 10, 20, 0.0, "fp32")]


def run_serving(args):
    import torch
    from paper_1611_09467_gb300 import build
    from paper_1611_09467_gb300.peps import PEPS
    from paper_1611_09467_gb300.serve import Server, poisson_arrivals

    build.build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(inputs.SEED_BASE + 5)
    models = []
    for k, (L, D, Dc, J2, prec) in enumerate(SERVE_MIX):
        A = inputs.make_tensors(L, L, D, inputs.SEED_BASE + 5 + k)
        models.append(PEPS(A, L, L, D, Dc, J1=1.0, J2=J2, prec=prec))
    budget = 48.0
    srv = Server(nlanes=args.lanes, hbm_budget_gb=budget)

    def make_request(k, seed):
        m = models[k]
        n = int(rng.integers(256, 1025))
        spins = inputs.random_sz0(n, m.N, seed)
        return k, torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()

    # per-model latency alone on one lane (also creates the workers), then the
    # sustained capacity: a closed-loop burst of 4 requests per lane, timed
    def finish(server, done):
        # drop the finished requests' outputs (Delta of a large request is GBs)
        for rid, _ in done:
            server.outputs.pop(rid, None)
        return [x for _, x in done]

    probe_ms = []
    for k in range(len(models)):
        _, S = make_request(k, 10_000 + k)
        srv.submit(models[k], S, O=True)
        done = srv.drain()
        probe_ms.append(done[0][1])
        finish(srv, done)
    burst = [make_request(int(rng.integers(len(models))), 15_000 + i) for i in range(4 * args.lanes)]
    torch.cuda.synchronize()
    tb = time.perf_counter()
    for k, S in burst:
        srv.submit(models[k], S, O=True)
    finish(srv, srv.drain())
    capacity = len(burst) / (time.perf_counter() - tb)                 # requests/s, all lanes busy
    rate = 0.8 * capacity
    arrivals = poisson_arrivals(rate, args.serve_seconds, inputs.SEED_BASE + 5)
    reqs = [make_request(int(rng.integers(len(models))), 20_000 + i) for i in range(len(arrivals))]
    torch.cuda.synchronize()
    srv2 = Server(nlanes=args.lanes, hbm_budget_gb=budget)
    srv2.set_packing(512, 4)
    srv2.set_policy(args.serve_policy)
    clk_serve = os.path.join(tempfile.gettempdir(), "peps_bench_clocks_serve.csv")
    sampler, fh = start_clock_sampler(clk_serve)
    t0 = time.perf_counter()
    lat = []
    for (k, S), ta in zip(reqs, arrivals):
        while time.perf_counter() - t0 < ta:
            lat += finish(srv2, srv2.poll(wait=False))
            time.sleep(0.0005)
        srv2.submit(models[k], S, O=True)
    lat += finish(srv2, srv2.drain())
    wall = time.perf_counter() - t0
    if sampler:
        sampler.terminate()
        sampler.wait()
        fh.close()
    st = srv2.stats()
    total = sum(int(S.shape[0]) for _, S in reqs)
    res = {
        "metric": "serving: aggregate configs/s (psi+E_loc+dln psi) and request latency p50/p99 ms, mixed lattices",
        "value": total / wall, "unit": "configs/s", "n_gpus": 1, "higher_is_better": True,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "requests": len(reqs), "configs": total, "wall_s": wall, "data": "synthetic",
        "config": {"mix": [dict(L=L, D=D, Dc=Dc, J2=J2, prec=pr) for (L, D, Dc, J2, pr) in SERVE_MIX],
                   "configs_per_request": "uniform 256..1024", "outputs": "ln|psi|, sign, E_loc, Delta",
                   "arrivals": f"Poisson, {rate:.2f}/s (80% of the closed-loop capacity {capacity:.2f}/s)",
                   "packing": "requests of <= 512 configurations, up to 4 models per launch",
                   "admission": {"fifo": "first come first served",
                                 "expected": "smallest expected run time less time waited first"}[args.serve_policy],
                   "lanes": args.lanes, "hbm_budget_gb": budget,
                   "duration_s": args.serve_seconds},
        "server": st, "probe_ms_per_model": probe_ms,
        "clocks": read_clocks(clk_serve, 0),
    }
    srv.close()
    srv2.close()
    return res


def run_reference(args, rank):
    """The reference arm: the FP64 oracle as it stands, on the host cores.
    Rank 0 alone runs it (other ranks return None and exit without work):
    W untimed warm-up steps, then K timed ones, each a bounded sample of the
    workload sized so that the whole run ends within a few minutes."""
    if rank != 0:
        return None
    w = inputs.WORKLOADS[args.workload]
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_rate(args.workload, per_step)
    t0 = time.perf_counter()
    samples = [cpu_oracle_rate(args.workload, per_step) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    rate = statistics.median([c["value"] for c in samples])
    cb = dict(samples[-1])
    cb["value"] = rate
    return {
        "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall * 1e3 / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": args.workload, "lattice": f"{w['L']}x{w['L']}", "D": w["D"], "Dc": w["Dc"],
                   "J2_over_J1": w["J2"], "sampling": "uniform random Sz=0 configurations"},
        "cpu_baseline": cb,
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.serve:
        print(json.dumps(run_serving(args), default=float), flush=True)
        return
    if args.impl == "reference":
        res = run_reference(args, rank)
        if res is not None:
            print(json.dumps(res, default=float), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the oracle pool is spawned before any GPU work
        cpu = cpu_oracle_rate(args.workload, args.cpu_seconds)
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        res["cpu_baseline"] = cpu
        print(json.dumps(res, default=float), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
