"""Where the time of a boundary sweep goes: the truncation's phases, measured.

A diagnostic, not part of the computation.  It builds the library a second
time with the phase counters compiled in (``build(phase_timing=True)``,
written to ``_lib/phase/libpeps.so``), loads that build instead of the
library in this process, evaluates ln|psi| of a batch of configurations
twice (a warm-up, then counted) and prints, per phase of the truncation of
the boundary MPS (Sec. II), the cycles of one CTA per configuration (thread
0's clock64, summed over CTAs).  Counter 7 holds everything between
truncations: the zip-up contractions, the row norms and the bookkeeping.
With ln|psi| alone only the top-down sweep runs, one work item per
configuration.  Every marker is a CTA barrier, so the totals are a little
above those of the library itself.

    python -m paper_1611_09467_gb300.phase_timing [--workload 16x16_D8_Dc16] [--n 1216] [--prec mixed_tf32]
"""
from __future__ import annotations

import argparse
import ctypes

import numpy as np

from . import build, inputs, peps

PHASES = {1: "bidiagonalisation", 2: "bisection", 3: "inverse iteration", 4: "CholeskyQR2",
          5: "back-transformation", 6: "Newton-Schulz and C'", 7: "zip-up GEMMs and the rest"}


def measure(workload: str = "16x16_D8_Dc16", n: int = 1216, prec: str = "mixed_tf32", seed: int = 5):
    """{phase name: M cycles per configuration} and the counted evaluation's
    milliseconds (CUDA events)."""
    import torch

    path = build.build(phase_timing=True)
    if peps._lib is not None and peps.LIB_PATH != path:
        raise RuntimeError("the library is already loaded in this process; run the diagnostic in its own process")
    peps.LIB_PATH = path
    lib = peps.lib()
    lib.peps_phase_read.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.peps_phase_read.restype = ctypes.c_int
    w = inputs.WORKLOADS[workload]
    L, D, Dc = w["L"], w["D"], w["Dc"]
    A, _ = inputs.workload_inputs(workload, n=1)
    S = torch.from_numpy(inputs.pack_spins(inputs.random_sz0(n, L * L, seed)).view(np.int64)).cuda()
    p = peps.PEPS(A, L, L, D, Dc, J1=1.0, J2=w["J2"], prec=prec)
    try:
        counts = (ctypes.c_ulonglong * 16)()
        p.evaluate(S, logabs=True, eloc=False)
        if lib.peps_phase_read(counts, 1) != 0:
            raise RuntimeError("reading the phase counters failed")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        p.evaluate(S, logabs=True, eloc=False)
        e1.record()
        torch.cuda.synchronize()
        if lib.peps_phase_read(counts, 1) != 0:
            raise RuntimeError("reading the phase counters failed")
    finally:
        p.close()
    return {name: counts[k] / n / 1e6 for k, name in PHASES.items()}, e0.elapsed_time(e1)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="16x16_D8_Dc16")
    ap.add_argument("--n", type=int, default=1216)
    ap.add_argument("--prec", default="mixed_tf32")
    a = ap.parse_args(argv)
    phases, ms = measure(a.workload, a.n, a.prec)
    total = sum(phases.values())
    print(f"{a.workload}, {a.prec}, {a.n} configurations: top-down sweeps {ms:.1f} ms, "
          f"{total:.1f} M cycles of one CTA per configuration")
    for name, v in phases.items():
        print(f"  {name:28s} {v:9.2f}  {v / total:6.3f}")


if __name__ == "__main__":
    main()
