"""Gradient optimisation (Sec. III) of a small PEPS with the exact gradient.

TEST INFRASTRUCTURE ONLY, like the oracle it drives.  Every S^z = 0
configuration is evaluated by the oracle and weighted by W^2 / Z, so the
energy and the gradient 2(<E O> - <E><O>) (Sec. II) are exact expectations.
The tensors are then updated by the GO rule A <- A - p dt sign(dE/dA).  Its
trace shows the four pieces together lowering the energy toward the ED
ground state and toward the paper's GO energies (Table I).

    python -m oracle.go_exact --L 4 --D 2 --J2 0 --steps 300 --hold 150

prints one line per step: step, dt, energy per site.  Configurations are
evaluated in spawned worker processes, one per core.
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import time

import numpy as np

_ARGS = None


def _init(args):
    global _ARGS
    _ARGS = args


def _evaluate_chunk(job):
    from oracle import peps_oracle as O
    A, chunk = job
    L, D, Dc, J2 = _ARGS
    out = []
    for s in chunk:
        ev = O.evaluate(A, s, L, L, Dc, 1.0, J2, want_O=True)
        out.append((ev.status, ev.logabs, ev.eloc, ev.O))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--L", type=int, default=4)
    ap.add_argument("--D", type=int, default=2)
    ap.add_argument("--Dc", type=int, default=0, help="boundary cut-off (default D^2)")
    ap.add_argument("--J2", type=float, default=0.0)
    ap.add_argument("--seed", type=int, default=201, help="tensor seed")
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--hold", type=int, default=150, help="steps at dt = 0.005 before the x0.968 decay")
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

    from oracle import peps_oracle as O
    from paper_1611_09467_gb300 import inputs
    L, D, J2 = args.L, args.D, args.J2
    Dc = args.Dc or D * D
    N = L * L
    spins = [[(int(x) >> i) & 1 for i in range(N)] for x in O.sz0_basis(N)]
    parts = 4 * args.workers
    chunks = [spins[i::parts] for i in range(parts)]
    order = [spins[i] for c in range(parts) for i in range(c, len(spins), parts)]
    A = inputs.make_tensors(L, L, D, seed=args.seed)
    print(f"# {L}x{L} D={D} Dc={Dc} J2={J2}: ED energy per site {O.ground_energy(L, L, 1.0, J2) / N:.8f}",
          flush=True)
    with mp.get_context("spawn").Pool(args.workers, initializer=_init, initargs=((L, D, Dc, J2),)) as pool:
        for n in range(args.steps):
            t = time.perf_counter()
            res = [r for part in pool.map(_evaluate_chunk, [(A, c) for c in chunks]) for r in part]
            evals = []
            for status, logabs, eloc, Ov in res:
                ev = O.Evaluation()
                ev.status, ev.logabs, ev.eloc, ev.O = status, logabs, eloc, Ov
                evals.append(ev)
            top = max(ev.logabs for ev in evals if ev.status == 0)
            w = np.array([math.exp(2 * (ev.logabs - top)) if ev.status == 0 else 0.0 for ev in evals])
            e_site, grad, _, _ = O.gradient(evals, order, N, D, weights=w)
            dt = O.go_dt(n, n_hold=args.hold)
            print(f"{n} {dt:.5f} {e_site:.8f}  ({time.perf_counter() - t:.1f} s)", flush=True)
            A = O.go_step(A, grad, dt, seed=7, step=n)


if __name__ == "__main__":
    main()
