"""Stand-alone block-Jacobi PCG workload: the Newton system of the eight-cube
scene (8 cubes x 16^3 cells) or of the spiky-ball compression scene (about
2.3M tets) assembled at a contact state, solved with bf_pcg in the
library's default (persistent) mode.

    python -m paper_2512_12151_b300.pcg_case [--scene eight_cubes|spiky_balls]
        [--precision 1] [--steps 14] [--solves 2] [--mode 1] [--timers] [--autotune]

The scene is first advanced `--steps` time steps with the per-phase PCG (so
that no persistent-PCG launch happens before the timed solves; profilers can
then select the n-th persistent launch directly), then the system
H p = -G of the first Newton iteration of the next subproblem (Alg. 2) is
assembled at x = x_hat = x^t and solved `--solves` times from p = 0 in PCG mode `--mode` (see
bf_set_pcg_mode).  Prints
one JSON line: iterations per solve, milliseconds per solve, microseconds per
iteration, the solver configuration and the system size.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--scene", default="eight_cubes", choices=["eight_cubes", "spiky_balls"])
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--steps", type=int, default=14)
    ap.add_argument("--solves", type=int, default=2)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--mode", type=int, default=1, help="bf_set_pcg_mode of the timed solves")
    ap.add_argument("--timers", action="store_true", help="also report the per-phase time of CTA 0")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the mode with bf_autotune_pcg on this system instead of --mode")
    args = ap.parse_args(argv)

    import torch
    from . import binding as B
    from . import scenes

    if args.scene == "eight_cubes":
        s = scenes.eight_cubes(args.seed, precision=args.precision)
    else:
        s = scenes.spiky_balls(args.seed, precision=args.precision)
    sim = B.Sim(s)
    B.bf_set_pcg_mode(sim.h, 0)
    for i in range(args.steps):
        if args.scene == "spiky_balls":
            B.bf_set_obstacle_targets(sim.h, scenes.plate_targets_schedule(s, i))
        sim.step(1)
    x, _ = sim.state()
    keys, _, _ = B.bf_get_active_set(sim.h)
    xd = torch.tensor(np.ascontiguousarray(x), device="cuda", dtype=torch.float64)
    xt = torch.zeros_like(xd)
    B.bf_xtilde(sim.h, xt)
    B.bf_mu_init(sim.h, xt, xd)
    B.bf_linearize(sim.h, xd)
    G = torch.zeros_like(xd)
    B.bf_assemble(sim.h, xt, xd, xd, G)
    b = -G
    B.bf_set_pcg_mode(sim.h, args.mode)
    tuned = None
    if args.autotune:
        best, timed = B.bf_autotune_pcg(sim.h, 64)
        tuned = {"best_mode": best, "us_per_iteration_by_mode": {str(k): round(v, 3) for k, v in timed.items()}}
    B.bf_enable_timers(sim.h, args.timers)
    iters, ms = [], []
    for _ in range(args.solves):
        p = torch.zeros_like(xd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, _ = B.bf_pcg(sim.h, b, p, s.params.cg_tol, s.params.max_cg)
        torch.cuda.synchronize()
        ms.append(1e3 * (time.perf_counter() - t0))
        iters.append(it)
    info = sim.info()
    phases = {}
    if args.timers:
        phases = {k[len("pcg_phase_"):]: round(1e3 * v[1] / v[0], 3)
                  for k, v in B.bf_get_timers(sim.h).items() if k.startswith("pcg_phase_") and v[0]}
    print(json.dumps({"workload": "%s Newton system after %d steps" % (s.name, args.steps),
                      "precision": "mixed" if args.precision else "fp64", "nv": s.nv, "nnzb": info["nnzb"],
                      "contacts": len(keys), "iterations": iters, "ms_per_solve": [round(v, 3) for v in ms],
                      "us_per_iteration": [round(1e3 * m / max(i, 1), 3) for m, i in zip(ms, iters)],
                      "pcg_config": B.bf_get_pcg_config(sim.h),
                      **({"us_per_iteration_by_phase_cta0": phases} if args.timers else {}),
                      **({"autotune": tuned} if tuned else {})}))
    sim.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
