"""Convergence of the gradient-norm residual within one time step (section
6): two balls collide (`scenes.colliding_balls`).  For each time step
size h the scene is advanced with Eq. termination to the time `--t` s (the
balls in contact), and from that state (positions, velocities, active set
with its multipliers and decay factors) one residual-terminated step
(res_tol) is taken; the residual (1/h) |H^-1 grad L|_inf at every outer
iterate is reported.

    python -m paper_2512_12151_b300.residual_study [--t 0.05] [--tol 1e-6]
        [--dts 0.01,0.005,0.0025,0.00125] [--precision 0]

Prints one JSON line: per time step size, the status, the outer
iterations and the residual sequence.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--t", type=float, default=0.05)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--dts", default="0.01,0.005,0.0025,0.00125")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--max-outer", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)

    from . import binding as B
    from . import scenes

    s = scenes.colliding_balls(args.seed)
    s.params.precision = args.precision
    runs = []
    for dt in [float(t) for t in args.dts.split(",")]:
        p = scenes.Params(**{**s.params.__dict__, "dt": dt})
        n = int(round(args.t / dt))
        sim = B.Sim(s, p)
        sim.step(n)
        x, v = sim.state()
        keys, lam, gam = B.bf_get_active_set(sim.h)
        sim.close()
        p = scenes.Params(**{**p.__dict__, "res_tol": args.tol, "max_outer": args.max_outer})
        sim = B.Sim(s, p)
        B.bf_set_state(sim.h, x, v)
        B.bf_set_active_set(sim.h, keys, lam, gam)
        st, stats = sim.step(1, ok=tuple(B.STATUS))
        log = B.bf_get_residual_log(sim.h)
        runs.append({"dt": dt, "steps_before": n, "contacts": len(keys), "status": int(st),
                     "outer_iters": stats[0]["outer_iters"], "newton_iters": stats[0]["newton_iters"],
                     "residuals": [float("%.4g" % r) for r in log]})
        sim.close()
    print(json.dumps({"scene": s.name, "nv": s.nv, "nt": int(len(s.tets)), "start_time_s": args.t,
                      "res_tol": args.tol, "precision": "mixed" if args.precision else "fp64", "runs": runs}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
