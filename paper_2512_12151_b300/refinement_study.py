"""Convergence under time-step refinement (section 6, the three-dimensional
test): two balls collide and separate (`scenes.colliding_balls`, no
gravity).  The scene is simulated to the time `--t` with each step size h
of `--dts` and with the reference step `--ref`; the errors are the RMS over
vertices of |x_h(T) - x_ref(T)| and |v_h(T) - v_ref(T)| (the averaged L2
norm of the accumulated errors), and the observed order between
successive h is log2 of the error ratio (per halving of h).

    python -m paper_2512_12151_b300.refinement_study [--t 0.25]
        [--dts 0.008,0.004,0.002,0.001,0.0005] [--ref 1e-4]
        [--deltas 1e-3,1e-4] [--cells 4] [--precision 0]

Prints one JSON line per contact offset delta.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np


def run(B, s, params, t_end):
    n = int(round(t_end / params.dt))
    sim = B.Sim(s, params)
    st, stats = sim.step(n, ok=tuple(B.STATUS))
    x, v = sim.state()
    sim.close()
    return st, n, x, v, stats


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--t", type=float, default=0.25)
    ap.add_argument("--dts", default="0.008,0.004,0.002,0.001,0.0005")
    ap.add_argument("--ref", type=float, default=1e-4)
    ap.add_argument("--deltas", default="1e-3,1e-4")
    ap.add_argument("--cells", type=int, default=4)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)

    from . import binding as B
    from . import scenes

    s = scenes.colliding_balls(args.seed, cells=args.cells)
    for delta in [float(d) for d in args.deltas.split(",")]:
        base = {**s.params.__dict__, "delta": delta, "precision": args.precision, "max_outer": 5000}
        st_r, n_r, xr, vr, _ = run(B, s, scenes.Params(**{**base, "dt": args.ref}), args.t)
        rows = []
        for h in [float(t) for t in args.dts.split(",")]:
            st, n, x, v, stats = run(B, s, scenes.Params(**{**base, "dt": h}), args.t)
            ex = float(np.sqrt(np.mean(np.sum((x - xr) ** 2, axis=1))))
            ev = float(np.sqrt(np.mean(np.sum((v - vr) ** 2, axis=1))))
            rows.append({"dt": h, "steps": n, "status": int(st), "err_x": ex, "err_v": ev,
                         "mean_outer_iters": float(np.mean([q["outer_iters"] for q in stats])) if stats else None})
        for a, b in zip(rows, rows[1:]):
            for k in ("err_x", "err_v"):
                b["order_" + k[4:]] = (math.log(a[k] / b[k]) / math.log(a["dt"] / b["dt"])
                                       if a[k] > 0 and b[k] > 0 else None)
        print(json.dumps({"scene": s.name, "nv": s.nv, "nt": int(len(s.tets)), "t_end": args.t, "delta": delta,
                          "reference": {"dt": args.ref, "steps": n_r, "status": int(st_r),
                                        "centre_velocities": [vr[: s.nv // 2].mean(axis=0).round(5).tolist(),
                                                              vr[s.nv // 2:].mean(axis=0).round(5).tolist()]},
                          "precision": "mixed" if args.precision else "fp64", "runs": rows}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
