"""Writes accd_closed_form.json: linear-approach cases whose conservative
time of impact has a closed form.

A primitive pair whose distance decreases linearly, d(t) = d0 - v t, reaches
the ACCD target gap s*d0 (section 5.1 narrow phase; target gap reading
s = 0.1) at t* = (1 - s) d0 / v; t* > 1 means no hit within the step.
Nothing here calls the oracle or the CUDA library."""
import json
import os


def pt_case(d0, v, s=0.1):
    x0 = [0.2, 0.2, d0, 0, 0, 0, 1, 0, 0, 0, 1, 0]
    x1 = [0.2, 0.2, d0 - v, 0, 0, 0, 1, 0, 0, 0, 1, 0]
    t = (1 - s) * d0 / v if v > 0 else None
    return {"type": 0, "x0": x0, "x1": x1, "s": s, "t_star": t if t is not None and t <= 1 else None}


def ee_case(d0, v, s=0.1):
    x0 = [-1, 0, d0, 1, 0, d0, 0, -1, 0, 0, 1, 0]
    x1 = [-1, 0, d0 - v, 1, 0, d0 - v, 0, -1, 0, 0, 1, 0]
    t = (1 - s) * d0 / v if v > 0 else None
    return {"type": 1, "x0": x0, "x1": x1, "s": s, "t_star": t if t is not None and t <= 1 else None}


cases = [pt_case(0.01, 0.02), pt_case(0.01, 0.5), pt_case(0.01, 0.005), pt_case(0.003, 0.1),
         ee_case(0.01, 0.02), ee_case(0.002, 0.7), ee_case(0.01, 0.004), pt_case(0.01, -0.05),
         ee_case(0.01, -0.3)]
out = {"source": "closed form d(t) = d0 - v t, t* = (1 - s) d0 / v (linear approach)", "cases": cases}
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "accd_closed_form.json"), "w") as f:
    json.dump(out, f, indent=1)
