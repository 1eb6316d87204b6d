"""Writes eight_cubes_oracle.npz: reference values of the FP64 oracle on the
eight-cube scene (8 cubes of 16^3 cells, 196,608 tets, seed 0) dropped into
the open box, advanced from rest by Alg. 1 for N_STEPS time steps.

Stored (everything computed by oracle/ alone; the scene generator only
supplies the inputs):
- `sample_ids`: 1,024 vertex ids drawn with a fixed seed from the free
  vertices, and `traj`: their positions after each step (N_STEPS x 1024 x 3,
  FP64), for the per-step error curve of a free-running GPU trajectory;
- `x16`, `v16`, `keys16`, `lam16`, `gam16`: the complete state after 16 steps
  (the cubes are in contact from step 15 on), with the active set as
  canonical pair keys and its multipliers and decay factors, for
  teacher-forced steps;
- `stats`: per step outer iterations, CG iterations and active pairs.

Run from the repository root:  python tests/golden/make_eight_cubes_oracle.py
(about four minutes on one core)."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2512_12151_b300 import scenes  # noqa: E402

N_STEPS = 24
STATE_STEP = 16


def main():
    O.build()
    s = scenes.eight_cubes(0)
    free = np.flatnonzero(s.dirichlet == 0)
    ids = np.sort(np.random.default_rng(2024).choice(free, 1024, replace=False))
    o = O.Oracle(s)
    traj = np.zeros((N_STEPS, len(ids), 3))
    stats = np.zeros((N_STEPS, 3), np.int64)
    out = {}
    t0 = time.time()
    for i in range(N_STEPS):
        status, st = o.step(1)
        assert status == 0, (i, status)
        x, v = o.get_state()
        traj[i] = x[ids]
        stats[i] = (st[0]["outer_iters"], st[0]["cg_iters"], st[0]["n_contacts"])
        if i + 1 == STATE_STEP:
            keys, lam, gam = o.active_get()
            out.update(x16=x, v16=v, keys16=keys, lam16=lam, gam16=gam)
        print(f"step {i}: {st[0]['outer_iters']} outer, {st[0]['n_contacts']} pairs, {time.time() - t0:.0f} s",
              flush=True)
    np.savez_compressed(os.path.join(os.path.dirname(os.path.abspath(__file__)), "eight_cubes_oracle.npz"),
                        sample_ids=ids, traj=traj, stats=stats, n_steps=N_STEPS, state_step=STATE_STEP, **out)


if __name__ == "__main__":
    main()
