"""The eight-cube scene at full size (196,608 tets, 39,312 vertices) against
the FP64 oracle, per step, in mixed precision (FP32 Hessian blocks, SpMV and
preconditioner; FP64 CCD, TOIs, multipliers and PCG dots) and in FP64.

The oracle values come from `tests/golden/eight_cubes_oracle.npz`, written by
`tests/golden/make_eight_cubes_oracle.py` with the oracle alone: the state
after 16 steps from rest (cubes in contact, 6,292 active pairs) and the
positions of 1,024 sampled vertices after each of the first 24 steps.

- Teacher-forced: from the oracle's state at step 16, one GPU step and one
  oracle step (run here) land within 1e-4 x the bounding-box diagonal
  (mixed) and 1e-6 (FP64) of each other, at every vertex, with the same
  active set.
- Free-running: the GPU trajectory from rest, compared at the sampled
  vertices after every step with the oracle's; the per-step error curve is
  printed and bounded by 1e-4 x the diagonal (mixed)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2512_12151_b300 import binding as B
from paper_2512_12151_b300 import scenes

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "eight_cubes_oracle.npz")


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def golden():
    return dict(np.load(GOLDEN))


@pytest.fixture(scope="module")
def oracle_step16(golden):
    """the oracle's step 16 -> 17 from its own stored state"""
    s = scenes.eight_cubes(0)
    o = O.Oracle(s)
    o.set_state(golden["x16"], golden["v16"])
    o.active_set(golden["keys16"], golden["lam16"], golden["gam16"])
    status, st = o.step(1)
    assert status == 0
    x, v = o.get_state()
    keys, _, _ = o.active_get()
    # the stored trajectory is the same computation: sampled positions agree exactly
    assert np.array_equal(x[golden["sample_ids"]], golden["traj"][16])
    return x, keys, st[0]


@pytest.mark.parametrize("precision,tol", [(1, 1e-4), (0, 1e-6)])
def test_teacher_forced_contact_step(torch_cuda, golden, oracle_step16, precision, tol):
    xo, ko, st_o = oracle_step16
    s = scenes.eight_cubes(0, precision=precision)
    sim = B.Sim(s)
    B.bf_set_state(sim.h, golden["x16"], golden["v16"])
    B.bf_set_active_set(sim.h, golden["keys16"], golden["lam16"], golden["gam16"])
    _, st = sim.step(1)
    xg, _ = sim.state()
    kg, _, _ = B.bf_get_active_set(sim.h)
    sim.close()
    err = float(np.abs(xg - xo).max() / s.bbox_diag())
    print(f"precision {precision}: step 16 -> 17 max vertex error / bbox diagonal {err:.3e}, "
          f"outer iterations GPU {st[0]['outer_iters']} oracle {st_o['outer_iters']}")
    assert err <= tol
    assert {tuple(k) for k in kg.tolist()} == {tuple(k) for k in ko.tolist()}


def test_free_running_error_curve(torch_cuda, golden):
    s = scenes.eight_cubes(0, precision=1)
    ids, traj = golden["sample_ids"], golden["traj"]
    diag = s.bbox_diag()
    sim = B.Sim(s)
    errs = []
    for i in range(int(golden["n_steps"])):
        sim.step(1)
        xg, _ = sim.state()
        errs.append(float(np.abs(xg[ids] - traj[i]).max() / diag))
    sim.close()
    print("mixed precision, free-running from rest, max sampled-vertex error / bbox diagonal per step:",
          " ".join("%.2e" % e for e in errs))
    assert max(errs) <= 1e-4
