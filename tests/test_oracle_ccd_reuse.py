"""Pins of the oracle's CCD-reuse option (ccd_reuse: the active set is
updated from the MaxStepSize segment x^[k] -> xhat^[k+1] instead of
Alg. 1's x^[k] -> xhat^[k]).  Without contact the option cannot matter: a
free fall is identical to Alg. 1 as printed.  With contact it changes only
which pairs join C when, so the invariants of the time step still hold:
momentum is conserved between free bodies (the AL contact forces are
internal) up to the termination threshold, every step is penetration-free,
and the pairs that cut a step are in C after it."""
import numpy as np
import pytest

import oracle as O
from paper_2512_12151_b300 import scenes


def test_free_fall_is_unchanged():
    runs = []
    for reuse in (0, 1):
        s = scenes.single_cube(seed=0, cells=2, z=0.5, with_ground=False)
        s.params.ccd_reuse = reuse
        o = O.Oracle(s)
        st, stats = o.step(3)
        assert st == 0
        runs.append((o.get_state(), [q["outer_iters"] for q in stats]))
    (xa, va), ia = runs[0]
    (xb, vb), ib = runs[1]
    assert ia == ib and np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_momentum_and_no_penetration_with_reuse():
    s = scenes.colliding_cubes(seed=0, cells=2, speed=1.0)
    s.params.ccd_reuse = 1
    o = O.Oracle(s)
    m = o.mass()
    P0 = (m[:, None] * s.v0).sum(0)
    nsteps = 6
    for _ in range(nsteps):
        st, stats = o.step(1)
        assert st == 0
        x, _ = o.get_state()
        assert o.min_distance(x) > 0
    assert stats[0]["n_contacts"] > 0
    _, v = o.get_state()
    P1 = (m[:, None] * v).sum(0)
    assert np.linalg.norm(P1 - P0) <= nsteps * (s.params.eps + 1e-5) * np.linalg.norm(P0)


def test_blocking_pairs_join_the_active_set_at_once():
    """one outer iteration by hand: after the update from the MaxStepSize
    segment, every pair whose TOI sets alpha is in C"""
    s = scenes.single_cube(seed=0, cells=2, z=0.012, with_ground=True, v0=(0.0, 0.0, -2.0))
    p = scenes.Params(**{**s.params.__dict__, "ccd_reuse": 1})
    o2 = O.Oracle(s, p)
    x, _ = o2.get_state()
    xt = o2.xtilde()
    o2.mu_init(x, xt)
    xh = o2.solve_subproblem(xt, x, x)[0]
    keys, toi = o2.ccd_hits(x, xh)
    assert len(keys) > 0
    o2.update_active_set(x, xh)
    C = {tuple(int(u) for u in k) for k in o2.active_get()[0]}
    a = min(toi)
    first = [tuple(int(u) for u in k) for k, t in zip(keys, toi) if t == a]
    assert o2.max_step_size(x, xh) == pytest.approx(a, abs=0)
    assert all(k in C for k in first)
