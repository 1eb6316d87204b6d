"""Pins of the oracle's gradient-norm residual (section 6: IPC's
(1/h) |H^-1 grad L|_inf) and of the residual-terminated time step.

The residual against a library dense solve of the assembled system at a
contact state and in closed form for free fall (a translation is in the
elastic Hessian's null space, so H^-1 grad L = x^t - x~); the residual mode
of the time step: one outer iteration for free fall (the step lands on
x~, where the residual vanishes), and on two colliding balls a log that
ends at the first value below the tolerance, agrees with the residual
recomputed at the result, and leaves a penetration-free state."""
import numpy as np
import pytest

import oracle as O
from paper_2512_12151_b300 import scenes


def test_free_fall_residual_closed_form():
    s = scenes.single_cube(seed=0, cells=2, z=0.5, with_ground=False)
    s.params.cg_tol = 1e-12
    s.v0[:] = np.array([0.3, -0.2, 0.5])
    o = O.Oracle(s)
    x, v = o.get_state()
    xt = o.xtilde()
    o.mu_init(x, xt)
    r = o.newton_residual(xt, x)
    h, g = s.params.dt, np.array(s.params.gravity)
    assert r == pytest.approx(np.abs(v[0] + h * g).max(), rel=1e-9)
    assert o.newton_residual(xt, xt) <= 1e-12  # at x~ the gradient vanishes


@pytest.fixture(scope="module")
def balls_state():
    s = scenes.colliding_balls(0)
    o = O.Oracle(s)
    st, _ = o.step(5)
    assert st == 0
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    assert len(keys) > 5
    return s, x, v, keys, lam, gam


def _oracle(state, **kw):
    s, x, v, keys, lam, gam = state
    p = scenes.Params(**{**s.params.__dict__, **kw})
    o = O.Oracle(s, p)
    o.set_state(x, v)
    o.active_set(keys, lam, gam)
    return o


def test_residual_matches_a_dense_solve(balls_state):
    x = balls_state[1]
    o = _oracle(balls_state, cg_tol=1e-12)
    xt = o.xtilde()
    o.mu_init(x, xt)
    r = o.newton_residual(xt, x)
    o.linearize(x)
    _, G = o.assemble(xt, x, x)
    H = o.hess_dense()
    p = np.linalg.solve(H, G.reshape(-1))
    assert r == pytest.approx(np.abs(p).max() / balls_state[0].params.dt, rel=1e-8)


def test_free_fall_step_in_residual_mode():
    s = scenes.single_cube(seed=0, cells=2, z=0.5, with_ground=False)
    s.params.res_tol = 1e-8
    s.params.cg_tol = 1e-12
    o = O.Oracle(s)
    st, stats = o.step(1)
    assert st == 0 and stats[0]["outer_iters"] == 1  # Eq. termination would need K_min = 2
    log = o.residual_log()
    h, g = s.params.dt, np.array(s.params.gravity)
    assert len(log) == 2 and log[0] == pytest.approx(np.abs(h * g).max(), rel=1e-9) and log[1] < 1e-8
    x, _ = o.get_state()
    assert np.abs(x - (s.x0 + h * h * g)).max() <= 1e-12


def test_residual_terminated_step_on_colliding_balls(balls_state):
    s, x0, v0 = balls_state[0], balls_state[1], balls_state[2]
    tol = 1e-6
    o = _oracle(balls_state, res_tol=tol)
    xt = o.xtilde()
    st, stats = o.step(1)
    assert st == 0
    log = o.residual_log()
    assert len(log) == stats[0]["outer_iters"] + 1
    assert log[-1] < tol and np.all(log[:-1] >= tol)
    assert log[0] > 1e3 * tol  # the state was far from converged
    x, _ = o.get_state()
    assert o.min_distance(x) > 0
    # the last entry is the residual at the result: recomputed from the
    # step's x~ with the final active set, multipliers, mu and delta
    keys, lam, gam = o.active_get()
    o2 = _oracle((s, x0, v0, keys, lam, gam))
    o2.set_mu_delta(stats[0]["mu"], stats[0]["delta"])
    assert o2.newton_residual(xt, x) == pytest.approx(log[-1], rel=1e-9)
