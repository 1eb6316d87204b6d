"""Pins of the oracle's semi-implicit friction (appendix A): the smoothed
norm's boundary values and smoothness, the friction energy's gradient and
Hessian by central differences, the normal-force coefficients against the
weight of a block resting on an incline, sliding on the incline at the
closed-form acceleration g (sin theta - mu_f cos theta) (the paper's
sliding-friction test), sticking below the slip threshold, and momentum
conservation with friction between free bodies."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2512_12151_b300 import scenes

TH = math.atan(0.5)


def test_f0_boundary_values_and_smoothness():
    eh = 1e-5
    # f0(0) = eh/3 with zero slope and curvature 2/eh; f0(y) = y from eh on
    f0, f1, f2 = O.friction_f0(0.0, eh)
    assert f0 == pytest.approx(eh / 3, rel=1e-15) and f1 == 0.0 and f2 == pytest.approx(2 / eh, rel=1e-15)
    for y in (eh, 2 * eh, 1.0):
        f0, f1, f2 = O.friction_f0(y, eh)
        assert (f0, f1, f2) == (y, 1.0, 0.0)
    # C^2 at eh: value, slope and curvature match from below
    f0, f1, f2 = O.friction_f0(eh * (1 - 1e-9), eh)
    assert f0 == pytest.approx(eh, rel=1e-8) and f1 == pytest.approx(1.0, abs=1e-8) and abs(f2) <= 1e-8 / eh * 10
    # derivatives by central differences inside the smoothed region
    for y in np.linspace(0.05, 0.95, 7) * eh:
        d = 1e-6 * eh
        assert (O.friction_f0(y + d, eh)[0] - O.friction_f0(y - d, eh)[0]) / (2 * d) == pytest.approx(
            O.friction_f0(y, eh)[1], rel=1e-7)
        assert (O.friction_f0(y + d, eh)[1] - O.friction_f0(y - d, eh)[1]) / (2 * d) == pytest.approx(
            O.friction_f0(y, eh)[2], rel=1e-6)
        assert O.friction_f0(y, eh)[2] >= 0 and O.friction_f0(y, eh)[1] >= 0  # PSD in u as it stands


@pytest.fixture(scope="module")
def resting_block():
    """a block settled on the incline with mu_f above the slip threshold"""
    s = scenes.slope_cube(0.6, n_steps=30)
    o = O.Oracle(s)
    st, _ = o.step(30)
    assert st == 0
    return s, o


def test_normal_force_coefficients_match_the_weight(resting_block):
    """at rest the pairs' normal forces carry the weight's normal part:
    sum_i k_i = mu_f h^2 m g cos(theta) (the h^2 of the incremental
    potential)"""
    s, o = resting_block
    o.friction_setup()
    v4, w4, n3, k = o.friction_get()
    m = float(o.mass()[s.dirichlet == 0].sum())
    assert len(k) > 4 and np.abs(n3[:, 2]).min() > 1 - 1e-9  # normals of the incline
    assert k.sum() == pytest.approx(0.6 * s.params.dt ** 2 * m * 9.8 * math.cos(TH), rel=1e-3)


def test_friction_gradient_and_hessian_by_differences(resting_block):
    s, o = resting_block
    nf = o.friction_setup()
    v4, w4, _, _ = o.friction_get()
    x, _ = o.get_state()
    free = (s.dirichlet == 0)[:, None]
    eh = s.params.dt * s.params.eps_v
    rng = np.random.default_rng(0)
    for scale in (0.1 * eh, 3 * eh, 100 * eh):  # inside, near and far beyond the smoothed region
        xh = x + scale * rng.standard_normal(x.shape) * free
        E, g, A = o.friction_eval(xh)
        dv = rng.standard_normal(x.shape) * free
        eps = 1e-4 * scale
        Ep, gp, _ = o.friction_eval(xh + eps * dv)
        Em, gm, _ = o.friction_eval(xh - eps * dv)
        assert (Ep - Em) / (2 * eps) == pytest.approx((g * dv).sum(), rel=1e-6)
        Hv = np.zeros_like(x)  # block (a, b) of pair j is w_a w_b A_j
        for j in range(nf):
            y = A[j] @ sum(w4[j, a] * dv[v4[j, a]] for a in range(4))
            for a in range(4):
                Hv[v4[j, a]] += w4[j, a] * y
        assert np.linalg.norm((gp - gm) / (2 * eps) - Hv) <= 1e-6 * np.linalg.norm(Hv)
        assert all(np.linalg.eigvalsh(Aj).min() >= -1e-12 * np.abs(Aj).max() for Aj in A)


def test_block_sticks_below_the_slip_threshold(resting_block):
    """mu_f = 0.6 > tan(theta) = 0.5: the block only creeps, slower than
    eps_v (the smoothed friction gives way below that velocity)"""
    s, o = resting_block
    _, v = o.get_state()
    assert np.abs(v[s.dirichlet == 0, 0]).max() <= s.params.eps_v


def test_block_slides_at_the_closed_form_acceleration():
    """mu_f = 0.2 < tan(theta): a = -g (sin theta - mu_f cos theta) along x
    once sliding (h = 2.5 ms; at h = 10 ms the lagged normal force lets this
    stiff block rock, see the design notes)"""
    mu, h = 0.2, 0.0025
    s = scenes.slope_cube(mu, n_steps=240)
    s.params.dt = h
    o = O.Oracle(s)
    free = s.dirichlet == 0
    vx = []
    for _ in range(240):
        st, _ = o.step(1)
        assert st == 0
        vx.append(o.get_state()[1][free, 0].mean())
    a = (vx[239] - vx[79]) / (160 * h)
    assert a == pytest.approx(-9.8 * (math.sin(TH) - mu * math.cos(TH)), rel=0.05)


def test_momentum_conserved_with_friction():
    """g = 0, two free bodies in frictional contact: friction is internal,
    so the momentum bound of the frictionless case holds"""
    s = scenes.colliding_cubes(seed=0, cells=2, speed=1.0)
    s.params.mu_f, s.params.k_min = 0.5, 6
    s.v0[:, 2] += 0.3 * (s.x0[:, 0] < s.x0[:, 0].mean())  # a tangential component for friction to act on
    o = O.Oracle(s)
    m = o.mass()
    P0 = (m[:, None] * s.v0).sum(0)
    nsteps = 8
    status, st = o.step(nsteps)
    assert status == 0 and max(x["n_contacts"] for x in st) > 0
    _, v = o.get_state()
    P1 = (m[:, None] * v).sum(0)
    assert np.linalg.norm(P1 - P0) <= nsteps * (s.params.eps + 1e-5) * np.linalg.norm(P0)
