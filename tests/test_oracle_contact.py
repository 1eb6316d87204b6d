"""Pins of the oracle's distances and additive CCD against brute force and
closed forms (section 4.2 distances d_i, section 5.1 ACCD narrow phase)."""
import json
import os

import numpy as np
import pytest
from scipy.optimize import minimize

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_pt(p, a, b, c, n=200):
    u = np.linspace(0, 1, n)
    U, V = np.meshgrid(u, u, indexing="ij")
    m = U + V <= 1
    Q = a[None] + U[m][:, None] * (b - a)[None] + V[m][:, None] * (c - a)[None]
    d2 = ((Q - p) ** 2).sum(1)
    k = np.argmin(d2)

    def f(z):
        q = a + z[0] * (b - a) + z[1] * (c - a)
        return ((q - p) ** 2).sum()
    cons = [{"type": "ineq", "fun": lambda z: z[0]}, {"type": "ineq", "fun": lambda z: z[1]},
            {"type": "ineq", "fun": lambda z: 1 - z[0] - z[1]}]
    r = minimize(f, [U[m][k], V[m][k]], method="SLSQP", constraints=cons,
                 options={"ftol": 1e-16, "maxiter": 500})
    uu, vv = np.clip(r.x, 0, 1)
    if uu + vv > 1:
        uu, vv = uu / (uu + vv), vv / (uu + vv)
    return min(d2[k], f([uu, vv]))


def brute_ee(a0, a1, b0, b1, n=400):
    s = np.linspace(0, 1, n)
    P = a0[None] + s[:, None] * (a1 - a0)[None]
    Q = b0[None] + s[:, None] * (b1 - b0)[None]
    d2 = ((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1)
    i, j = np.unravel_index(np.argmin(d2), d2.shape)

    def f(z):
        ss, tt = np.clip(z, 0, 1)
        return ((a0 + ss * (a1 - a0) - b0 - tt * (b1 - b0)) ** 2).sum()
    r = minimize(f, [s[i], s[j]], method="L-BFGS-B", bounds=[(0, 1), (0, 1)],
                 options={"ftol": 1e-16, "gtol": 1e-14, "maxiter": 500})
    return min(d2[i, j], f(r.x))


def test_pt_distance_brute_force(rng):
    for _ in range(40):
        a, b, c = rng.standard_normal((3, 3))
        p = rng.standard_normal(3) * 1.5
        d2 = O.pt_dist2(p, a, b, c)
        ref = brute_pt(p, a, b, c)
        assert d2 <= ref * (1 + 1e-9) + 1e-15
        assert d2 >= ref * (1 - 1e-6) - 1e-12


def test_ee_distance_brute_force(rng):
    for k in range(40):
        a0, a1, b0, b1 = rng.standard_normal((4, 3))
        if k % 5 == 0:  # (nearly) parallel pairs
            b1 = b0 + (a1 - a0) * rng.uniform(0.3, 2) + 1e-12 * rng.standard_normal(3)
        d2 = O.ee_dist2(a0, a1, b0, b1)
        ref = brute_ee(a0, a1, b0, b1)
        assert d2 <= ref * (1 + 1e-9) + 1e-15
        assert d2 >= ref * (1 - 1e-6) - 1e-12


def test_distance_special_cases():
    a, b, c = np.array([0, 0, 0.]), np.array([1, 0, 0.]), np.array([0, 1, 0.])
    assert O.pt_dist2(np.array([0.2, 0.2, 0.5]), a, b, c) == pytest.approx(0.25, rel=1e-15)  # face region
    assert O.pt_dist2(np.array([-1, -1, 0.]), a, b, c) == pytest.approx(2.0, rel=1e-15)      # vertex region
    assert O.pt_dist2(np.array([0.5, -2, 1.]), a, b, c) == pytest.approx(5.0, rel=1e-15)     # edge region
    # skew segments crossing at distance 1; collinear disjoint segments
    assert O.ee_dist2(np.array([-1, 0, 0.]), np.array([1, 0, 0.]), np.array([0, -1, 1.]), np.array([0, 1, 1.])) == pytest.approx(1.0)
    assert O.ee_dist2(np.array([0, 0, 0.]), np.array([1, 0, 0.]), np.array([3, 0, 0.]), np.array([4, 0, 0.])) == pytest.approx(4.0)


@pytest.mark.parametrize("ptype", [0, 1])
def test_distance_gradient_fd_and_translation(rng, ptype):
    for _ in range(30):
        x = rng.standard_normal(12)
        d, g = O.pair_dist_grad(ptype, x)
        h = 1e-7
        gfd = np.zeros(12)
        for k in range(12):
            xp, xm = x.copy(), x.copy()
            xp[k] += h
            xm[k] -= h
            gfd[k] = (O.pair_dist_grad(ptype, xp)[0] - O.pair_dist_grad(ptype, xm)[0]) / (2 * h)
        assert np.abs(g - gfd).max() <= 1e-5
        assert np.abs(g.reshape(4, 3).sum(0)).max() <= 1e-12
        assert d == pytest.approx(np.sqrt((O.pt_dist2 if ptype == 0 else O.ee_dist2)(*x.reshape(4, 3))), rel=1e-15)


def _dist(ptype, x):
    f = O.pt_dist2 if ptype == 0 else O.ee_dist2
    return np.sqrt(f(*np.asarray(x).reshape(4, 3)))


def test_accd_golden_closed_forms():
    """Closed-form cases (tests/golden/accd_closed_form.json): a point moving
    head-on toward a static triangle at constant speed v from distance d0
    reaches s*d0 at t* = (1 - s) d0 / v; ACCD's bound l_p equals v there,
    so its first step lands exactly on t*."""
    with open(os.path.join(GOLDEN, "accd_closed_form.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        x0 = np.array(c["x0"], float)
        x1 = np.array(c["x1"], float)
        t = O.accd(c["type"], x0, x1, s=c["s"])
        if c["t_star"] is None:
            assert t == np.inf
        else:
            assert t <= c["t_star"] * (1 + 1e-12)
            assert t >= c["t_star"] * (1 - 1e-12)


@pytest.mark.parametrize("ptype", [0, 1])
def test_accd_conservative_vs_bracketing(rng, ptype):
    s = 0.1
    nhit = 0
    for k in range(60):
        x0 = rng.standard_normal(12) * 0.1
        x1 = x0 + rng.standard_normal(12) * 0.15
        if k % 2 == 0:  # drive the first primitive through the second
            na = 1 if ptype == 0 else 2
            shift = x0.reshape(4, 3)[na:].mean(0) - x0.reshape(4, 3)[:na].mean(0)
            x1 = x1.reshape(4, 3)
            x1[:na] += 1.5 * shift
            x1 = x1.reshape(-1)
        t = O.accd(ptype, x0, x1, s=s)
        d0 = _dist(ptype, x0)
        ts = np.linspace(0, 1, 20001)
        ds = np.array([_dist(ptype, x0 + tt * (x1 - x0)) for tt in ts])
        below = np.nonzero(ds <= s * d0)[0]
        if t < np.inf:
            nhit += 1
            assert 0 < t <= 1
            # conservative: the gap at t is still at least s*d0 and no
            # sample before t went below s*d0
            assert _dist(ptype, x0 + t * (x1 - x0)) >= s * d0 * (1 - 1e-9)
            assert len(below) == 0 or ts[below[0]] >= t - 1e-4
        else:
            assert len(below) == 0  # no hit => distance never fell to s*d0
    assert nhit > 5


def test_accd_static_and_separating(rng):
    x0 = rng.standard_normal(12)
    assert O.accd(0, x0, x0) == np.inf  # no relative motion
    x1 = x0 + np.tile(rng.standard_normal(3), 4)  # pure translation
    assert O.accd(1, x0, x1) == np.inf
