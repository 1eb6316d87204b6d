"""Pins of the oracle's Newton / AL / active-set / time-stepping logic
(Alg. 1-3) against facts fixed outside it: finite differences of the
assembled gradient, a dense direct solve, an independent KKT solve (SLSQP),
closed forms (free fall, beta products, moving-boundary bound, decay count)
and invariants (momentum, penetration-free states)."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle as O
from paper_2512_12151_b300 import scenes


def two_cube_contact_state(seed=0):
    """Run the oracle to the first contact step and return it."""
    s = scenes.two_cubes(seed)
    o = O.Oracle(s)
    o.step(5)
    return s, o


def stretched_state(s, o):
    """x = c X with c^3 = 1 + mu/lam: every element's 9x9 Hessian is then
    positive definite, so the PSD projection is the identity."""
    mu, lam = O.lame(*s.mats[0, :2])
    c = (1 + mu / lam) ** (1 / 3)
    x = s.rest.copy()
    x[s.dirichlet == 0] *= c
    return x


def test_assembled_hessian_is_gradient_jacobian():
    s, o = two_cube_contact_state()
    keys, lam, gam = o.active_get()
    assert len(keys) > 20
    x = stretched_state(s, o)
    xt = o.xtilde()
    o.set_mu_delta(50.0, 1e-3)
    # large multipliers: every constraint active (s_i = 0), so the AL
    # gradient is linear in xhat with Jacobian mu gamma g g^T
    o.active_set(keys, np.full(len(keys), 10.0), np.full(len(keys), 0.7))
    o.linearize(x)
    rng = np.random.default_rng(3)
    xh = x + 1e-5 * rng.standard_normal(x.shape) * (s.dirichlet == 0)[:, None]
    E, g = o.assemble(xt, x, xh)
    H = o.hess_dense()
    assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    free = np.repeat(s.dirichlet == 0, 3)
    h = 1e-7
    cols = np.nonzero(free)[0][::7]
    for j in cols:
        xp, xm = xh.reshape(-1).copy(), xh.reshape(-1).copy()
        xp[j] += h
        xm[j] -= h
        gp = o.assemble(xt, x, xp.reshape(-1, 3))[1].reshape(-1)
        gm = o.assemble(xt, x, xm.reshape(-1, 3))[1].reshape(-1)
        col = (gp - gm) / (2 * h)
        assert np.abs(col[free] - H[free, j]).max() <= 1e-5 * np.abs(H[free, j]).max()
        assert np.abs(col[~free]).max() == 0.0  # eliminated DoFs: zero gradient
    o.assemble(xt, x, xh)
    # eliminated DoFs: rows and columns zero except the diagonal (section 5.3)
    Hd = H[~free][:, ~free]
    assert np.abs(H[~free][:, free]).max() == 0.0 and np.abs(H[free][:, ~free]).max() == 0.0
    assert np.allclose(Hd, np.diag(np.diag(Hd)))


def test_pcg_matches_dense_solve():
    s, o = two_cube_contact_state()
    x, _ = o.get_state()
    xt = o.xtilde()
    o.mu_init(x, xt)
    o.linearize(x)
    E, g = o.assemble(xt, x, x)
    H = o.hess_dense()
    b = -g.reshape(-1)
    ref = np.linalg.solve(H, b)
    for tol in (1e-6, 1e-10):
        p, it = o.pcg(-g, tol=tol, maxit=100000)
        assert it > 0
        p = p.reshape(-1)
        assert np.linalg.norm(H @ p - b) <= tol * np.linalg.norm(b) * (1 + 1e-6)
        kappa = np.linalg.cond(H)
        assert np.linalg.norm(p - ref) <= tol * kappa * np.linalg.norm(ref)
    # a single free vertex system is solved exactly in one iteration
    assert o.pcg(np.zeros_like(g))[1] == 0


def test_al_subproblem_converges_to_kkt_point():
    """Repeated SolveSubproblem calls at fixed x, x~ and C (Alg. 2) drive
    xhat to the KKT point of Eq. sub-problem and lambda to its multipliers,
    computed here independently with SLSQP on min E s.t. c_i(xhat) >= 0."""
    # cube off the ground quad's diagonal: one point-triangle constraint per
    # bottom vertex, linearly independent, so the KKT multipliers are unique
    s = scenes.single_cube(seed=1, cells=1, z=0.004, with_ground=True, v0=(0, 0, -1.0), xy=(0.4, -0.4))
    o = O.Oracle(s)
    x, _ = o.get_state()
    xt = o.xtilde()
    keys, toi = o.ccd_hits(x, xt)
    keys = keys[keys[:, 0] == 0]
    assert len(keys) == 4
    o.active_set(keys, np.zeros(len(keys)), np.ones(len(keys)))
    o.mu_init(x, xt)
    xh = x.copy()
    for _ in range(300):
        xh, nn, cg, lsf = o.solve_subproblem(xt, x, xh)
    _, lam, gam = o.active_get()
    d, g = o.linearize(x)
    v4 = o.active_verts()
    m = o.mass()
    fidx = np.nonzero(s.dirichlet == 0)[0]
    mu_l, lam_l = O.lame(*s.mats[0, :2])
    h2, delta = s.params.dt ** 2, s.params.delta
    elems = []
    for t in s.tets:
        Dm = (s.rest[t[1:]] - s.rest[t[0]]).T
        elems.append((t, np.linalg.inv(Dm), np.linalg.det(Dm) / 6))

    def full(z):
        y = x.copy()
        y[fidx] = z.reshape(-1, 3)
        return y

    def energy(z):
        y = full(z)
        e = 0.5 * (m[fidx, None] * (y[fidx] - xt[fidx]) ** 2).sum()
        for t, Bi, vi in elems:
            e += h2 * O.elem_grad_hess(y[t].reshape(-1), Bi, vi, mu_l, lam_l, True)[0]
        return e

    def c_lin(z, i):
        y = full(z)
        return d[i] + float((g[i] * (y[v4[i]] - x[v4[i]]).reshape(-1)).sum()) - delta

    cons = [{"type": "ineq", "fun": (lambda z, i=i: c_lin(z, i))} for i in range(len(d))]
    r = minimize(energy, xh[fidx].reshape(-1), method="SLSQP", constraints=cons,
                 options={"ftol": 1e-16, "maxiter": 2000})
    diag = np.linalg.norm(s.x0.max(0) - s.x0.min(0))
    assert np.abs(full(r.x) - xh).max() <= 1e-7 * diag
    assert (lam >= 0).all()
    active = np.array([c_lin(r.x, i) for i in range(len(d))]) < 1e-9
    assert active.any()
    # KKT stationarity with the AL multipliers: grad E = sum_i lambda_i grad c_i
    gE = np.zeros_like(x)
    eps = 1e-7
    z0 = xh[fidx].reshape(-1)
    for j in range(len(z0)):
        zp, zm = z0.copy(), z0.copy()
        zp[j] += eps
        zm[j] -= eps
        gE[fidx[j // 3], j % 3] = (energy(zp) - energy(zm)) / (2 * eps)
    gc = np.zeros_like(x)
    for i in range(len(d)):
        np.add.at(gc, v4[i], lam[i] * g[i].reshape(4, 3))
    assert np.abs(gE[fidx] - gc[fidx]).max() <= 1e-5 * np.abs(gE[fidx]).max()


def test_free_fall_closed_form():
    """No contact: x~ is a rigid translation of the stress-free x^t, so the
    first Newton step lands on x~ and, with K_min = 2 and alpha = 1, the step
    ends after exactly 2 outer iterations (section 4.4)."""
    s = scenes.single_cube(seed=2, cells=2, v0=(0.3, -0.2, 0.5))
    o = O.Oracle(s)
    status, st = o.step(1)
    assert status == 0 and st[0]["outer_iters"] == 2
    x, v = o.get_state()
    h, g = s.params.dt, np.array(s.params.gravity)
    ref = s.x0 + h * s.v0 + h * h * g
    assert np.abs(x - ref).max() <= 1e-9
    assert np.abs(v - (s.v0 + h * g)).max() <= 1e-7


def test_momentum_conservation():
    """g = 0, no obstacles: each solved state has total momentum
    sum M xhat = sum M x~, so the blend keeps (1 - beta_0) of P^t:
    |P^{t+1} - P^t| <= eps |P^t| up to the CG tolerance."""
    s = scenes.colliding_cubes(seed=0, cells=2, speed=1.0)
    o = O.Oracle(s)
    m = o.mass()
    P0 = (m[:, None] * s.v0).sum(0)
    nsteps = 6
    status, st = o.step(nsteps)
    assert status == 0
    assert max(x["n_contacts"] for x in st) > 0
    x, v = o.get_state()
    P1 = (m[:, None] * v).sum(0)
    assert np.linalg.norm(P1 - P0) <= nsteps * (s.params.eps + 1e-5) * np.linalg.norm(P0)


def test_constraint_decay_removes_after_44_inactive_subproblems():
    s = scenes.single_cube(seed=0, cells=1, z=0.5, with_ground=True)
    o = O.Oracle(s)
    x, _ = o.get_state()
    xt = o.xtilde()
    keys, _ = o.ccd_hits(x, x - np.array([0, 0, 0.6]) * (s.dirichlet == 0)[:, None])
    assert len(keys)
    o.active_set(keys[:1], np.zeros(1), np.ones(1))
    o.mu_init(x, xt)
    for k in range(1, 60):
        xh, *_ = o.solve_subproblem(xt, x, x.copy())
        n = o.update_active_set(x, x)
        assert (n == 1) == (k < 44), k
    assert 0.9 ** 43 >= 0.01 > 0.9 ** 44


def test_broad_phase_sweep_equals_brute_force():
    s, o = two_cube_contact_state(1)
    x, v = o.get_state()
    rng = np.random.default_rng(0)
    x1 = x + 0.004 * rng.standard_normal(x.shape) * (s.dirichlet == 0)[:, None] - np.array([0, 0, 0.003])
    ka, ta = o.ccd_hits(x, x1, brute=True)
    kb, tb = o.ccd_hits(x, x1, brute=False)
    assert len(ka) > 10
    A = {tuple(k): t for k, t in zip(ka, ta)}
    B = {tuple(k): t for k, t in zip(kb, tb)}
    assert A == B


def _beta_weights(alphas):
    """beta_i^[K], i = 0..K, of the termination criterion written out from
    its definition: alpha^[i] times the product of (1 - alpha^[j]) for j > i,
    with alpha^[0] = 1 (so x^[K] = sum_i beta_i x_hat^[i], x_hat^[0] = x^t)"""
    a = np.concatenate([[1.0], alphas])
    K = len(alphas)
    return np.array([a[i] * np.prod(1.0 - a[i + 1:K + 1]) for i in range(K + 1)])


@pytest.mark.parametrize("k_min", [1, 2, 3])
def test_beta_expansion_and_termination(k_min):
    """Eq. termination from its definition, not from the loop's recurrence:
    x^[K] equals the weighted sum of x^t and the logged intermediate states
    x_hat^[i] with the weights beta_i^[K] computed from the logged step
    sizes; the weights sum to one; the reported beta is the total weight of
    the first K_min states (indices 0..K_min-1), below eps, while the same
    sum after K - 1 iterations was not (the loop could not stop earlier);
    and every step stays penetration-free (section 3 path constraint)."""
    s = scenes.two_cubes(0)
    p = scenes.Params(**{**s.params.__dict__, "k_min": k_min})
    o = O.Oracle(s, p)
    total = 0
    for step in range(8):
        xt, _ = o.get_state()
        status, st, alphas, xhats = o.step_logged()
        assert status == 0
        K = st[0]["outer_iters"]
        assert K >= k_min and (alphas > 0).all() and (alphas <= 1).all()
        w = _beta_weights(alphas)
        x, _ = o.get_state()
        recon = w[0] * xt + np.tensordot(w[1:], xhats, axes=1)
        assert np.abs(recon - x).max() <= 1e-12 * max(1.0, np.abs(x).max())
        assert abs(w.sum() - 1.0) <= 1e-12
        beta = w[:k_min].sum()
        assert abs(beta - st[0]["beta"]) <= 1e-14 and beta <= s.params.eps
        if K > k_min:  # with K = k_min the loop could not have stopped earlier anyway
            assert _beta_weights(alphas[:-1])[:k_min].sum() > s.params.eps
        assert o.min_distance(x) > 0
        total += K
    assert total > 16


def test_moving_boundary_error_bound():
    """Section 5.3: the prescribed vertices end within eps h v / (1 - eps)
    of their targets."""
    s = scenes.moving_plate(seed=0)
    o = O.Oracle(s)
    v = s.meta["plate_speed"]
    bound = s.params.eps * s.params.dt * v / (1 - s.params.eps)
    for step in range(6):
        tgt = scenes.plate_targets(s, step)
        o.set_dirichlet_targets(tgt)
        status, st = o.step(1)
        assert status == 0
        x, _ = o.get_state()
        err = np.abs(x[s.dirichlet == 1] - tgt).max()
        assert err <= bound * (1 + 1e-9)


def test_lumped_mass_and_mu_init_closed_form():
    """Unjittered 2^3-cell cube (side 0.1, Kuhn split) with a vanishing
    Young's modulus: every vertex mass is rho V_e / 4 summed over its tets,
    so the interior vertex (24 tets of volume h^3/6) weighs rho h^3 and the
    total is rho side^3; the Hessian diagonal is then the mass, and
    mu_init = 0.1 x max diagonal (section 5.2) = 0.1 rho h^3."""
    v, t = scenes.cube_mesh(2, 0.1)
    b = scenes._Builder()
    b.add_solid(v, t, 0)
    s = b.build("cube_2", [[1e-9, 0.3, 1000.0]], scenes.Params(), 1)
    o = O.Oracle(s)
    m = o.mass()
    h = 0.05
    assert np.isclose(m.sum(), 1000.0 * 0.1 ** 3, rtol=1e-12)
    center = 1 + 3 * 1 + 9 * 1
    assert np.isclose(m[center], 1000.0 * h ** 3, rtol=1e-12)
    assert m.argmax() == center
    # corners: rho h^3 / 4 on the two cell-diagonal corners, rho h^3 / 12 elsewhere
    corners = [0, 2, 6, 8, 18, 20, 24, 26]
    assert np.allclose(np.sort(m[corners] / (1000.0 * h ** 3)), [1 / 12] * 6 + [0.25] * 2, rtol=1e-12)
    x, _ = o.get_state()
    mu = o.mu_init(x, o.xtilde())
    assert np.isclose(mu, 0.1 * 1000.0 * h ** 3, rtol=1e-9)


def test_update_active_set_keeps_per_vertex_first_hits():
    """Alg. 3 on a hand-built case: one tet translating 0.2 m down through
    two stacked static quads (z = 0 and z = -0.05).  Its lowest vertex a
    meets the upper quad first (t ~ 0.1), the others b, c, d later (t ~ 0.5);
    all meet the lower quad later still.  Filter: a new pair stays iff its
    TOI is the minimum over the pairs of one of its vertices.  Expected: the
    four pairs with the upper quad stay (each is its free vertex's first
    hit), (a, lower) stays (the lower quad's vertices are first hit by a),
    and (b|c|d, lower) are dropped (later than both their vertex's first
    hit and the lower quad's first hit)."""
    pa, pb, pc, pd = [0.5, -0.5, 0.02], [0.55, -0.5, 0.1], [0.5, -0.45, 0.1], [0.47, -0.53, 0.12]
    tv = np.array([pa, pb, pc, pd])
    tet = np.array([[0, 1, 2, 3]], np.int32)
    if np.linalg.det(tv[1:] - tv[0]) < 0:
        tet = np.array([[0, 2, 1, 3]], np.int32)
    b = scenes._Builder()
    b.add_solid(tv, tet, 0)
    gv, gt = scenes.ground_quad(1.0, 0.0)
    b.add_obstacle(gv, gt)  # vertices 4..7, triangle (4, 5, 6) under the tet
    lv, lt = scenes.ground_quad(1.0, -0.05)
    b.add_obstacle(lv, lt)  # vertices 8..11, triangle (8, 9, 10) under the tet
    s = b.build("tet_two_quads", [[1e5, 0.4, 1000.0]], scenes.Params(), 1)
    o = O.Oracle(s)
    x0 = s.x0.copy()
    x1 = x0.copy()
    x1[:4, 2] -= 0.2
    keys, toi = o.ccd_hits(x0, x1)
    got = {tuple(k) for k in keys.tolist()}
    upper = [(0, v, 4, 5, 6) for v in range(4)]
    lower = [(0, v, 8, 9, 10) for v in range(4)]
    assert got == set(upper + lower)  # every vertex crosses both quads, nothing else
    n = o.update_active_set(x0, x1)
    kept, lam, gam = o.active_get()
    assert n == 5
    assert {tuple(k) for k in kept.tolist()} == set(upper + lower[:1])
    assert (lam == 0).all() and (gam == 1).all()
