"""Pins of the oracle's Neo-Hookean material (NH, one of the models of
Tab. 2) and of the inversion-aware step bound that section 4.1 asks of
MaxStepSize for non-invertible materials.

NH: stress and Hessian by central differences of the energy, rotation
invariance, zero energy and stress at rest, the small-strain Hessian equal
to the linear elasticity tensor in closed form, +inf for inverted elements,
and the spectrum of the dense Hessian equal to the closed-form eigenvalues
of an isotropic energy written in the singular values (a second,
independent derivation).

Step bound: the cubic's first root against numpy's polynomial roots, the
cubic's coefficients against numpy determinants, and the bound of whole
motions against closed forms (uniform compression, one vertex crossing
its opposite faces, rigid motion) and against dense sampling of det F(t)."""
import numpy as np
import pytest

import oracle as O
from paper_2512_12151_b300 import scenes

MU, LAM = 2.0, 3.0


def rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


def vec(M):  # column-major, the oracle's 9-vector order
    return M.T.reshape(-1)


def random_F(rng, scale=0.3):
    while True:
        F = np.eye(3) + scale * rng.standard_normal((3, 3))
        if np.linalg.det(F) > 0.2:
            return F


def test_stress_and_hessian_by_differences():
    rng = np.random.default_rng(3)
    for _ in range(6):
        F = random_F(rng)
        P, H = O.nh_pk1(F, MU, LAM), O.nh_hess9(F, MU, LAM)
        eps = 1e-6
        for a in range(3):
            for b in range(3):
                E = np.zeros((3, 3))
                E[a, b] = eps
                fd = (O.nh_psi(F + E, MU, LAM) - O.nh_psi(F - E, MU, LAM)) / (2 * eps)
                assert fd == pytest.approx(P[a, b], abs=1e-8 * np.abs(P).max())
                dP = (O.nh_pk1(F + E, MU, LAM) - O.nh_pk1(F - E, MU, LAM)) / (2 * eps)
                assert np.abs(vec(dP) - H[:, a + 3 * b]).max() <= 1e-7 * np.abs(H).max()
        assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


def test_rotation_invariance_and_rest_state():
    rng = np.random.default_rng(1)
    F = random_F(rng, 0.2)
    for _ in range(3):
        Q = rotation(rng)
        assert O.nh_psi(Q @ F, MU, LAM) == pytest.approx(O.nh_psi(F, MU, LAM), rel=1e-12)
        assert np.abs(O.nh_pk1(Q @ F, MU, LAM) - Q @ O.nh_pk1(F, MU, LAM)).max() <= 1e-12
        assert abs(O.nh_psi(Q, MU, LAM)) <= 1e-14 and np.abs(O.nh_pk1(Q, MU, LAM)).max() <= 1e-12


def test_small_strain_hessian_is_the_linear_elasticity_tensor():
    """d2Psi/dF2 at F = I: 2 mu (symmetrisation) + lam vec(I) vec(I)^T"""
    H = O.nh_hess9(np.eye(3), MU, LAM)
    sym = np.zeros((9, 9))
    for a in range(3):
        for b in range(3):
            E = np.zeros((3, 3))
            E[a, b] = 1.0
            sym[:, a + 3 * b] = vec(0.5 * (E + E.T))
    ref = 2 * MU * sym + LAM * np.outer(vec(np.eye(3)), vec(np.eye(3)))
    assert np.abs(H - ref).max() <= 1e-12


def test_inverted_and_degenerate_elements_have_infinite_energy():
    F = np.diag([1.0, 1.0, -0.5])
    assert O.nh_psi(F, MU, LAM) == np.inf
    assert O.nh_psi(np.diag([1.0, 1.0, 0.0]), MU, LAM) == np.inf
    vals = [O.nh_psi(np.diag([1.0, 1.0, j]), MU, LAM) for j in (1e-2, 1e-4, 1e-8)]
    assert vals[0] < vals[1] < vals[2] and vals[2] > 100 * MU


def test_spectrum_matches_the_singular_value_eigensystem():
    """For Psi(s1, s2, s3) isotropic, d2Psi/dF2 has the eigenvalues of the
    3x3 block d2Psi/ds_i ds_j and, per axis pair (i, j), (Psi_i - Psi_j) /
    (s_i - s_j) and (Psi_i + Psi_j) / (s_i + s_j).  With NH written in the
    singular values these are mu + (mu - lam ln J) / (s_i s_j) and
    mu + (lam ln J - mu) / (s_i s_j)."""
    rng = np.random.default_rng(11)
    for _ in range(5):
        F = random_F(rng, 0.4)
        s = np.linalg.svd(F, compute_uv=False)
        L = np.log(np.prod(s))
        # d2Psi/ds_i ds_j = lam / (s_i s_j) + [i = j] (mu + (mu - lam ln J) / s_i^2)
        S3 = np.array([[LAM / (s[i] * s[j]) + (MU + (MU - LAM * L) / s[i] ** 2 if i == j else 0.0)
                        for j in range(3)] for i in range(3)])
        ev = list(np.linalg.eigvalsh(S3))
        for i, j in ((0, 1), (0, 2), (1, 2)):
            ev += [MU + (MU - LAM * L) / (s[i] * s[j]), MU + (LAM * L - MU) / (s[i] * s[j])]
        got = np.linalg.eigvalsh(O.nh_hess9(F, MU, LAM))
        assert np.abs(np.sort(ev) - got).max() <= 1e-10 * np.abs(got).max()


def test_element_gradient_by_differences_and_psd_projection():
    rng = np.random.default_rng(5)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]) * 0.1
    Dm = (X[1:] - X[0]).T
    B = np.linalg.inv(Dm)
    vol = np.linalg.det(Dm) / 6
    x = (X + 0.01 * rng.standard_normal(X.shape)).reshape(-1)
    psi, g, H = O.elem_grad_hess(x, B.reshape(-1), vol, MU, LAM, project=True, model=2)
    eps = 1e-7
    for k in range(12):
        d = np.zeros(12)
        d[k] = eps
        fd = (O.elem_grad_hess(x + d, B.reshape(-1), vol, MU, LAM, model=2)[0] -
              O.elem_grad_hess(x - d, B.reshape(-1), vol, MU, LAM, model=2)[0]) / (2 * eps)
        assert fd == pytest.approx(g[k], abs=1e-7 * np.abs(g).max())
    assert np.linalg.eigvalsh(H).min() >= -1e-10 * np.abs(H).max()


# ---------------- the inversion-aware step bound ----------------
def test_cubic_first_root_against_numpy_roots():
    rng = np.random.default_rng(2)
    hits = 0
    for _ in range(2000):
        c = rng.standard_normal(4)
        c[0] = abs(c[0]) + 1e-3
        if rng.random() < 0.2:
            c[3] = 0.0  # quadratics
        r = np.roots(c[::-1])
        real = [t.real for t in r if abs(t.imag) <= 1e-9 * max(1.0, abs(t)) and 0.0 < t.real <= 1.0]
        got = O.cubic_first_root(c)
        if real:
            hits += 1
            assert got == pytest.approx(min(real), abs=1e-7)
            p = np.polyval(c[::-1], got)
            assert p > 0 or abs(p) <= 1e-12
        else:
            assert got == 1.0 or np.polyval(c[::-1], got) <= 1e-9  # a double root grazing zero
    assert hits > 300


def test_cubic_first_root_special_cases():
    assert O.cubic_first_root([1.0, 0.0, 0.0, 0.0]) == 1.0
    assert O.cubic_first_root([1.0, -2.0, 0.0, 0.0]) == pytest.approx(0.5, abs=1e-15)
    assert O.cubic_first_root([1.0, -1.0, 0.0, 0.0]) == pytest.approx(1.0, abs=1e-15)
    assert O.cubic_first_root([0.0, 1.0, 0.0, 0.0]) == 0.0  # no positive start: no step
    # (1 - 4 t)^2 (1 + t): a double root at 1/4 is reached, not skipped
    c = np.polynomial.polynomial.polymul(np.polynomial.polynomial.polymul([1, -4], [1, -4]), [1, 1])
    assert O.cubic_first_root(c) == pytest.approx(0.25, abs=1e-7)


def test_det_cubic_against_numpy_determinants():
    rng = np.random.default_rng(4)
    for _ in range(20):
        A, Bm = rng.standard_normal((3, 3)), rng.standard_normal((3, 3))
        s = rng.random()
        c = O.det_cubic(A, Bm, s)
        for t in (-1.3, 0.0, 0.4, 1.0, 2.5):
            ref = np.linalg.det(A + t * Bm) - s * np.linalg.det(A)
            assert np.polyval(c[::-1], t) == pytest.approx(ref, abs=1e-12 * (1 + abs(t)) ** 3 * 10)


def _cube():
    s = scenes.single_cube(seed=0, cells=2, z=0.5, with_ground=False)
    s.params.model = 2
    return s


def _J(s, x):
    x = x.reshape(-1, 3)
    Ds = np.stack([x[s.tets[:, k]] - x[s.tets[:, 0]] for k in (1, 2, 3)], axis=2)
    R = s.rest
    Dm = np.stack([R[s.tets[:, k]] - R[s.tets[:, 0]] for k in (1, 2, 3)], axis=2)
    return np.linalg.det(Ds) / np.linalg.det(Dm)


def test_inversion_bound_uniform_compression_closed_form():
    """x(t) = c + (1 - t k)(x0 - c): J(t) = (1 - t k)^3 J(0), so the bound is
    (1 - s^(1/3)) / k"""
    s = _cube()
    o = O.Oracle(s)
    c = s.x0.mean(axis=0)
    for k in (1.5, 2.0, 0.95):
        x1 = c + (1.0 - k) * (s.x0 - c)
        exp = min(1.0, (1.0 - s.params.s_ccd ** (1.0 / 3.0)) / k)
        assert o.inversion_step(s.x0, x1) == pytest.approx(exp, abs=1e-12)
    x1 = c + 0.5 * (s.x0 - c)  # k = 0.5: the volume falls to 1/8 > s of its start
    assert o.inversion_step(s.x0, x1) == 1.0


def test_inversion_bound_single_vertex_and_rigid_motion():
    """Moving one vertex changes det F linearly in t (matrix determinant
    lemma), so each element it touches bounds t by (1 - s) J0 / (J0 - J1)."""
    s = _cube()
    o = O.Oracle(s)
    rng = np.random.default_rng(9)
    sp = s.params.s_ccd
    for v in rng.choice(s.nv, 4, replace=False):
        x1 = s.x0.copy()
        x1[v] += 0.3 * rng.standard_normal(3)
        J0, J1 = _J(s, s.x0), _J(s, x1)
        lim = [(1 - sp) * a / (a - b) for a, b in zip(J0, J1) if b < sp * a]
        exp = min([1.0] + [t for t in lim if t <= 1.0])
        assert o.inversion_step(s.x0, x1) == pytest.approx(exp, abs=1e-12)
    # rotation by th plus a translation: F(t) = (1 - t) I + t Q has
    # det >= cos^2(th / 2) > s on the chord, so nothing bounds the step
    th = np.pi / 6
    Q = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    x1 = (s.x0 - s.x0.mean(axis=0)) @ Q.T + s.x0.mean(axis=0) + 0.2
    assert o.inversion_step(s.x0, x1) == 1.0


def test_inversion_bound_against_dense_sampling():
    s = _cube()
    o = O.Oracle(s)
    rng = np.random.default_rng(6)
    ts = np.linspace(0.0, 1.0, 20001)
    for trial in range(4):
        x1 = s.x0 + 0.04 * rng.standard_normal(s.x0.shape)
        got = o.inversion_step(s.x0, x1)
        J0 = _J(s, s.x0)
        below = None
        for t in ts:
            if np.any(_J(s, s.x0 + t * (x1 - s.x0)) <= s.params.s_ccd * J0):
                below = t
                break
        if below is None:
            assert got == 1.0
        else:
            assert below - 1.0 / 20000 - 1e-12 <= got <= below


def test_free_fall_with_nh():
    """translation keeps F = I, so one step of free fall lands on
    x + h v + h^2 g as with SNH (exactly 2 outer iterations)"""
    s = _cube()
    o = O.Oracle(s)
    st, stats = o.step(1)
    assert st == 0 and stats[0]["outer_iters"] == 2
    x, v = o.get_state()
    h, g = s.params.dt, np.array(s.params.gravity)
    assert np.abs(x - (s.x0 + h * s.v0 + h * h * g)).max() <= 1e-9


def _implosion():
    s = scenes.single_cube(seed=0, cells=3, z=0.5, with_ground=False, gravity=(0, 0, 0))
    s.mats[:, 0] = 1e3
    s.params.model = 2
    c = s.x0.mean(axis=0)
    s.v0[:] = -300.0 * (s.x0 - c)
    return s


def test_max_step_size_is_the_smaller_of_ccd_and_inversion_bounds():
    """A soft NH cube given an inward velocity field v = -k (x - c) whose
    inertial target x~ = x + h v is inverted.  Along the outer loop of
    Alg. 1, MaxStepSize equals min(1, CCD's minimum TOI, the inversion
    bound), and the inversion bound decides some of the steps."""
    s = _implosion()
    o = O.Oracle(s)
    x, _ = o.get_state()
    xt = o.xtilde()
    xk, xh = x.copy(), x.copy()
    o.mu_init(xh, xt)
    decided = 0
    for k in range(3):
        xhn = o.solve_subproblem(xt, xk, xh)[0]
        o.update_active_set(xk, xh)
        a = o.max_step_size(xk, xhn)
        _, toi = o.ccd_hits(xk, xhn)
        ac = min([1.0] + list(toi))
        ai = o.inversion_step(xk, xhn)
        assert a == min(ac, ai)
        decided += ai < ac
        xk = (1 - a) * xk + a * xhn
        xh = xhn
        assert _J(s, xk).min() > 0.0
    assert decided >= 1


def test_implosion_stays_inversion_free():
    """The same scene through whole time steps: every element keeps J > 0
    at the end of every step (SNH, invertible, has no such bound)."""
    s = _implosion()
    o = O.Oracle(s)
    for _ in range(3):
        st, stats = o.step(1)
        assert st == 0
        x, _ = o.get_state()
        assert _J(s, x).min() > 0.0
