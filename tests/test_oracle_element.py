"""Pins of the oracle's element math (stable Neo-Hookean energy, its
derivatives, the PSD projection of section 5.1) against facts fixed outside
the oracle: finite differences, the linear-elasticity limit, rotation
invariance, numpy's symmetric eigensolver, and the analytic SVD-frame
eigensystem of the 9x9 Hessian derived independently here."""
import numpy as np
import pytest

import oracle as O

E, NU = 1e5, 0.4


def lame_textbook(E, nu):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


def rand_F(rng, scale=0.3, allow_inverted=False):
    F = np.eye(3) + scale * rng.standard_normal((3, 3))
    if not allow_inverted and np.linalg.det(F) <= 0.05:
        F[:, 0] *= -1
    return F


def vec_cm(M):
    """column-major vec (index r + 3c), the oracle's convention"""
    return M.T.reshape(-1)


def test_lame_shift():
    mu, lam = O.lame(E, NU)
    mu_t, lam_t = lame_textbook(E, NU)
    assert mu == pytest.approx(mu_t, rel=1e-15)
    assert lam == pytest.approx(lam_t + mu_t, rel=1e-15)


def test_rest_state_is_stress_free():
    mu, lam = O.lame(E, NU)
    assert O.snh_psi(np.eye(3), mu, lam) == 0.0
    assert np.abs(O.snh_pk1(np.eye(3), mu, lam)).max() == 0.0


@pytest.mark.parametrize("inv", [False, True])
def test_pk1_is_energy_gradient(rng, inv):
    mu, lam = O.lame(E, NU)
    for _ in range(20):
        F = rand_F(rng, 0.4, allow_inverted=inv)
        P = O.snh_pk1(F, mu, lam)
        h = 1e-6
        Pfd = np.zeros((3, 3))
        for r in range(3):
            for c in range(3):
                Fp, Fm = F.copy(), F.copy()
                Fp[r, c] += h
                Fm[r, c] -= h
                Pfd[r, c] = (O.snh_psi(Fp, mu, lam) - O.snh_psi(Fm, mu, lam)) / (2 * h)
        assert np.abs(P - Pfd).max() <= 1e-6 * np.abs(P).max() + 1e-3


@pytest.mark.parametrize("inv", [False, True])
def test_hess9_is_pk1_jacobian(rng, inv):
    mu, lam = O.lame(E, NU)
    for _ in range(20):
        F = rand_F(rng, 0.4, allow_inverted=inv)
        H = O.snh_hess9(F, mu, lam)
        h = 1e-6
        Hfd = np.zeros((9, 9))
        for r in range(3):
            for c in range(3):
                Fp, Fm = F.copy(), F.copy()
                Fp[r, c] += h
                Fm[r, c] -= h
                dP = (O.snh_pk1(Fp, mu, lam) - O.snh_pk1(Fm, mu, lam)) / (2 * h)
                Hfd[:, r + 3 * c] = vec_cm(dP)
        assert np.abs(H - Hfd).max() <= 1e-6 * np.abs(H).max()
        assert np.allclose(H, H.T, rtol=0, atol=1e-9 * np.abs(H).max())


def test_small_strain_limit_is_linear_elasticity():
    """At F = I the 9x9 Hessian equals the isotropic elasticity tensor
    C_ijkl = mu (d_ik d_jl + d_il d_jk) + lambda d_ij d_kl (textbook Lame)."""
    mu, lam = O.lame(E, NU)
    mu_t, lam_t = lame_textbook(E, NU)
    H = O.snh_hess9(np.eye(3), mu, lam)
    d = np.eye(3)
    C = np.zeros((9, 9))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i + 3 * j, k + 3 * l] = mu_t * (d[i, k] * d[j, l] + d[i, l] * d[j, k]) + lam_t * d[i, j] * d[k, l]
    assert np.allclose(H, C, rtol=1e-14, atol=1e-9)


def test_rotation_invariance(rng):
    mu, lam = O.lame(E, NU)
    for _ in range(10):
        F = rand_F(rng)
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        assert O.snh_psi(Q @ F, mu, lam) == pytest.approx(O.snh_psi(F, mu, lam), rel=1e-12, abs=1e-9)
        assert np.allclose(O.snh_pk1(Q @ F, mu, lam), Q @ O.snh_pk1(F, mu, lam), rtol=1e-11, atol=1e-6)


@pytest.mark.parametrize("n", [3, 9, 12])
def test_jacobi_eig_vs_numpy(rng, n):
    for _ in range(10):
        A = rng.standard_normal((n, n))
        A = A + A.T
        w, Q = O.sym_eig(A)
        wn = np.linalg.eigvalsh(A)
        assert np.allclose(np.sort(w), wn, rtol=1e-12, atol=1e-12 * np.abs(wn).max())
        assert np.allclose(Q @ np.diag(w) @ Q.T, A, atol=1e-12 * np.abs(A).max())
        assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-13)


def test_psd_projection(rng):
    for n in (9, 12):
        A = rng.standard_normal((n, n))
        A = A + A.T
        Ap = O.psd_project(A)
        w, V = np.linalg.eigh(A)
        ref = (V * np.maximum(w, 0)) @ V.T
        assert np.allclose(Ap, ref, atol=1e-12 * np.abs(A).max())
        assert np.linalg.eigvalsh(Ap).min() >= -1e-12 * np.abs(A).max()
        S = A @ A.T  # already PSD -> unchanged
        assert np.allclose(O.psd_project(S), S, atol=1e-12 * np.abs(S).max())


def analytic_snh_eigs(F, mu, lam):
    """Eigenvalues of d2Psi/dF2 in the SVD frame (twist, flip, scaling),
    derived independently of the oracle's cofactor form."""
    U, s, Vt = np.linalg.svd(F)
    if np.linalg.det(U) * np.linalg.det(Vt) < 0:
        s[2] = -s[2]
    J = s[0] * s[1] * s[2]
    k = lam * (J - 1) - mu
    out = []
    for (i, j, m) in ((0, 1, 2), (1, 2, 0), (0, 2, 1)):
        out += [mu + k * s[m], mu - k * s[m]]
    A = mu * np.eye(3) + k * np.array([[0, s[2], s[1]], [s[2], 0, s[0]], [s[1], s[0], 0]])
    g = np.array([s[1] * s[2], s[0] * s[2], s[0] * s[1]])
    A += lam * np.outer(g, g)
    out += list(np.linalg.eigvalsh(A))
    return np.sort(out)


@pytest.mark.parametrize("inv", [False, True])
def test_hessian_eigensystem_two_derivations(rng, inv):
    mu, lam = O.lame(E, NU)
    for _ in range(20):
        F = rand_F(rng, 0.5, allow_inverted=inv)
        w, _ = O.sym_eig(O.snh_hess9(F, mu, lam))
        ref = analytic_snh_eigs(F, mu, lam)
        assert np.allclose(np.sort(w), ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def rest_tet(rng):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]) * 0.02 + 1e-3 * rng.standard_normal((4, 3))
    Dm = (X[1:] - X[0]).T
    assert np.linalg.det(Dm) > 0
    return X, np.linalg.inv(Dm), np.linalg.det(Dm) / 6


def test_deformation_gradient(rng):
    X, B, vol = rest_tet(rng)
    assert np.allclose(O.elem_F(X.reshape(-1), B), np.eye(3), atol=1e-12)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Y = X @ Q.T + 0.3
    assert np.allclose(O.elem_F(Y.reshape(-1), B), Q, atol=1e-12)


def test_element_gradient_and_hessian_fd(rng):
    mu, lam = O.lame(E, NU)
    for _ in range(10):
        X, B, vol = rest_tet(rng)
        x = (X + 0.004 * rng.standard_normal((4, 3))).reshape(-1)
        psi, g, H = O.elem_grad_hess(x, B, vol, mu, lam, project=False)
        h = 1e-8
        gfd, Hfd = np.zeros(12), np.zeros((12, 12))
        for k in range(12):
            xp, xm = x.copy(), x.copy()
            xp[k] += h
            xm[k] -= h
            gfd[k] = (O.elem_grad_hess(xp, B, vol, mu, lam, False)[0] - O.elem_grad_hess(xm, B, vol, mu, lam, False)[0]) / (2 * h)
            Hfd[:, k] = (O.elem_grad_hess(xp, B, vol, mu, lam, False)[1] - O.elem_grad_hess(xm, B, vol, mu, lam, False)[1]) / (2 * h)
        assert np.abs(g - gfd).max() <= 1e-5 * np.abs(g).max()
        assert np.abs(H - Hfd).max() <= 1e-5 * np.abs(H).max()


def test_projected_element_hessian_psd_and_translation_null(rng):
    mu, lam = O.lame(E, NU)
    for _ in range(10):
        X, B, vol = rest_tet(rng)
        x = (X + 0.01 * rng.standard_normal((4, 3))).reshape(-1)
        _, _, Hp = O.elem_grad_hess(x, B, vol, mu, lam, project=True)
        assert np.linalg.eigvalsh(Hp).min() >= -1e-10 * np.abs(Hp).max()
        t = np.tile(rng.standard_normal(3), 4)
        assert np.abs(Hp @ t).max() <= 1e-10 * np.abs(Hp).max()
        # near the stretch J = 1 + mu/lam, where lam (J - 1) - mu = 0, every
        # eigenvalue of the 9x9 Hessian is positive (twist and flip modes
        # equal mu), so the projection changes nothing
        Fs = np.diag((1 + mu / lam) ** (1 / 3) * (1 + 0.01 * rng.standard_normal(3)))
        assert np.linalg.eigvalsh(O.snh_hess9(Fs, mu, lam)).min() > 0
        x0 = (X @ Fs.T).reshape(-1)
        _, _, H0 = O.elem_grad_hess(x0, B, vol, mu, lam, project=False)
        _, _, H0p = O.elem_grad_hess(x0, B, vol, mu, lam, project=True)
        assert np.allclose(H0, H0p, atol=1e-10 * np.abs(H0).max())
