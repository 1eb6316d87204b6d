/*
 * Plain FP64 CPU oracle of the barrier-free augmented-Lagrangian contact
 * method (arXiv 2512.12151).  TEST INFRASTRUCTURE ONLY: it exists to check
 * the CUDA library, shares no code with it, and is loaded only by the test
 * suite, the smoke check and the benchmark's CPU-baseline leg.
 *
 * The method is iterative (Alg. 1-3), so this file follows the algorithms
 * step by step in the paper's order and notation.  Where the paper is
 * silent, the reading taken is stated at the routine.  Build with
 * -O2 -ffp-contract=off (no FMA contraction), single-threaded.
 *
 * Conventions: positions are (nv, 3) row-major doubles; F and Dm^-1 are
 * 3x3 row-major; vec(F) for the 9x9 Hessian is column-major
 * (index r + 3c), matching the paper's column blocks f_0, f_1, f_2.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PT 0
#define OR_EE 1
#define OR_ACCD_MAX_ITER 100000

struct or_scene {
    int nv, nt, nm;
    double *X, *x, *v, *targets;
    int has_targets;
    int *tets, *tmat;
    double *mats;
    uint8_t *dir;
    double *B, *vol, *emu, *elam, *mass;
    /* surface primitives */
    int nsv, nst, nse;
    int *sv, *st, *se;
    int64_t *tri_key_sorted; /* sorted (key, index) pairs for triangle lookup */
    int *tri_key_idx;
    /* elastic Hessian: full 3x3-block CSR over all vertices */
    int nnzb;
    int *rp, *ci, *tmap;
    double *val;
    double *grad;
    /* active set C = {(i, lambda_i, gamma_i)} and its linearisation */
    int nc, ccap;
    int *ctype, *ca, *cb;
    double *clam, *cgam, *cd, *cg, *cs;
    or_params p;
    double mu, delta;
    double L_scale; /* |L| at the time step's first Newton iterate (< 0: unset) */
    /* friction pairs of the time step (appendix A): vertices, closest-point
     * weights and unit normal at x^t, coefficient mu_f F; fA: the 3x3
     * tangent Hessian of each pair at the last assembly */
    int nf, fcap;
    int *fv;
    double *fw, *fn, *fk, *fA;
    /* gradient-norm residuals of the last step's outer iterations */
    int nres, rescap;
    double *res;
    /* optional log of the intermediate states xhat^[k] of the next time
     * steps' outer iterations (caller-owned, 3 nv doubles each) */
    double *xhat_log;
    int xhat_cap, xhat_n;
};

/* ------------------------------------------------------------------ */
/* small dense helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double det3(const double *M)
{
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}
static void inv3(const double *M, double *o)
{
    double d = det3(M);
    o[0] = (M[4] * M[8] - M[5] * M[7]) / d;
    o[1] = (M[2] * M[7] - M[1] * M[8]) / d;
    o[2] = (M[1] * M[5] - M[2] * M[4]) / d;
    o[3] = (M[5] * M[6] - M[3] * M[8]) / d;
    o[4] = (M[0] * M[8] - M[2] * M[6]) / d;
    o[5] = (M[2] * M[3] - M[0] * M[5]) / d;
    o[6] = (M[3] * M[7] - M[4] * M[6]) / d;
    o[7] = (M[1] * M[6] - M[0] * M[7]) / d;
    o[8] = (M[0] * M[4] - M[1] * M[3]) / d;
}
static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

/* ------------------------------------------------------------------ */
/* Stable Neo-Hookean (Tab. 2 caption: SNH).  The paper names the model   */
/* only; reading: Psi = mu/2 (|F|^2 - 3) - mu (J - 1) + lam/2 (J - 1)^2  */
/* with lam = lambda_Lame + mu, which reproduces linear elasticity at    */
/* small strain.                                                          */
/* ------------------------------------------------------------------ */
void or_lame(double E, double nu, double *mu, double *lam)
{
    *mu = E / (2.0 * (1.0 + nu));
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)) + *mu;
}

static void cofactor(const double F[9], double C[9])
{
    /* columns of dJ/dF: f1 x f2, f2 x f0, f0 x f1 (f_c = column c of F) */
    double f0[3] = {F[0], F[3], F[6]}, f1[3] = {F[1], F[4], F[7]}, f2[3] = {F[2], F[5], F[8]};
    double c0[3], c1[3], c2[3];
    cross3(f1, f2, c0);
    cross3(f2, f0, c1);
    cross3(f0, f1, c2);
    for (int r = 0; r < 3; ++r) {
        C[3 * r + 0] = c0[r];
        C[3 * r + 1] = c1[r];
        C[3 * r + 2] = c2[r];
    }
}

double or_snh_psi(const double F[9], double mu, double lam)
{
    double I2 = 0.0;
    for (int k = 0; k < 9; ++k) I2 += F[k] * F[k];
    double J = det3(F);
    return 0.5 * mu * (I2 - 3.0) - mu * (J - 1.0) + 0.5 * lam * (J - 1.0) * (J - 1.0);
}

void or_snh_pk1(const double F[9], double mu, double lam, double P[9])
{
    double C[9];
    cofactor(F, C);
    double J = det3(F);
    for (int k = 0; k < 9; ++k) P[k] = mu * F[k] + (lam * (J - 1.0) - mu) * C[k];
}

void or_snh_hess9(const double F[9], double mu, double lam, double H[81])
{
    /* d2Psi/dF2 = mu I + lam vec(cof) vec(cof)^T + (lam (J-1) - mu) d2J/dF2 */
    double C[9], g[9];
    cofactor(F, C);
    double J = det3(F);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) g[r + 3 * c] = C[3 * r + c];
    double f[3][3];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) f[c][r] = F[3 * r + c];
    double k = lam * (J - 1.0) - mu;
    memset(H, 0, 81 * sizeof(double));
    for (int i = 0; i < 9; ++i) {
        H[9 * i + i] += mu;
        for (int j = 0; j < 9; ++j) H[9 * i + j] += lam * g[i] * g[j];
    }
    /* block (c1, c2) of d2J/dF2 is d(df_c1 J)/d f_c2 = sign * [f_c3]x */
    for (int c1 = 0; c1 < 3; ++c1)
        for (int c2 = 0; c2 < 3; ++c2) {
            if (c1 == c2) continue;
            int c3 = 3 - c1 - c2;
            double sgn = (c2 == (c1 + 1) % 3) ? -1.0 : 1.0;
            const double *a = f[c3];
            double S[9] = {0, -a[2], a[1], a[2], 0, -a[0], -a[1], a[0], 0};
            for (int r1 = 0; r1 < 3; ++r1)
                for (int r2 = 0; r2 < 3; ++r2) H[9 * (r1 + 3 * c1) + (r2 + 3 * c2)] += k * sgn * S[3 * r1 + r2];
        }
}

/* Cyclic Jacobi eigendecomposition of a symmetric n x n matrix (textbook
 * method, Golub & Van Loan 8.5).  w: eigenvalues; Q: eigenvectors as
 * columns (row-major).  Returns the number of sweeps. */
int or_sym_eig(int n, const double *A0, double *w, double *Q)
{
    double *A = (double *)malloc((size_t)n * n * sizeof(double));
    memcpy(A, A0, (size_t)n * n * sizeof(double));
    for (int i = 0; i < n * n; ++i) Q[i] = 0.0;
    for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
    double fro = 0.0;
    for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
    int sweep = 0;
    for (; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (i != j) off += A[i * n + j] * A[i * n + j];
        if (off <= 1e-30 * fro || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* A <- A J */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* A <- J^T A */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) { /* Q <- Q J */
                    double qkp = Q[k * n + p], qkq = Q[k * n + q];
                    Q[k * n + p] = c * qkp - s * qkq;
                    Q[k * n + q] = s * qkp + c * qkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
    free(A);
    return sweep;
}

/* Section 5.1: (d2Psi/dF2)^+ = sum_k max(omega_k, 0) q_k q_k^T, here with
 * the eigenpairs from a dense Jacobi eigendecomposition. */
void or_psd_project(int n, const double *A, double *Ap)
{
    double *w = (double *)malloc(n * sizeof(double)), *Q = (double *)malloc((size_t)n * n * sizeof(double));
    or_sym_eig(n, A, w, Q);
    for (int i = 0; i < n * n; ++i) Ap[i] = 0.0;
    for (int k = 0; k < n; ++k) {
        double wk = w[k] > 0.0 ? w[k] : 0.0;
        if (wk == 0.0) continue;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) Ap[i * n + j] += wk * Q[i * n + k] * Q[j * n + k];
    }
    free(w);
    free(Q);
}

/* ------------------------------------------------------------------ */
/* Corotated linear elasticity (COR, one of the models of Tab. 2;       */
/* McAdams et al. 2011): Psi = mu |F - R|^2 + lam/2 (tr(S) - 3)^2 with  */
/* F = R S the polar decomposition (R a rotation also for inverted F:   */
/* the rotation-variant SVD F = U diag(s) V^T, U and V rotations, s_2   */
/* negative when det F < 0), lam the Lame constant (no shift: the small  */
/* strain limit is linear elasticity as it stands).                     */
/* ------------------------------------------------------------------ */
static void rot_svd(const double F[9], double U[9], double s[3], double V[9])
{
    /* V, s^2 from F^T F (descending); U = F V / s, completed to a rotation */
    double FtF[9], w[3], Q[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double t = 0.0;
            for (int r = 0; r < 3; ++r) t += F[3 * r + a] * F[3 * r + b];
            FtF[3 * a + b] = t;
        }
    or_sym_eig(3, FtF, w, Q); /* unordered; Q columns */
    int ord[3] = {0, 1, 2};   /* descending eigenvalues */
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (w[ord[j]] > w[ord[i]]) { int t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) V[3 * r + k] = Q[3 * r + ord[k]];
    if (det3(V) < 0.0)
        for (int r = 0; r < 3; ++r) V[3 * r + 2] = -V[3 * r + 2];
    double u[3][3];
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) {
            double t = 0.0;
            for (int c = 0; c < 3; ++c) t += F[3 * r + c] * V[3 * c + k];
            u[k][r] = t; /* F v_k */
        }
    double n0 = sqrt(dot3(u[0], u[0]));
    for (int r = 0; r < 3; ++r) u[0][r] = n0 > 0.0 ? u[0][r] / n0 : (r == 0 ? 1.0 : 0.0);
    double p = dot3(u[0], u[1]);
    for (int r = 0; r < 3; ++r) u[1][r] -= p * u[0][r];
    double n1 = sqrt(dot3(u[1], u[1]));
    if (n1 > 1e-300) {
        for (int r = 0; r < 3; ++r) u[1][r] /= n1;
    } else { /* any unit vector orthogonal to u0 */
        double e[3] = {0, 0, 0};
        e[fabs(u[0][0]) < 0.9 ? 0 : 1] = 1.0;
        double t = dot3(e, u[0]);
        for (int r = 0; r < 3; ++r) u[1][r] = e[r] - t * u[0][r];
        double nn = sqrt(dot3(u[1], u[1]));
        for (int r = 0; r < 3; ++r) u[1][r] /= nn;
    }
    double u2[3];
    cross3(u[0], u[1], u2);
    for (int r = 0; r < 3; ++r) {
        U[3 * r + 0] = u[0][r];
        U[3 * r + 1] = u[1][r];
        U[3 * r + 2] = u2[r];
    }
    /* s_k = u_k^T F v_k (s_2 carries the sign of det F) */
    for (int k = 0; k < 3; ++k) {
        double t = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) t += U[3 * r + k] * F[3 * r + c] * V[3 * c + k];
        s[k] = t;
    }
}

double or_cor_psi(const double F[9], double mu, double lam)
{
    double U[9], s[3], V[9];
    rot_svd(F, U, s, V);
    double e = 0.0, tr = 0.0;
    for (int k = 0; k < 3; ++k) {
        e += (s[k] - 1.0) * (s[k] - 1.0);
        tr += s[k];
    }
    return mu * e + 0.5 * lam * (tr - 3.0) * (tr - 3.0); /* |F - R|^2 = |diag(s) - I|^2 */
}

/* R = U V^T and tr(S) = sum s */
static double cor_rotation(const double F[9], double R[9], double U[9], double s[3], double V[9])
{
    rot_svd(F, U, s, V);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double t = 0.0;
            for (int k = 0; k < 3; ++k) t += U[3 * r + k] * V[3 * c + k];
            R[3 * r + c] = t;
        }
    return s[0] + s[1] + s[2];
}

void or_cor_pk1(const double F[9], double mu, double lam, double P[9])
{
    double R[9], U[9], s[3], V[9];
    double tr = cor_rotation(F, R, U, s, V);
    for (int k = 0; k < 9; ++k) P[k] = 2.0 * mu * (F[k] - R[k]) + lam * (tr - 3.0) * R[k];
}

/* d2Psi/dF2 = 2 mu (I - dR/dF) + lam vec(R) vec(R)^T + lam (tr S - 3) dR/dF,
 * with the derivative of the polar rotation: for dF, W = U^T dR V is skew
 * with W_ij = ((U^T dF V)_ij - (U^T dF V)_ji) / (s_i + s_j). */
void or_cor_hess9(const double F[9], double mu, double lam, double H[81])
{
    double R[9], U[9], s[3], V[9];
    double tr = cor_rotation(F, R, U, s, V);
    memset(H, 0, 81 * sizeof(double));
    for (int col = 0; col < 9; ++col) { /* dF = E_ab, vec index a + 3 b */
        int a = col % 3, b = col / 3;
        double Fh[3][3], W[3][3] = {{0}}, dR[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Fh[i][j] = U[3 * a + i] * V[3 * b + j];
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j) {
                double w = (Fh[i][j] - Fh[j][i]) / (s[i] + s[j]);
                W[i][j] = w;
                W[j][i] = -w;
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double t = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) t += U[3 * r + i] * W[i][j] * V[3 * c + j];
                dR[3 * r + c] = t;
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                int row = r + 3 * c;
                double v = -2.0 * mu * dR[3 * r + c] + lam * (tr - 3.0) * dR[3 * r + c];
                if (row == col) v += 2.0 * mu;
                v += lam * R[3 * r + c] * R[3 * a + b];
                H[9 * row + col] = v;
            }
    }
}

/* ------------------------------------------------------------------ */
/* Neo-Hookean (NH, one of the models of Tab. 2):                         */
/* Psi = mu/2 (|F|^2 - 3) - mu ln J + lam/2 (ln J)^2, lam the Lame        */
/* constant.  It is undefined for J <= 0 (the paper's example of a        */
/* non-invertible material, section 4.1); the energy is +inf there, so a  */
/* line search backtracks out of inverted states.                         */
/* ------------------------------------------------------------------ */
double or_nh_psi(const double F[9], double mu, double lam)
{
    double J = det3(F);
    if (!(J > 0.0)) return INFINITY;
    double I2 = 0.0;
    for (int k = 0; k < 9; ++k) I2 += F[k] * F[k];
    double L = log(J);
    return 0.5 * mu * (I2 - 3.0) - mu * L + 0.5 * lam * L * L;
}

/* P = mu (F - F^-T) + lam ln J F^-T */
void or_nh_pk1(const double F[9], double mu, double lam, double P[9])
{
    double Fi[9];
    inv3(F, Fi);
    double L = log(det3(F));
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double fit = Fi[3 * c + r]; /* (F^-T)_rc */
            P[3 * r + c] = mu * (F[3 * r + c] - fit) + lam * L * fit;
        }
}

/* d2Psi / dF_ij dF_kl = mu d_ik d_jl + (mu - lam ln J) (F^-1)_jk (F^-1)_li
 *                       + lam (F^-T)_ij (F^-T)_kl,
 * from d(F^-1) = -F^-1 dF F^-1 and d(ln J) = F^-T : dF. */
void or_nh_hess9(const double F[9], double mu, double lam, double H[81])
{
    double Fi[9];
    inv3(F, Fi);
    double L = log(det3(F));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double v = (mu - lam * L) * Fi[3 * j + k] * Fi[3 * l + i] + lam * Fi[3 * j + i] * Fi[3 * l + k];
                    if (i == k && j == l) v += mu;
                    H[9 * (i + 3 * j) + (k + 3 * l)] = v;
                }
}

/* Smallest root in (0, 1] of p(t) = c0 + c1 t + c2 t^2 + c3 t^3 with
 * p(0) = c0 > 0; returns 1 when p stays positive on [0, 1].  The real
 * roots of p' split [0, 1] into pieces on which p is monotone; the first
 * piece whose right end has p <= 0 holds the root, which bisection brackets
 * to adjacent doubles.  The returned t is the bracket's left end (p > 0). */
double or_cubic_first_root(const double c[4])
{
    if (!(c[0] > 0.0)) return 0.0;
    double br[4];
    int nb = 0;
    br[nb++] = 0.0;
    /* critical points: 3 c3 t^2 + 2 c2 t + c1 = 0 */
    double qa = 3.0 * c[3], qb = 2.0 * c[2], qc = c[1], crit[2];
    int nc = 0;
    if (qa != 0.0) {
        double disc = qb * qb - 4.0 * qa * qc;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            crit[nc++] = (-qb - sq) / (2.0 * qa);
            crit[nc++] = (-qb + sq) / (2.0 * qa);
        }
    } else if (qb != 0.0) {
        crit[nc++] = -qc / qb;
    }
    if (nc == 2 && crit[0] > crit[1]) { double t = crit[0]; crit[0] = crit[1]; crit[1] = t; }
    for (int k = 0; k < nc; ++k)
        if (crit[k] > 0.0 && crit[k] < 1.0) br[nb++] = crit[k];
    br[nb++] = 1.0;
    for (int k = 0; k + 1 < nb; ++k) {
        double lo = br[k], hi = br[k + 1];
        double phi = c[0] + hi * (c[1] + hi * (c[2] + hi * c[3]));
        if (phi > 0.0) continue;
        for (;;) {
            double mid = 0.5 * (lo + hi);
            if (!(mid > lo && mid < hi)) break;
            double pm = c[0] + mid * (c[1] + mid * (c[2] + mid * c[3]));
            if (pm > 0.0) lo = mid;
            else hi = mid;
        }
        return lo;
    }
    return 1.0;
}

/* Coefficients of det(A + t B) - s det(A) (3x3, row-major), from the
 * multilinearity of det in the columns: t^k collects the determinants with
 * k columns taken from B and 3 - k from A. */
void or_det_cubic(const double A[9], const double B[9], double s, double c[4])
{
    c[0] = c[1] = c[2] = c[3] = 0.0;
    for (int mask = 0; mask < 8; ++mask) {
        double M[9];
        int k = 0;
        for (int col = 0; col < 3; ++col) {
            const double *src = (mask >> col) & 1 ? B : A;
            k += (mask >> col) & 1;
            for (int r = 0; r < 3; ++r) M[3 * r + col] = src[3 * r + col];
        }
        c[k] += det3(M);
    }
    c[0] -= s * det3(A);
}

/* F = Ds Dm^-1 with Ds = [x1 - x0, x2 - x0, x3 - x0] (section 3). */
void or_elem_F(const double x[12], const double B[9], double F[9])
{
    double Ds[9];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) Ds[3 * r + k] = x[3 * (k + 1) + r] - x[r];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Ds[3 * r + k] * B[3 * k + c];
            F[3 * r + c] = s;
        }
}

/* A_i' rows (section 5.1): dF = dx_i' A_i'; A_0 = -(A_1 + A_2 + A_3). */
static void elem_A(const double B[9], double A[4][3])
{
    for (int c = 0; c < 3; ++c) {
        A[1][c] = B[c];
        A[2][c] = B[3 + c];
        A[3][c] = B[6 + c];
        A[0][c] = -(B[c] + B[3 + c] + B[6 + c]);
    }
}

/* Element energy vol*Psi, gradient d(vol Psi)/dx (12) and Hessian
 * vol * D^T (d2Psi/dF2)[+] D (12x12), D = dvec(F)/dx.  With project != 0
 * the 9x9 F-space Hessian is PSD-projected first (section 5.1). */
void or_elem_grad_hess(const double x[12], const double B[9], double vol, double mu, double lam,
                       int project, double *psi, double g[12], double H[144])
{
    or_elem_grad_hess_model(0, x, B, vol, mu, lam, project, psi, g, H);
}

double or_model_psi(int model, const double F[9], double mu, double lam)
{
    if (model == 1) return or_cor_psi(F, mu, lam);
    if (model == 2) return or_nh_psi(F, mu, lam);
    return or_snh_psi(F, mu, lam);
}

void or_elem_grad_hess_model(int model, const double x[12], const double B[9], double vol, double mu, double lam,
                             int project, double *psi, double g[12], double H[144])
{
    double F[9], P[9], H9[81], H9p[81], A[4][3];
    or_elem_F(x, B, F);
    elem_A(B, A);
    if (psi) *psi = vol * or_model_psi(model, F, mu, lam);
    if (g) {
        if (model == 1) or_cor_pk1(F, mu, lam, P);
        else if (model == 2) or_nh_pk1(F, mu, lam, P);
        else or_snh_pk1(F, mu, lam, P);
        for (int i = 0; i < 4; ++i)
            for (int r = 0; r < 3; ++r) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c) s += P[3 * r + c] * A[i][c];
                g[3 * i + r] = vol * s;
            }
    }
    if (H) {
        if (model == 1) or_cor_hess9(F, mu, lam, H9);
        else if (model == 2) or_nh_hess9(F, mu, lam, H9);
        else or_snh_hess9(F, mu, lam, H9);
        if (project) or_psd_project(9, H9, H9p);
        else memcpy(H9p, H9, sizeof(H9p));
        for (int i = 0; i < 4; ++i)
            for (int a = 0; a < 3; ++a)
                for (int j = 0; j < 4; ++j)
                    for (int b = 0; b < 3; ++b) {
                        double s = 0.0;
                        for (int c = 0; c < 3; ++c)
                            for (int d = 0; d < 3; ++d) s += H9p[9 * (a + 3 * c) + (b + 3 * d)] * A[i][c] * A[j][d];
                        H[12 * (3 * i + a) + (3 * j + b)] = vol * s;
                    }
    }
}

/* ------------------------------------------------------------------ */
/* Unsigned distances between closed primitives (section 3: d_i over      */
/* vertex-face and edge-edge pairs; the paper gives no formulas).         */
/* The closest point of a closed triangle is its plane projection when   */
/* that lies inside, else the closest point of one of its edges; the     */
/* closest pair of two closed segments is the interior-interior critical  */
/* pair or involves an endpoint.  The evaluation order below is fixed     */
/* (the CCD relies on it).                                                */
/* ------------------------------------------------------------------ */
static double ps2(const double *p, const double *a, const double *b, double *tout)
{
    double e[3], ap[3], q[3], r[3];
    sub3(b, a, e);
    sub3(p, a, ap);
    double ee = dot3(e, e);
    double t = 0.0;
    if (ee > 0.0) t = dot3(ap, e) / ee;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    q[0] = a[0] + t * e[0];
    q[1] = a[1] + t * e[1];
    q[2] = a[2] + t * e[2];
    sub3(p, q, r);
    if (tout) *tout = t;
    return dot3(r, r);
}

/* returns d^2; w[0..2] barycentric weights of the closest point on (a,b,c) */
static double pt_closest(const double *p, const double *a, const double *b, const double *c, double w[3])
{
    double ab[3], ac[3], ap[3];
    sub3(b, a, ab);
    sub3(c, a, ac);
    sub3(p, a, ap);
    double d00 = dot3(ab, ab), d01 = dot3(ab, ac), d11 = dot3(ac, ac);
    double d20 = dot3(ap, ab), d21 = dot3(ap, ac);
    double den = d00 * d11 - d01 * d01;
    if (den > 0.0) {
        double v = (d11 * d20 - d01 * d21) / den;
        double ww = (d00 * d21 - d01 * d20) / den;
        double u = (1.0 - v) - ww;
        if (u >= 0.0 && v >= 0.0 && ww >= 0.0) {
            double q[3], r[3];
            for (int k = 0; k < 3; ++k) q[k] = (a[k] + v * ab[k]) + ww * ac[k];
            sub3(p, q, r);
            w[0] = u;
            w[1] = v;
            w[2] = ww;
            return dot3(r, r);
        }
    }
    double t, best;
    best = ps2(p, a, b, &t);
    w[0] = 1.0 - t; w[1] = t; w[2] = 0.0;
    double c2 = ps2(p, b, c, &t);
    if (c2 < best) { best = c2; w[0] = 0.0; w[1] = 1.0 - t; w[2] = t; }
    double c3 = ps2(p, c, a, &t);
    if (c3 < best) { best = c3; w[0] = t; w[1] = 0.0; w[2] = 1.0 - t; }
    return best;
}

/* returns d^2; wa, wb: weights of the closest points on (a0,a1), (b0,b1) */
static double ee_closest(const double *a0, const double *a1, const double *b0, const double *b1,
                         double wa[2], double wb[2])
{
    double ea[3], eb[3], w[3];
    sub3(a1, a0, ea);
    sub3(b1, b0, eb);
    sub3(a0, b0, w);
    double A = dot3(ea, ea), B = dot3(ea, eb), C = dot3(eb, eb), D = dot3(ea, w), E = dot3(eb, w);
    double den = A * C - B * B;
    double best = INFINITY;
    if (den > 0.0) {
        double s = (B * E - C * D) / den;
        double t = (A * E - B * D) / den;
        if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
            double P[3], Q[3], r[3];
            for (int k = 0; k < 3; ++k) { P[k] = a0[k] + s * ea[k]; Q[k] = b0[k] + t * eb[k]; }
            sub3(P, Q, r);
            best = dot3(r, r);
            wa[0] = 1.0 - s; wa[1] = s; wb[0] = 1.0 - t; wb[1] = t;
        }
    }
    double t, c;
    c = ps2(a0, b0, b1, &t);
    if (c < best) { best = c; wa[0] = 1.0; wa[1] = 0.0; wb[0] = 1.0 - t; wb[1] = t; }
    c = ps2(a1, b0, b1, &t);
    if (c < best) { best = c; wa[0] = 0.0; wa[1] = 1.0; wb[0] = 1.0 - t; wb[1] = t; }
    c = ps2(b0, a0, a1, &t);
    if (c < best) { best = c; wb[0] = 1.0; wb[1] = 0.0; wa[0] = 1.0 - t; wa[1] = t; }
    c = ps2(b1, a0, a1, &t);
    if (c < best) { best = c; wb[0] = 0.0; wb[1] = 1.0; wa[0] = 1.0 - t; wa[1] = t; }
    return best;
}

double or_pt_dist2(const double p[3], const double a[3], const double b[3], const double c[3])
{
    double w[3];
    return pt_closest(p, a, b, c, w);
}

double or_ee_dist2(const double a0[3], const double a1[3], const double b0[3], const double b1[3])
{
    double wa[2], wb[2];
    return ee_closest(a0, a1, b0, b1, wa, wb);
}

static double pair_dist2(int type, const double *x)
{
    if (type == OR_PT) return or_pt_dist2(x, x + 3, x + 6, x + 9);
    return or_ee_dist2(x, x + 3, x + 6, x + 9);
}

/* d and its gradient (envelope theorem: n = (P - Q)/d weighted by the
 * closest points' barycentric weights); x holds the 4 vertices of the pair
 * (PT: point, tri0, tri1, tri2; EE: a0, a1, b0, b1). */
double or_pair_dist_grad(int type, const double x[12], double g[12])
{
    double cw[4]; /* signed weights: P - Q = sum_k cw_k x_k */
    double d2;
    if (type == OR_PT) {
        double w[3];
        d2 = pt_closest(x, x + 3, x + 6, x + 9, w);
        cw[0] = 1.0; cw[1] = -w[0]; cw[2] = -w[1]; cw[3] = -w[2];
    } else {
        double wa[2], wb[2];
        d2 = ee_closest(x, x + 3, x + 6, x + 9, wa, wb);
        cw[0] = wa[0]; cw[1] = wa[1]; cw[2] = -wb[0]; cw[3] = -wb[1];
    }
    double d = sqrt(d2);
    double diff[3] = {0, 0, 0};
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 3; ++c) diff[c] += cw[k] * x[3 * k + c];
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 3; ++c) g[3 * k + c] = d > 0.0 ? cw[k] * diff[c] / d : 0.0;
    return d;
}

/* ------------------------------------------------------------------ */
/* Additive CCD (the narrow phase the paper uses, section 5.1, after Li, */
/* Kaufman and Jiang 2021), thickness 0.  Reading: conservative rescaling */
/* s (0.1), target gap s*d(x0), iteration cap -> the current t.           */
/* Returns 1 with *toi = t in [0, tmax] on a hit, else 0.                 */
/* ------------------------------------------------------------------ */
int or_accd(int type, const double x0[12], const double x1[12], double s, double tmax,
            int32_t max_iter, double *toi)
{
    double p[12], x[12], pbar[3], n[4];
    for (int k = 0; k < 12; ++k) p[k] = x1[k] - x0[k];
    for (int c = 0; c < 3; ++c) pbar[c] = (((p[c] + p[3 + c]) + p[6 + c]) + p[9 + c]) * 0.25;
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 3; ++c) p[3 * k + c] = p[3 * k + c] - pbar[c];
    for (int k = 0; k < 4; ++k) n[k] = sqrt(dot3(p + 3 * k, p + 3 * k));
    double lp;
    if (type == OR_PT) lp = n[0] + fmax(fmax(n[1], n[2]), n[3]);
    else lp = fmax(n[0], n[1]) + fmax(n[2], n[3]);
    if (lp == 0.0) return 0;
    memcpy(x, x0, sizeof(x));
    double d = sqrt(pair_dist2(type, x));
    double g = s * d;
    double t = 0.0;
    double tl = ((1.0 - s) * d) / lp;
    for (int it = 0; it < max_iter; ++it) {
        for (int k = 0; k < 12; ++k) x[k] = x[k] + tl * p[k];
        d = sqrt(pair_dist2(type, x));
        if (t > 0.0 && d < g) {
            *toi = t;
            return 1;
        }
        t = t + tl;
        if (t > tmax) return 0;
        tl = (0.9 * d) / lp;
    }
    *toi = t;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Scene set-up: mass, Dm^-1, surface primitives, Hessian pattern.       */
/* ------------------------------------------------------------------ */
static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}
typedef struct { int64_t key; int idx; } keyidx;
static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx *x = (const keyidx *)a, *y = (const keyidx *)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->idx > y->idx) - (x->idx < y->idx);
}
static void sort3i(int *t)
{
    int a = t[0], b = t[1], c = t[2], s;
    if (a > b) { s = a; a = b; b = s; }
    if (b > c) { s = b; b = c; c = s; }
    if (a > b) { s = a; a = b; b = s; }
    t[0] = a; t[1] = b; t[2] = c;
}
static int64_t tri_key(const int *t3)
{
    int t[3] = {t3[0], t3[1], t3[2]};
    sort3i(t);
    return ((int64_t)t[0] << 42) | ((int64_t)t[1] << 21) | (int64_t)t[2];
}

static void build_surface(or_scene *S, int nx, const int32_t *xtris)
{
    /* boundary faces = tet faces that occur exactly once */
    static const int fl[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
    int nf = 4 * S->nt;
    keyidx *F = (keyidx *)xcalloc(nf, sizeof(keyidx));
    for (int e = 0; e < S->nt; ++e)
        for (int f = 0; f < 4; ++f) {
            int t[3] = {S->tets[4 * e + fl[f][0]], S->tets[4 * e + fl[f][1]], S->tets[4 * e + fl[f][2]]};
            F[4 * e + f].key = tri_key(t);
            F[4 * e + f].idx = 4 * e + f;
        }
    qsort(F, nf, sizeof(keyidx), cmp_keyidx);
    S->st = (int *)xcalloc(3 * (nf + nx), sizeof(int));
    int nst = 0;
    for (int i = 0; i < nf;) {
        int j = i;
        while (j < nf && F[j].key == F[i].key) ++j;
        if (j - i == 1) {
            int e = F[i].idx / 4, f = F[i].idx % 4;
            for (int k = 0; k < 3; ++k) S->st[3 * nst + k] = S->tets[4 * e + fl[f][k]];
            ++nst;
        }
        i = j;
    }
    free(F);
    for (int i = 0; i < nx; ++i) {
        for (int k = 0; k < 3; ++k) S->st[3 * nst + k] = xtris[3 * i + k];
        ++nst;
    }
    S->nst = nst;
    /* edges of surface triangles, unique, sorted by (lo, hi) */
    int64_t *E = (int64_t *)xcalloc(3 * nst, sizeof(int64_t));
    for (int i = 0; i < nst; ++i)
        for (int k = 0; k < 3; ++k) {
            int a = S->st[3 * i + k], b = S->st[3 * i + (k + 1) % 3];
            int lo = a < b ? a : b, hi = a < b ? b : a;
            E[3 * i + k] = ((int64_t)lo << 32) | (int64_t)hi;
        }
    qsort(E, 3 * nst, sizeof(int64_t), cmp_i64);
    S->se = (int *)xcalloc(2 * 3 * nst, sizeof(int));
    int nse = 0;
    for (int i = 0; i < 3 * nst; ++i) {
        if (i > 0 && E[i] == E[i - 1]) continue;
        S->se[2 * nse] = (int)(E[i] >> 32);
        S->se[2 * nse + 1] = (int)(E[i] & 0xffffffff);
        ++nse;
    }
    S->nse = nse;
    free(E);
    /* surface vertices */
    char *on = (char *)xcalloc(S->nv, 1);
    for (int i = 0; i < 3 * nst; ++i) on[S->st[i]] = 1;
    S->sv = (int *)xcalloc(S->nv, sizeof(int));
    int nsv = 0;
    for (int v = 0; v < S->nv; ++v)
        if (on[v]) S->sv[nsv++] = v;
    S->nsv = nsv;
    free(on);
    /* triangle lookup by sorted vertex key */
    keyidx *T = (keyidx *)xcalloc(nst, sizeof(keyidx));
    for (int i = 0; i < nst; ++i) { T[i].key = tri_key(S->st + 3 * i); T[i].idx = i; }
    qsort(T, nst, sizeof(keyidx), cmp_keyidx);
    S->tri_key_sorted = (int64_t *)xcalloc(nst, sizeof(int64_t));
    S->tri_key_idx = (int *)xcalloc(nst, sizeof(int));
    for (int i = 0; i < nst; ++i) { S->tri_key_sorted[i] = T[i].key; S->tri_key_idx[i] = T[i].idx; }
    free(T);
}

static int find_block(const or_scene *S, int r, int c)
{
    for (int k = S->rp[r]; k < S->rp[r + 1]; ++k)
        if (S->ci[k] == c) return k;
    return -1;
}

static void build_pattern(or_scene *S)
{
    int64_t *P = (int64_t *)xcalloc((size_t)16 * S->nt + S->nv, sizeof(int64_t));
    int np = 0;
    for (int v = 0; v < S->nv; ++v) P[np++] = ((int64_t)v << 32) | v;
    for (int e = 0; e < S->nt; ++e)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j)
                P[np++] = ((int64_t)S->tets[4 * e + i] << 32) | (int64_t)S->tets[4 * e + j];
    qsort(P, np, sizeof(int64_t), cmp_i64);
    S->rp = (int *)xcalloc(S->nv + 1, sizeof(int));
    S->ci = (int *)xcalloc(np, sizeof(int));
    int nnzb = 0;
    for (int i = 0; i < np; ++i) {
        if (i > 0 && P[i] == P[i - 1]) continue;
        int r = (int)(P[i] >> 32);
        S->ci[nnzb++] = (int)(P[i] & 0xffffffff);
        S->rp[r + 1]++;
    }
    for (int v = 0; v < S->nv; ++v) S->rp[v + 1] += S->rp[v];
    S->nnzb = nnzb;
    free(P);
    S->val = (double *)xcalloc((size_t)9 * nnzb, sizeof(double));
    S->tmap = (int *)xcalloc((size_t)16 * S->nt, sizeof(int));
    for (int e = 0; e < S->nt; ++e)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j)
                S->tmap[16 * e + 4 * i + j] = find_block(S, S->tets[4 * e + i], S->tets[4 * e + j]);
}

or_scene *or_create(int32_t nv, const double *rest, const double *x0, const double *v0, int32_t nt,
                    const int32_t *tets, const int32_t *tet_mat, int32_t nm, const double *mats,
                    int32_t nx, const int32_t *xtris, const uint8_t *dir, const or_params *prm)
{
    or_scene *S = (or_scene *)calloc(1, sizeof(or_scene));
    S->nv = nv; S->nt = nt; S->nm = nm; S->p = *prm;
    S->X = (double *)xcalloc(3 * nv, sizeof(double));
    S->x = (double *)xcalloc(3 * nv, sizeof(double));
    S->v = (double *)xcalloc(3 * nv, sizeof(double));
    S->targets = (double *)xcalloc(3 * nv, sizeof(double));
    S->grad = (double *)xcalloc(3 * nv, sizeof(double));
    memcpy(S->X, rest, 3 * nv * sizeof(double));
    memcpy(S->x, x0, 3 * nv * sizeof(double));
    memcpy(S->v, v0, 3 * nv * sizeof(double));
    S->tets = (int *)xcalloc(4 * nt, sizeof(int));
    S->tmat = (int *)xcalloc(nt, sizeof(int));
    memcpy(S->tets, tets, 4 * nt * sizeof(int));
    memcpy(S->tmat, tet_mat, nt * sizeof(int));
    S->mats = (double *)xcalloc(3 * nm, sizeof(double));
    memcpy(S->mats, mats, 3 * nm * sizeof(double));
    S->dir = (uint8_t *)xcalloc(nv, 1);
    if (dir) memcpy(S->dir, dir, nv);
    /* Dm^-1, rest volume, Lame parameters, lumped mass m_v = sum rho V_e / 4 */
    S->B = (double *)xcalloc(9 * nt, sizeof(double));
    S->vol = (double *)xcalloc(nt, sizeof(double));
    S->emu = (double *)xcalloc(nt, sizeof(double));
    S->elam = (double *)xcalloc(nt, sizeof(double));
    S->mass = (double *)xcalloc(nv, sizeof(double));
    for (int e = 0; e < nt; ++e) {
        double Dm[9];
        const int *t = S->tets + 4 * e;
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) Dm[3 * r + k] = S->X[3 * t[k + 1] + r] - S->X[3 * t[0] + r];
        inv3(Dm, S->B + 9 * e);
        S->vol[e] = det3(Dm) / 6.0;
        const double *m = S->mats + 3 * S->tmat[e];
        or_lame(m[0], m[1], &S->emu[e], &S->elam[e]);
        if (prm->model == 1 || prm->model == 2) S->elam[e] -= S->emu[e]; /* COR, NH: the Lame constant itself */
        for (int k = 0; k < 4; ++k) S->mass[t[k]] += m[2] * S->vol[e] / 4.0;
    }
    for (int v = 0; v < nv; ++v)
        if (S->dir[v]) S->mass[v] = 1.0;
    build_surface(S, nx, xtris);
    build_pattern(S);
    S->ccap = 1024;
    S->ctype = (int *)xcalloc(S->ccap, sizeof(int));
    S->ca = (int *)xcalloc(S->ccap, sizeof(int));
    S->cb = (int *)xcalloc(S->ccap, sizeof(int));
    S->clam = (double *)xcalloc(S->ccap, sizeof(double));
    S->cgam = (double *)xcalloc(S->ccap, sizeof(double));
    S->cd = (double *)xcalloc(S->ccap, sizeof(double));
    S->cs = (double *)xcalloc(S->ccap, sizeof(double));
    S->cg = (double *)xcalloc(12 * S->ccap, sizeof(double));
    S->mu = 0.0;
    S->delta = prm->delta;
    S->L_scale = -1.0;
    return S;
}

void or_destroy(or_scene *S)
{
    if (!S) return;
    void *ptrs[] = {S->X, S->x, S->v, S->targets, S->grad, S->tets, S->tmat, S->mats, S->dir, S->B,
                    S->vol, S->emu, S->elam, S->mass, S->sv, S->st, S->se, S->tri_key_sorted,
                    S->tri_key_idx, S->rp, S->ci, S->tmap, S->val, S->ctype, S->ca, S->cb,
                    S->clam, S->cgam, S->cd, S->cs, S->cg, S->fv, S->fw, S->fn, S->fk, S->fA, S->res};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(S);
}

void or_get_state(const or_scene *S, double *x, double *v)
{
    if (x) memcpy(x, S->x, 3 * S->nv * sizeof(double));
    if (v) memcpy(v, S->v, 3 * S->nv * sizeof(double));
}
void or_set_state(or_scene *S, const double *x, const double *v)
{
    if (x) memcpy(S->x, x, 3 * S->nv * sizeof(double));
    if (v) memcpy(S->v, v, 3 * S->nv * sizeof(double));
}
void or_set_dirichlet_targets(or_scene *S, const double *targets)
{
    int j = 0;
    for (int v = 0; v < S->nv; ++v)
        if (S->dir[v]) {
            for (int c = 0; c < 3; ++c) S->targets[3 * v + c] = targets[3 * j + c];
            ++j;
        }
    S->has_targets = 1;
}
void or_surface_sizes(const or_scene *S, int32_t *nsv, int32_t *nst, int32_t *nse)
{
    *nsv = S->nsv; *nst = S->nst; *nse = S->nse;
}
void or_surface(const or_scene *S, int32_t *sv, int32_t *st, int32_t *se)
{
    memcpy(sv, S->sv, S->nsv * sizeof(int));
    memcpy(st, S->st, 3 * S->nst * sizeof(int));
    memcpy(se, S->se, 2 * S->nse * sizeof(int));
}
void or_mass(const or_scene *S, double *m) { memcpy(m, S->mass, S->nv * sizeof(double)); }
double or_get_mu(const or_scene *S) { return S->mu; }
void or_set_mu_delta(or_scene *S, double mu, double delta) { S->mu = mu; S->delta = delta; }

/* ------------------------------------------------------------------ */
/* Active set bookkeeping                                                */
/* ------------------------------------------------------------------ */
static void pair_verts(const or_scene *S, int type, int a, int b, int v[4])
{
    if (type == OR_PT) {
        v[0] = a; v[1] = S->st[3 * b]; v[2] = S->st[3 * b + 1]; v[3] = S->st[3 * b + 2];
    } else {
        v[0] = S->se[2 * a]; v[1] = S->se[2 * a + 1]; v[2] = S->se[2 * b]; v[3] = S->se[2 * b + 1];
    }
}
static void gather12(const double *x, const int v[4], double o[12])
{
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 3; ++c) o[3 * k + c] = x[3 * v[k] + c];
}
static int64_t pair_key(int type, int a, int b) { return ((int64_t)type << 62) | ((int64_t)a << 31) | (int64_t)b; }

static void canon_key(const or_scene *S, int type, int a, int b, int32_t *k)
{
    int v[4];
    pair_verts(S, type, a, b, v);
    k[0] = type;
    if (type == OR_PT) {
        int t[3] = {v[1], v[2], v[3]};
        sort3i(t);
        k[1] = v[0]; k[2] = t[0]; k[3] = t[1]; k[4] = t[2];
    } else {
        k[1] = v[0]; k[2] = v[1]; k[3] = v[2]; k[4] = v[3]; /* edges are stored (lo, hi), ea < eb */
    }
}

static void c_reserve(or_scene *S, int n)
{
    if (n <= S->ccap) return;
    int cap = S->ccap;
    while (cap < n) cap *= 2;
    S->ctype = (int *)realloc(S->ctype, cap * sizeof(int));
    S->ca = (int *)realloc(S->ca, cap * sizeof(int));
    S->cb = (int *)realloc(S->cb, cap * sizeof(int));
    S->clam = (double *)realloc(S->clam, cap * sizeof(double));
    S->cgam = (double *)realloc(S->cgam, cap * sizeof(double));
    S->cd = (double *)realloc(S->cd, cap * sizeof(double));
    S->cs = (double *)realloc(S->cs, cap * sizeof(double));
    S->cg = (double *)realloc(S->cg, 12 * cap * sizeof(double));
    S->ccap = cap;
}

int32_t or_active_count(const or_scene *S) { return S->nc; }

void or_active_get(const or_scene *S, int32_t *keys, double *lam, double *gam)
{
    for (int i = 0; i < S->nc; ++i) {
        if (keys) canon_key(S, S->ctype[i], S->ca[i], S->cb[i], keys + 5 * i);
        if (lam) lam[i] = S->clam[i];
        if (gam) gam[i] = S->cgam[i];
    }
}

/* vertex ids of each pair in the order its linearisation uses */
void or_active_verts(const or_scene *S, int32_t *v4)
{
    for (int i = 0; i < S->nc; ++i) pair_verts(S, S->ctype[i], S->ca[i], S->cb[i], v4 + 4 * i);
}

static int find_tri(const or_scene *S, const int *t3)
{
    int64_t k = tri_key(t3);
    int lo = 0, hi = S->nst - 1;
    while (lo <= hi) {
        int m = (lo + hi) / 2;
        if (S->tri_key_sorted[m] == k) return S->tri_key_idx[m];
        if (S->tri_key_sorted[m] < k) lo = m + 1; else hi = m - 1;
    }
    return -1;
}
static int find_edge(const or_scene *S, int a, int b)
{
    int lo = 0, hi = S->nse - 1;
    while (lo <= hi) {
        int m = (lo + hi) / 2;
        int ma = S->se[2 * m], mb = S->se[2 * m + 1];
        if (ma == a && mb == b) return m;
        if (ma < a || (ma == a && mb < b)) lo = m + 1; else hi = m - 1;
    }
    return -1;
}

int32_t or_active_set(or_scene *S, int32_t n, const int32_t *keys, const double *lam, const double *gam)
{
    c_reserve(S, n);
    S->nc = 0;
    for (int i = 0; i < n; ++i) {
        const int32_t *k = keys + 5 * i;
        int a, b;
        if (k[0] == OR_PT) {
            a = k[1];
            b = find_tri(S, k + 2);
        } else {
            a = find_edge(S, k[1], k[2]);
            b = find_edge(S, k[3], k[4]);
        }
        if (a < 0 || b < 0) return -1;
        S->ctype[S->nc] = k[0]; S->ca[S->nc] = a; S->cb[S->nc] = b;
        S->clam[S->nc] = lam[i]; S->cgam[S->nc] = gam[i];
        S->nc++;
    }
    return S->nc;
}

/* ------------------------------------------------------------------ */
/* Incremental potential and its derivatives (section 3, Alg. 2)         */
/* ------------------------------------------------------------------ */
void or_xtilde(const or_scene *S, double *xt)
{
    double h = S->p.dt;
    for (int v = 0; v < S->nv; ++v)
        for (int c = 0; c < 3; ++c) {
            double xv = S->x[3 * v + c];
            xt[3 * v + c] = S->dir[v] ? xv : xv + h * S->v[3 * v + c] + h * h * S->p.gravity[c];
        }
}

/* Elastic + inertia gradient and PSD-projected Hessian at xhat. */
static double assemble_elastic(or_scene *S, const double *xtilde, const double *xhat)
{
    double h2 = S->p.dt * S->p.dt;
    double energy = 0.0;
    memset(S->grad, 0, 3 * S->nv * sizeof(double));
    memset(S->val, 0, (size_t)9 * S->nnzb * sizeof(double));
    for (int v = 0; v < S->nv; ++v) {
        int k = find_block(S, v, v);
        for (int c = 0; c < 3; ++c) S->val[9 * k + 4 * c] += S->mass[v];
        if (S->dir[v]) continue;
        for (int c = 0; c < 3; ++c) {
            double dx = xhat[3 * v + c] - xtilde[3 * v + c];
            S->grad[3 * v + c] += S->mass[v] * dx;
            energy += 0.5 * S->mass[v] * dx * dx;
        }
    }
    for (int e = 0; e < S->nt; ++e) {
        double x12[12], g[12], H[144], psi;
        const int *t = S->tets + 4 * e;
        gather12(xhat, t, x12);
        or_elem_grad_hess_model(S->p.model, x12, S->B + 9 * e, S->vol[e], S->emu[e], S->elam[e], 1, &psi, g, H);
        energy += h2 * psi;
        for (int i = 0; i < 4; ++i) {
            for (int c = 0; c < 3; ++c) S->grad[3 * t[i] + c] += h2 * g[3 * i + c];
            for (int j = 0; j < 4; ++j) {
                double *blk = S->val + 9 * S->tmap[16 * e + 4 * i + j];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) blk[3 * a + b] += h2 * H[12 * (3 * i + a) + (3 * j + b)];
            }
        }
    }
    return energy;
}

/* Section 5.2: mu_init = C * max_i (grad^2 E)_ii over free DoFs, here
 * evaluated on the projected Hessian at xhat. */
double or_mu_init(or_scene *S, const double *xhat, const double *xtilde)
{
    assemble_elastic(S, xtilde, xhat);
    double mx = 0.0;
    for (int v = 0; v < S->nv; ++v) {
        if (S->dir[v]) continue;
        int k = find_block(S, v, v);
        for (int c = 0; c < 3; ++c)
            if (S->val[9 * k + 4 * c] > mx) mx = S->val[9 * k + 4 * c];
    }
    S->mu = S->p.c_mu * mx;
    return S->mu;
}

/* Alg. 2, linearisation: d_i(x) and grad d_i(x) at the intersection-free x. */
void or_linearize(or_scene *S, const double *xlin, double *d, double *g)
{
    for (int i = 0; i < S->nc; ++i) {
        int v[4];
        double x12[12];
        pair_verts(S, S->ctype[i], S->ca[i], S->cb[i], v);
        gather12(xlin, v, x12);
        S->cd[i] = or_pair_dist_grad(S->ctype[i], x12, S->cg + 12 * i);
        if (d) d[i] = S->cd[i];
        if (g) memcpy(g + 12 * i, S->cg + 12 * i, 12 * sizeof(double));
    }
}

/* c_i(xhat) = d_i(x) + grad d_i(x)^T (xhat - x) - delta (section 4.2) */
static double constraint_c(const or_scene *S, int i, const double *xlin, const double *xhat)
{
    int v[4];
    pair_verts(S, S->ctype[i], S->ca[i], S->cb[i], v);
    double s = 0.0;
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 3; ++c) s += S->cg[12 * i + 3 * k + c] * (xhat[3 * v[k] + c] - xlin[3 * v[k] + c]);
    return S->cd[i] + s - S->delta;
}

/* ------------------------------------------------------------------ */
/* Semi-implicit friction (appendix A, the model of IPC, Li et al.     */
/* 2020): U_f = sum_i mu_f F_i f0(|u_i|; h eps_v) over the pairs active */
/* at x^t, F_i from the AL state of the previous step and the tangent   */
/* operator fixed at x^t.  Readings: F_i is the magnitude               */
/* h^-2 mu max(0, lambda_i/mu - c_i(x^t)) (the printed expression is    */
/* its negative), with mu, delta and lambda as the previous step left   */
/* them; in the incremental potential h^2 U_f the h^-2 cancels.  u_i is */
/* the relative displacement of the closest points (weights w_k at x^t) */
/* projected on the plane normal to n = (P - Q) / d at x^t, so |u_i|    */
/* needs no basis.  f0(y) = y for y >= eh = h eps_v, else               */
/* -y^3/(3 eh^2) + y^2/eh + eh/3 (C^2 at eh).  Its Hessian in u,        */
/* f0''(y) t t^T + f0'(y)/y (I - t t^T) with t = u/|u|, is PSD as it    */
/* stands (f0'' >= 0, f0' >= 0 here), so no projection is needed.       */
/* ------------------------------------------------------------------ */
double or_friction_f0(double y, double eh, double *f1, double *f2)
{
    if (y >= eh) {
        if (f1) *f1 = 1.0;
        if (f2) *f2 = 0.0;
        return y;
    }
    double s = y / eh;
    if (f1) *f1 = s * (2.0 - s);
    if (f2) *f2 = 2.0 * (1.0 - s) / eh;
    return eh * (s * s * (1.0 - s / 3.0) + 1.0 / 3.0);
}

/* f0'(y) / y, finite at y = 0 */
static double friction_f1_over_y(double y, double eh)
{
    if (y >= eh) return 1.0 / y;
    return (2.0 - y / eh) / eh;
}

/* signed weights w (P - Q = sum_k w_k x_k) and unit normal (P - Q)/d */
static double pair_closest(int type, const double *x, double w[4], double n[3])
{
    double d2;
    if (type == OR_PT) {
        double b[3];
        d2 = pt_closest(x, x + 3, x + 6, x + 9, b);
        w[0] = 1.0; w[1] = -b[0]; w[2] = -b[1]; w[3] = -b[2];
    } else {
        double wa[2], wb[2];
        d2 = ee_closest(x, x + 3, x + 6, x + 9, wa, wb);
        w[0] = wa[0]; w[1] = wa[1]; w[2] = -wb[0]; w[3] = -wb[1];
    }
    double d = sqrt(d2), diff[3] = {0, 0, 0};
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 3; ++c) diff[c] += w[k] * x[3 * k + c];
    for (int c = 0; c < 3; ++c) n[c] = d > 0.0 ? diff[c] / d : 0.0;
    return d;
}

int32_t or_friction_setup(or_scene *S)
{
    S->nf = 0;
    if (!(S->p.mu_f > 0.0) || !(S->mu > 0.0)) return 0;
    if (S->fcap < S->nc) {
        free(S->fv); free(S->fw); free(S->fn); free(S->fk); free(S->fA);
        S->fcap = S->nc;
        S->fv = (int *)xcalloc(4 * S->fcap, sizeof(int));
        S->fw = (double *)xcalloc(4 * S->fcap, sizeof(double));
        S->fn = (double *)xcalloc(3 * S->fcap, sizeof(double));
        S->fk = (double *)xcalloc(S->fcap, sizeof(double));
        S->fA = (double *)xcalloc(9 * S->fcap, sizeof(double));
    }
    for (int i = 0; i < S->nc; ++i) {
        int v[4];
        double x12[12], w[4], n[3];
        pair_verts(S, S->ctype[i], S->ca[i], S->cb[i], v);
        gather12(S->x, v, x12);
        double d = pair_closest(S->ctype[i], x12, w, n);
        double F = S->clam[i] / S->mu - (d - S->delta); /* lambda/mu - c(x^t), times mu below */
        if (!(d > 0.0) || !(F > 0.0)) continue;
        int j = S->nf++;
        memcpy(S->fv + 4 * j, v, sizeof(v));
        memcpy(S->fw + 4 * j, w, sizeof(w));
        memcpy(S->fn + 3 * j, n, sizeof(n));
        S->fk[j] = S->p.mu_f * S->mu * F;
    }
    return S->nf;
}

int32_t or_friction_count(const or_scene *S) { return S->nf; }

void or_friction_get(const or_scene *S, int32_t *v4, double *w4, double *n3, double *k)
{
    if (v4) memcpy(v4, S->fv, 4 * (size_t)S->nf * sizeof(int));
    if (w4) memcpy(w4, S->fw, 4 * (size_t)S->nf * sizeof(double));
    if (n3) memcpy(n3, S->fn, 3 * (size_t)S->nf * sizeof(double));
    if (k) memcpy(k, S->fk, (size_t)S->nf * sizeof(double));
}

/* tangential relative displacement of friction pair j at xhat (from x^t) */
static double friction_slip(const or_scene *S, int j, const double *xhat, double ut[3])
{
    const int *v = S->fv + 4 * j;
    const double *w = S->fw + 4 * j, *n = S->fn + 3 * j;
    double D[3] = {0, 0, 0};
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 3; ++c) D[c] += w[k] * (xhat[3 * v[k] + c] - S->x[3 * v[k] + c]);
    double dn = dot3(D, n);
    for (int c = 0; c < 3; ++c) ut[c] = D[c] - dn * n[c];
    return sqrt(dot3(ut, ut));
}

double or_friction_eval(or_scene *S, const double *xhat, double *grad, double *A9)
{
    double eh = S->p.dt * S->p.eps_v, E = 0.0;
    if (grad) memset(grad, 0, 3 * (size_t)S->nv * sizeof(double));
    for (int j = 0; j < S->nf; ++j) {
        double ut[3], f1, f2;
        double y = friction_slip(S, j, xhat, ut);
        E += S->fk[j] * or_friction_f0(y, eh, &f1, &f2);
        double fy = friction_f1_over_y(y, eh), k = S->fk[j];
        const int *v = S->fv + 4 * j;
        const double *w = S->fw + 4 * j, *n = S->fn + 3 * j;
        if (grad)
            for (int a = 0; a < 4; ++a)
                for (int c = 0; c < 3; ++c) grad[3 * v[a] + c] += k * fy * w[a] * ut[c];
        if (A9) {
            /* k [f0'' t t^T + f0'/y (P - t t^T)], P = I - n n^T, t = ut / y */
            double t[3] = {0, 0, 0};
            if (y > 0.0)
                for (int c = 0; c < 3; ++c) t[c] = ut[c] / y;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double P = (a == b ? 1.0 : 0.0) - n[a] * n[b];
                    double tt = t[a] * t[b];
                    A9[9 * j + 3 * a + b] = y > 0.0 ? k * (f2 * tt + fy * (P - tt)) : k * fy * P;
                }
        }
    }
    return E;
}

/* Alg. 2, Newton system: G and H of E (PSD-projected) plus the AL contact
 * terms with s_i = max(0, c_i - lambda_i/mu); the slack values are kept
 * for the line search.  Dirichlet DoFs are eliminated (section 5.3):
 * their gradient entries are zero and H is applied with their rows and
 * columns zeroed except for the diagonal entries. */
double or_assemble(or_scene *S, const double *xtilde, const double *xlin, const double *xhat, double *grad)
{
    double E = assemble_elastic(S, xtilde, xhat);
    double mu = S->mu;
    for (int i = 0; i < S->nc; ++i) {
        double c = constraint_c(S, i, xlin, xhat);
        double s = c - S->clam[i] / mu;
        if (s < 0.0) s = 0.0;
        S->cs[i] = s;
        double coef = mu * S->cgam[i] * (c - S->clam[i] / mu - s);
        int v[4];
        pair_verts(S, S->ctype[i], S->ca[i], S->cb[i], v);
        for (int k = 0; k < 4; ++k)
            for (int cc = 0; cc < 3; ++cc) S->grad[3 * v[k] + cc] += coef * S->cg[12 * i + 3 * k + cc];
    }
    if (S->nf) { /* friction (appendix A): its gradient, and its Hessian blocks kept in fA */
        double *gf = (double *)xcalloc(3 * S->nv, sizeof(double));
        E += or_friction_eval(S, xhat, gf, S->fA);
        for (int i = 0; i < 3 * S->nv; ++i) S->grad[i] += gf[i];
        free(gf);
    }
    for (int v = 0; v < S->nv; ++v)
        if (S->dir[v])
            for (int c = 0; c < 3; ++c) S->grad[3 * v + c] = 0.0;
    if (grad) memcpy(grad, S->grad, 3 * S->nv * sizeof(double));
    return E;
}

/* slack values s_i of the last or_assemble */
void or_slacks(const or_scene *S, double *s) { memcpy(s, S->cs, S->nc * sizeof(double)); }

/* Per-vertex diagonal 3x3 blocks of the full H (elastic + mass + the
 * contact terms mu gamma_i g_ia g_ia^T + the friction terms w_a^2 A_j),
 * before Dirichlet elimination. */
static double *diag_blocks(const or_scene *S)
{
    double *D = (double *)xcalloc((size_t)9 * S->nv, sizeof(double));
    for (int v = 0; v < S->nv; ++v) memcpy(D + 9 * v, S->val + 9 * find_block(S, v, v), 9 * sizeof(double));
    for (int i = 0; i < S->nc; ++i) {
        int pv[4];
        pair_verts(S, S->ctype[i], S->ca[i], S->cb[i], pv);
        for (int k = 0; k < 4; ++k) {
            const double *g = S->cg + 12 * i + 3 * k;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) D[9 * pv[k] + 3 * a + b] += S->mu * S->cgam[i] * g[a] * g[b];
        }
    }
    for (int j = 0; j < S->nf; ++j)
        for (int k = 0; k < 4; ++k) {
            double w2 = S->fw[4 * j + k] * S->fw[4 * j + k];
            for (int e = 0; e < 9; ++e) D[9 * S->fv[4 * j + k] + e] += w2 * S->fA[9 * j + e];
        }
    return D;
}

void or_hess_apply(const or_scene *S, const double *in, double *out)
{
    int n = 3 * S->nv;
    double *xm = (double *)xcalloc(n, sizeof(double));
    for (int v = 0; v < S->nv; ++v)
        for (int c = 0; c < 3; ++c) xm[3 * v + c] = S->dir[v] ? 0.0 : in[3 * v + c];
    for (int r = 0; r < S->nv; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = S->rp[r]; k < S->rp[r + 1]; ++k)
                for (int b = 0; b < 3; ++b) s += S->val[9 * k + 3 * c + b] * xm[3 * S->ci[k] + b];
            out[3 * r + c] = s;
        }
    /* H += mu gamma_i grad d_i grad d_i^T (Alg. 2, contact Hessian) */
    for (int i = 0; i < S->nc; ++i) {
        int v[4];
        pair_verts(S, S->ctype[i], S->ca[i], S->cb[i], v);
        const double *g = S->cg + 12 * i;
        double t = 0.0;
        for (int k = 0; k < 4; ++k)
            for (int c = 0; c < 3; ++c) t += g[3 * k + c] * xm[3 * v[k] + c];
        t *= S->mu * S->cgam[i];
        for (int k = 0; k < 4; ++k)
            for (int c = 0; c < 3; ++c) out[3 * v[k] + c] += t * g[3 * k + c];
    }
    /* friction (appendix A): block (a, b) of pair j is w_a w_b A_j */
    for (int j = 0; j < S->nf; ++j) {
        const int *v = S->fv + 4 * j;
        const double *w = S->fw + 4 * j, *A = S->fA + 9 * j;
        double D3[3] = {0, 0, 0}, y3[3];
        for (int k = 0; k < 4; ++k)
            for (int c = 0; c < 3; ++c) D3[c] += w[k] * xm[3 * v[k] + c];
        for (int a = 0; a < 3; ++a) y3[a] = (A[3 * a] * D3[0] + A[3 * a + 1] * D3[1]) + A[3 * a + 2] * D3[2];
        for (int k = 0; k < 4; ++k)
            for (int c = 0; c < 3; ++c) out[3 * v[k] + c] += w[k] * y3[c];
    }
    double *D = diag_blocks(S);
    for (int v = 0; v < S->nv; ++v)
        if (S->dir[v])
            for (int c = 0; c < 3; ++c) out[3 * v + c] = D[9 * v + 4 * c] * in[3 * v + c];
    free(D);
    free(xm);
}

void or_hess_dense(const or_scene *S, double *out)
{
    int n = 3 * S->nv;
    double *e = (double *)xcalloc(n, sizeof(double)), *col = (double *)xcalloc(n, sizeof(double));
    for (int j = 0; j < n; ++j) {
        e[j] = 1.0;
        or_hess_apply(S, e, col);
        for (int i = 0; i < n; ++i) out[(size_t)i * n + j] = col[i];
        e[j] = 0.0;
    }
    free(e);
    free(col);
}

/* Block-Jacobi PCG (section 5.1): H x = b, x0 = 0, stop when
 * ||r||_2 <= tol ||b||_2 or after maxit iterations (returns -iters then). */
int32_t or_pcg(const or_scene *S, const double *b, double *x, double tol, int32_t maxit)
{
    int n = 3 * S->nv;
    double *r = (double *)xcalloc(n, sizeof(double)), *z = (double *)xcalloc(n, sizeof(double));
    double *p = (double *)xcalloc(n, sizeof(double)), *q = (double *)xcalloc(n, sizeof(double));
    double *Pinv = (double *)xcalloc(9 * S->nv, sizeof(double));
    double *Dall = diag_blocks(S);
    for (int v = 0; v < S->nv; ++v) {
        double D[9];
        memcpy(D, Dall + 9 * v, sizeof(D));
        if (S->dir[v]) /* eliminated DoFs keep only their diagonal entries */
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    if (a != b) D[3 * a + b] = 0.0;
        inv3(D, Pinv + 9 * v);
    }
    free(Dall);
    double bb = 0.0;
    for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; bb += b[i] * b[i]; }
    int it = 0;
    if (bb == 0.0) goto done;
    double bn = sqrt(bb);
    for (int v = 0; v < S->nv; ++v)
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += Pinv[9 * v + 3 * a + c] * r[3 * v + c];
            z[3 * v + a] = s;
        }
    double rz = 0.0;
    for (int i = 0; i < n; ++i) { p[i] = z[i]; rz += r[i] * z[i]; }
    for (it = 0; it < maxit;) {
        or_hess_apply(S, p, q);
        double pq = 0.0;
        for (int i = 0; i < n; ++i) pq += p[i] * q[i];
        double alpha = rz / pq;
        double rr = 0.0;
        for (int i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            rr += r[i] * r[i];
        }
        ++it;
        if (sqrt(rr) <= tol * bn) break;
        for (int v = 0; v < S->nv; ++v)
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c) s += Pinv[9 * v + 3 * a + c] * r[3 * v + c];
                z[3 * v + a] = s;
            }
        double rz2 = 0.0;
        for (int i = 0; i < n; ++i) rz2 += r[i] * z[i];
        double beta = rz2 / rz;
        rz = rz2;
        for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        if (it == maxit) { it = -it; break; }
    }
done:
    free(r); free(z); free(p); free(q); free(Pinv);
    return it;
}

/* Eq. total-energy with the slack variables held at sfix. */
double or_energy_L(or_scene *S, const double *xtilde, const double *xlin, const double *xhat, const double *sfix)
{
    double h2 = S->p.dt * S->p.dt;
    double L = 0.0;
    for (int v = 0; v < S->nv; ++v) {
        if (S->dir[v]) continue;
        for (int c = 0; c < 3; ++c) {
            double dx = xhat[3 * v + c] - xtilde[3 * v + c];
            L += 0.5 * S->mass[v] * dx * dx;
        }
    }
    for (int e = 0; e < S->nt; ++e) {
        double x12[12], F[9];
        gather12(xhat, S->tets + 4 * e, x12);
        or_elem_F(x12, S->B + 9 * e, F);
        L += h2 * S->vol[e] * or_model_psi(S->p.model, F, S->emu[e], S->elam[e]);
    }
    for (int i = 0; i < S->nc; ++i) {
        double cs = constraint_c(S, i, xlin, xhat) - sfix[i];
        L += S->cgam[i] * (0.5 * S->mu * cs * cs - S->clam[i] * cs);
    }
    if (S->nf) L += or_friction_eval(S, xhat, NULL, NULL);
    return L;
}

/* Alg. 2 SolveSubproblem.  Readings: the line search holds s fixed at the
 * values of the current Newton iteration and accepts
 * L(xhat + r p) <= L(xhat) + 1e-12 max(|L(xhat)|, L_s) for r = 1, 1/2,
 * ..., 2^-max_ls, L_s being |L| at the first Newton iterate of the time step
 * (of this call when called alone).  The paper's strict "<" can loop forever
 * once p ~ 0, and a tolerance relative to |L(xhat)| alone rejects full steps
 * by round-off once L has converged to about zero, as in free fall, where
 * a later subproblem starts at its optimum.  A failed
 * line search ends the Newton loop without a step; the Newton loop is
 * capped at max_newton iterations.  xhat is updated in place and the
 * multipliers and decay factors of C are updated as in the multiplier and decay update of Alg. 2.
 * Returns the number of Newton iterations. */
static int32_t solve_subproblem(or_scene *S, const double *xtilde, const double *xlin, double *xhat,
                                int32_t *cg_iters, int32_t *ls_fail);

int32_t or_solve_subproblem(or_scene *S, const double *xtilde, const double *xlin, double *xhat,
                            int32_t *cg_iters, int32_t *ls_fail)
{
    S->L_scale = -1.0;
    return solve_subproblem(S, xtilde, xlin, xhat, cg_iters, ls_fail);
}

static int32_t solve_subproblem(or_scene *S, const double *xtilde, const double *xlin, double *xhat,
                                int32_t *cg_iters, int32_t *ls_fail)
{
    int n = 3 * S->nv;
    double *g = (double *)xcalloc(n, sizeof(double)), *b = (double *)xcalloc(n, sizeof(double));
    double *pdir = (double *)xcalloc(n, sizeof(double)), *xt = (double *)xcalloc(n, sizeof(double));
    double *sfix = (double *)xcalloc(S->nc, sizeof(double));
    or_linearize(S, xlin, NULL, NULL);
    int newton = 0;
    int32_t cgsum = 0, lsf = 0;
    while (newton < S->p.max_newton) {
        or_assemble(S, xtilde, xlin, xhat, g);
        memcpy(sfix, S->cs, S->nc * sizeof(double));
        for (int i = 0; i < n; ++i) b[i] = -g[i];
        int it = or_pcg(S, b, pdir, S->p.cg_tol, S->p.max_cg);
        cgsum += it < 0 ? -it : it;
        double L0 = or_energy_L(S, xtilde, xlin, xhat, sfix);
        if (S->L_scale < 0.0) S->L_scale = fabs(L0);
        double ls_tol = 1e-12 * fmax(fabs(L0), S->L_scale);
        double r = 1.0;
        int ok = 0;
        for (int j = 0; j <= S->p.max_ls; ++j) {
            for (int i = 0; i < n; ++i) xt[i] = xhat[i] + r * pdir[i];
            double L1 = or_energy_L(S, xtilde, xlin, xt, sfix);
            if (L1 <= L0 + ls_tol) { ok = 1; break; }
            r *= 0.5;
        }
        ++newton;
        if (!ok) { ++lsf; break; }
        memcpy(xhat, xt, n * sizeof(double));
        if (r == 1.0) break;
    }
    /* multiplier and decay update (Alg. 2) */
    for (int i = 0; i < S->nc; ++i) {
        double c = constraint_c(S, i, xlin, xhat);
        double mu = S->mu;
        if (c - S->clam[i] / mu <= 0.0) {
            S->clam[i] = S->clam[i] - mu * c;
            S->cgam[i] = 1.0;
        } else {
            S->clam[i] = 0.0;
            S->cgam[i] = S->p.gamma_decay * S->cgam[i];
        }
    }
    if (cg_iters) *cg_iters = cgsum;
    if (ls_fail) *ls_fail = lsf;
    free(g); free(b); free(pdir); free(xt); free(sfix);
    return newton;
}

/* ------------------------------------------------------------------ */
/* CCD over all primitive pairs (section 5.1 uses an LBVH + ACCD; any    */
/* exact superset works).  Candidates are the PT / EE pairs whose swept  */
/* bounding boxes (all vertices at both ends of the linear motion)       */
/* overlap as closed boxes, excluding pairs that share a vertex and pairs */
/* whose four vertices are all prescribed.                                */
/* ------------------------------------------------------------------ */
typedef struct { int type, a, b; double toi; } hit_t;
typedef struct { hit_t *h; int n, cap; } hitvec;
static void hv_push(hitvec *v, int type, int a, int b, double toi)
{
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 256;
        v->h = (hit_t *)realloc(v->h, v->cap * sizeof(hit_t));
    }
    v->h[v->n].type = type; v->h[v->n].a = a; v->h[v->n].b = b; v->h[v->n].toi = toi;
    v->n++;
}

static void swept_box(const double *x0, const double *x1, const int *v, int nvtx, double lo[3], double hi[3])
{
    for (int c = 0; c < 3; ++c) { lo[c] = INFINITY; hi[c] = -INFINITY; }
    for (int k = 0; k < nvtx; ++k)
        for (int c = 0; c < 3; ++c) {
            double a = x0[3 * v[k] + c], b = x1[3 * v[k] + c];
            lo[c] = fmin(lo[c], fmin(a, b));
            hi[c] = fmax(hi[c], fmax(a, b));
        }
}
static int box_overlap(const double *l1, const double *h1, const double *l2, const double *h2)
{
    for (int c = 0; c < 3; ++c)
        if (l1[c] > h2[c] || l2[c] > h1[c]) return 0;
    return 1;
}

static int pair_admissible(const or_scene *S, int type, int a, int b)
{
    int v[4];
    pair_verts(S, type, a, b, v);
    if (type == OR_PT) {
        if (v[0] == v[1] || v[0] == v[2] || v[0] == v[3]) return 0;
    } else {
        if (v[0] == v[2] || v[0] == v[3] || v[1] == v[2] || v[1] == v[3]) return 0;
    }
    return !(S->dir[v[0]] && S->dir[v[1]] && S->dir[v[2]] && S->dir[v[3]]);
}

static void test_pair(or_scene *S, const double *x0, const double *x1, int type, int a, int b, hitvec *out)
{
    if (!pair_admissible(S, type, a, b)) return;
    int v[4];
    double p0[12], p1[12], toi;
    pair_verts(S, type, a, b, v);
    gather12(x0, v, p0);
    gather12(x1, v, p1);
    if (or_accd(type, p0, p1, S->p.s_ccd, 1.0, OR_ACCD_MAX_ITER, &toi)) hv_push(out, type, a, b, toi);
}

typedef struct { double lo, hi; int kind, id; } sweep_t;
static int cmp_sweep(const void *a, const void *b)
{
    const sweep_t *x = (const sweep_t *)a, *y = (const sweep_t *)b;
    if (x->lo != y->lo) return (x->lo > y->lo) - (x->lo < y->lo);
    if (x->kind != y->kind) return x->kind - y->kind;
    return x->id - y->id;
}

static void ccd_collect(or_scene *S, const double *x0, const double *x1, int brute, hitvec *out)
{
    int nsv = S->nsv, nst = S->nst, nse = S->nse;
    double *vl = (double *)xcalloc(3 * nsv, sizeof(double)), *vh = (double *)xcalloc(3 * nsv, sizeof(double));
    double *tl = (double *)xcalloc(3 * nst, sizeof(double)), *th = (double *)xcalloc(3 * nst, sizeof(double));
    double *el = (double *)xcalloc(3 * nse, sizeof(double)), *eh = (double *)xcalloc(3 * nse, sizeof(double));
    for (int i = 0; i < nsv; ++i) swept_box(x0, x1, S->sv + i, 1, vl + 3 * i, vh + 3 * i);
    for (int i = 0; i < nst; ++i) swept_box(x0, x1, S->st + 3 * i, 3, tl + 3 * i, th + 3 * i);
    for (int i = 0; i < nse; ++i) swept_box(x0, x1, S->se + 2 * i, 2, el + 3 * i, eh + 3 * i);
    if (brute) {
        for (int i = 0; i < nsv; ++i)
            for (int j = 0; j < nst; ++j)
                if (box_overlap(vl + 3 * i, vh + 3 * i, tl + 3 * j, th + 3 * j))
                    test_pair(S, x0, x1, OR_PT, S->sv[i], j, out);
        for (int i = 0; i < nse; ++i)
            for (int j = i + 1; j < nse; ++j)
                if (box_overlap(el + 3 * i, eh + 3 * i, el + 3 * j, eh + 3 * j))
                    test_pair(S, x0, x1, OR_EE, i, j, out);
    } else {
        /* sort-and-sweep along x: same overlap predicate, fewer tests */
        int n = nsv + nst;
        sweep_t *L = (sweep_t *)xcalloc(n, sizeof(sweep_t));
        for (int i = 0; i < nsv; ++i) { L[i].lo = vl[3 * i]; L[i].hi = vh[3 * i]; L[i].kind = 0; L[i].id = i; }
        for (int j = 0; j < nst; ++j) { L[nsv + j].lo = tl[3 * j]; L[nsv + j].hi = th[3 * j]; L[nsv + j].kind = 1; L[nsv + j].id = j; }
        qsort(L, n, sizeof(sweep_t), cmp_sweep);
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n && L[j].lo <= L[i].hi; ++j) {
                if (L[i].kind == L[j].kind) continue;
                int vi = L[i].kind == 0 ? L[i].id : L[j].id, ti = L[i].kind == 1 ? L[i].id : L[j].id;
                if (box_overlap(vl + 3 * vi, vh + 3 * vi, tl + 3 * ti, th + 3 * ti))
                    test_pair(S, x0, x1, OR_PT, S->sv[vi], ti, out);
            }
        free(L);
        L = (sweep_t *)xcalloc(nse, sizeof(sweep_t));
        for (int i = 0; i < nse; ++i) { L[i].lo = el[3 * i]; L[i].hi = eh[3 * i]; L[i].kind = 0; L[i].id = i; }
        qsort(L, nse, sizeof(sweep_t), cmp_sweep);
        for (int i = 0; i < nse; ++i)
            for (int j = i + 1; j < nse && L[j].lo <= L[i].hi; ++j) {
                int a = L[i].id < L[j].id ? L[i].id : L[j].id, b = L[i].id < L[j].id ? L[j].id : L[i].id;
                if (box_overlap(el + 3 * a, eh + 3 * a, el + 3 * b, eh + 3 * b)) test_pair(S, x0, x1, OR_EE, a, b, out);
            }
        free(L);
    }
    free(vl); free(vh); free(tl); free(th); free(el); free(eh);
}

int32_t or_ccd_hits(or_scene *S, const double *x0, const double *x1, int32_t brute, int32_t cap,
                    int32_t *keys, double *toi)
{
    hitvec hv = {0, 0, 0};
    ccd_collect(S, x0, x1, brute, &hv);
    for (int i = 0; i < hv.n && i < cap; ++i) {
        if (keys) canon_key(S, hv.h[i].type, hv.h[i].a, hv.h[i].b, keys + 5 * i);
        if (toi) toi[i] = hv.h[i].toi;
    }
    int n = hv.n;
    free(hv.h);
    return n;
}

/* Alg. 3 UpdateActiveSet(x, xhat, C).  Reading of its intersection step: the
 * intersecting pairs are the CCD hits (t <= 1) along x -> xhat. */
int32_t or_update_active_set(or_scene *S, const double *x, const double *xhat)
{
    hitvec hv = {0, 0, 0};
    ccd_collect(S, x, xhat, 0, &hv);
    /* I' <- I' \ I_C */
    int64_t *ck = (int64_t *)xcalloc(S->nc, sizeof(int64_t));
    for (int i = 0; i < S->nc; ++i) ck[i] = pair_key(S->ctype[i], S->ca[i], S->cb[i]);
    qsort(ck, S->nc, sizeof(int64_t), cmp_i64);
    int nn = 0;
    for (int i = 0; i < hv.n; ++i) {
        int64_t k = pair_key(hv.h[i].type, hv.h[i].a, hv.h[i].b);
        if (S->nc && bsearch(&k, ck, S->nc, sizeof(int64_t), cmp_i64)) continue;
        hv.h[nn++] = hv.h[i];
    }
    free(ck);
    /* T_v = min over new pairs containing v (Alg. 3, per-vertex minimum) */
    double *Tv = (double *)xcalloc(S->nv, sizeof(double));
    for (int v = 0; v < S->nv; ++v) Tv[v] = INFINITY;
    for (int i = 0; i < nn; ++i) {
        int v[4];
        pair_verts(S, hv.h[i].type, hv.h[i].a, hv.h[i].b, v);
        for (int k = 0; k < 4; ++k)
            if (hv.h[i].toi < Tv[v[k]]) Tv[v[k]] = hv.h[i].toi;
    }
    /* keep pairs whose T_i equals T_v of one of their vertices (Alg. 3, filter) */
    for (int i = 0; i < nn; ++i) {
        int v[4];
        pair_verts(S, hv.h[i].type, hv.h[i].a, hv.h[i].b, v);
        int keep = 0;
        for (int k = 0; k < 4; ++k)
            if (hv.h[i].toi == Tv[v[k]]) keep = 1;
        if (!keep) continue;
        c_reserve(S, S->nc + 1);
        S->ctype[S->nc] = hv.h[i].type; S->ca[S->nc] = hv.h[i].a; S->cb[S->nc] = hv.h[i].b;
        S->clam[S->nc] = 0.0; S->cgam[S->nc] = 1.0;
        S->nc++;
    }
    free(Tv);
    free(hv.h);
    /* prune gamma < 0.01 (Alg. 3, decay pruning) */
    int m = 0;
    for (int i = 0; i < S->nc; ++i) {
        if (S->cgam[i] < 0.01) continue;
        S->ctype[m] = S->ctype[i]; S->ca[m] = S->ca[i]; S->cb[m] = S->cb[i];
        S->clam[m] = S->clam[i]; S->cgam[m] = S->cgam[i];
        ++m;
    }
    S->nc = m;
    return m;
}

/* Inversion-aware step bound (section 4.1: for a non-invertible material
 * such as NH, MaxStepSize also keeps the trajectory inversion-free).
 * Reading: along x0 + t (x1 - x0) each element's J(t) = det F(t), a cubic
 * in t, may fall to the fraction s_ccd of J(0) and no further, the same
 * fraction ACCD keeps of a gap; the bound is the smallest t in (0, 1] with
 * J(t) = s J(0) over the elements with a free vertex, else 1.  An element
 * with J(0) <= 0 allows no step (0). */
double or_inversion_step(or_scene *S, const double *x0, const double *x1)
{
    double a = 1.0;
    for (int e = 0; e < S->nt; ++e) {
        const int *t = S->tets + 4 * e;
        if (S->dir[t[0]] && S->dir[t[1]] && S->dir[t[2]] && S->dir[t[3]]) continue;
        double xa[12], xb[12], dx[12], F0[9], dF[9], c[4];
        gather12(x0, t, xa);
        gather12(x1, t, xb);
        for (int k = 0; k < 12; ++k) dx[k] = xb[k] - xa[k];
        or_elem_F(xa, S->B + 9 * e, F0);
        or_elem_F(dx, S->B + 9 * e, dF); /* F is linear in x: F(t) = F0 + t dF */
        or_det_cubic(F0, dF, S->p.s_ccd, c);
        double te = or_cubic_first_root(c);
        if (te < a) a = te;
    }
    return a;
}

/* MaxStepSize (section 4.1): alpha = min(1, min_i TOI_i) over x0 -> x1,
 * and for NH also at most the inversion bound. */
double or_max_step_size(or_scene *S, const double *x0, const double *x1)
{
    hitvec hv = {0, 0, 0};
    ccd_collect(S, x0, x1, 0, &hv);
    double a = 1.0;
    for (int i = 0; i < hv.n; ++i)
        if (hv.h[i].toi < a) a = hv.h[i].toi;
    free(hv.h);
    if (S->p.model == 2) {
        double ai = or_inversion_step(S, x0, x1);
        if (ai < a) a = ai;
    }
    return a;
}

/* Gradient-norm residual of IPC (section 6, convergence of the
 * gradient-norm residual): r = (1/h) |H^-1 grad L|_inf.  Reading: at an
 * outer iterate x = x^[k], L is the next subproblem's energy (Eq.
 * total-energy linearised at x, with the current active set, multipliers,
 * decay factors, mu and delta, the slacks at their optimal values) taken at
 * xhat = x, and H its projected Hessian; the solve is the same PCG. */
double or_newton_residual(or_scene *S, const double *xtilde, const double *x)
{
    int n = 3 * S->nv;
    double *g = (double *)xcalloc(n, sizeof(double)), *p = (double *)xcalloc(n, sizeof(double));
    or_linearize(S, x, NULL, NULL);
    or_assemble(S, xtilde, x, x, g);
    or_pcg(S, g, p, S->p.cg_tol, S->p.max_cg);
    double m = 0.0;
    for (int i = 0; i < n; ++i)
        if (fabs(p[i]) > m) m = fabs(p[i]);
    free(g);
    free(p);
    return m / S->p.dt;
}

int32_t or_get_residual_log(const or_scene *S, int32_t cap, double *out)
{
    for (int i = 0; i < S->nres && i < cap; ++i) out[i] = S->res[i];
    return S->nres;
}

static void res_push(or_scene *S, double r)
{
    if (S->nres == S->rescap) {
        S->rescap = S->rescap ? 2 * S->rescap : 64;
        S->res = (double *)realloc(S->res, S->rescap * sizeof(double));
    }
    S->res[S->nres++] = r;
}

/* Minimum unsigned distance over all admissible PT / EE pairs at x. */
int32_t or_min_distance(or_scene *S, const double *x, double *dmin)
{
    double best = INFINITY;
    int cnt = 0;
    for (int i = 0; i < S->nsv; ++i)
        for (int j = 0; j < S->nst; ++j) {
            if (!pair_admissible(S, OR_PT, S->sv[i], j)) continue;
            int v[4];
            double x12[12];
            pair_verts(S, OR_PT, S->sv[i], j, v);
            gather12(x, v, x12);
            double d = pair_dist2(OR_PT, x12);
            if (d < best) best = d;
            ++cnt;
        }
    for (int i = 0; i < S->nse; ++i)
        for (int j = i + 1; j < S->nse; ++j) {
            if (!pair_admissible(S, OR_EE, i, j)) continue;
            int v[4];
            double x12[12];
            pair_verts(S, OR_EE, i, j, v);
            gather12(x, v, x12);
            double d = pair_dist2(OR_EE, x12);
            if (d < best) best = d;
            ++cnt;
        }
    *dmin = sqrt(best);
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Alg. 1: one time step per iteration of the outer loop below.          */
/* Readings: mu_init is evaluated at xhat^[0] each time step; the stall  */
/* rule of section 5.2 (alpha < 1e-4 for 50 consecutive iterations ->   */
/* mu *= 2, delta /= 2) acts within the step, and delta is reset each    */
/* step; the outer loop is capped at max_outer (status -7).  With        */
/* ccd_reuse the active set is updated from the MaxStepSize segment      */
/* x^[k] -> xhat^[k+1] instead of Alg. 1's x^[k] -> xhat^[k]: one CCD    */
/* per outer iteration, fitted to the constraint-set expansion (the      */
/* direction the paper's conclusion names); the pairs that cut this step */
/* join C one iteration earlier.  With                                   */
/* res_tol > 0 the loop ends instead once the gradient-norm residual at  */
/* x^[k] falls below res_tol (the IPC-style termination of section 6),   */
/* checked before each outer iteration, from x^[0] = x^t on.             */
/* ------------------------------------------------------------------ */
/* The intermediate states xhat^[1], xhat^[2], ... of the outer iterations
 * of the following or_step calls are copied into buf (cap states of 3 nv
 * doubles; NULL stops the log); returns the count logged so far.  Test
 * hook for the expansion of x^[k] in the termination criterion. */
int32_t or_set_xhat_log(or_scene *S, double *buf, int32_t cap)
{
    S->xhat_log = buf;
    S->xhat_cap = buf ? cap : 0;
    S->xhat_n = 0;
    return 0;
}

int32_t or_xhat_log_count(const or_scene *S) { return S->xhat_n; }

int32_t or_step(or_scene *S, int32_t nsteps, or_stats *stats, double *alpha_log, int32_t alpha_cap)
{
    int n = 3 * S->nv;
    double *xt = (double *)xcalloc(n, sizeof(double)), *xtilde = (double *)xcalloc(n, sizeof(double));
    double *xk = (double *)xcalloc(n, sizeof(double)), *xh = (double *)xcalloc(n, sizeof(double));
    double *xhn = (double *)xcalloc(n, sizeof(double));
    int status = 0, alog = 0;
    for (int step = 0; step < nsteps; ++step) {
        or_stats st;
        memset(&st, 0, sizeof(st));
        st.min_alpha = 1.0;
        memcpy(xt, S->x, n * sizeof(double));
        or_xtilde(S, xtilde);
        memcpy(xk, S->x, n * sizeof(double));
        memcpy(xh, S->x, n * sizeof(double));
        if (S->has_targets)
            for (int v = 0; v < S->nv; ++v)
                if (S->dir[v])
                    for (int c = 0; c < 3; ++c) xh[3 * v + c] = S->targets[3 * v + c];
        or_friction_setup(S); /* from the AL state the previous step left (appendix A) */
        S->delta = S->p.delta;
        S->L_scale = -1.0; /* set by the step's first Newton iterate */
        or_mu_init(S, xh, xtilde);
        double beta = 1.0, asum = 0.0;
        int k = 0, stall = 0;
        const int resmode = S->p.res_tol > 0.0;
        S->nres = 0;
        for (;;) {
            if (resmode) {
                double r = or_newton_residual(S, xtilde, xk);
                res_push(S, r);
                if (r < S->p.res_tol) break;
            } else if (!(beta > S->p.eps)) {
                break;
            }
            if (k >= S->p.max_outer) { status = -7; break; }
            memcpy(xhn, xh, n * sizeof(double));
            int32_t cgi = 0, lsf = 0;
            st.newton_iters += solve_subproblem(S, xtilde, xk, xhn, &cgi, &lsf);
            st.cg_iters += cgi;
            st.ls_fail += lsf;
            or_update_active_set(S, xk, S->p.ccd_reuse ? xhn : xh);
            if (S->xhat_log && S->xhat_n < S->xhat_cap)
                memcpy(S->xhat_log + (size_t)n * S->xhat_n++, xhn, n * sizeof(double));
            double alpha = or_max_step_size(S, xk, xhn);
            for (int i = 0; i < n; ++i) xk[i] = (1.0 - alpha) * xk[i] + alpha * xhn[i];
            if (k + 1 >= S->p.k_min) beta = (1.0 - alpha) * beta;
            ++k;
            memcpy(xh, xhn, n * sizeof(double));
            asum += alpha;
            if (alpha < st.min_alpha) st.min_alpha = alpha;
            if (alpha_log && alog < alpha_cap) alpha_log[alog++] = alpha;
            if (alpha < 1e-4) {
                if (++stall >= 50) { S->mu *= 2.0; S->delta *= 0.5; stall = 0; st.stalls++; }
            } else stall = 0;
        }
        for (int i = 0; i < n; ++i) S->v[i] = (xk[i] - xt[i]) / S->p.dt;
        memcpy(S->x, xk, n * sizeof(double));
        st.outer_iters = k;
        st.n_contacts = S->nc;
        st.mean_alpha = k ? asum / k : 0.0;
        st.mu = S->mu;
        st.beta = beta;
        st.delta = S->delta;
        st.status = status;
        if (stats) stats[step] = st;
        if (status) break;
    }
    free(xt); free(xtilde); free(xk); free(xh); free(xhn);
    return status;
}
