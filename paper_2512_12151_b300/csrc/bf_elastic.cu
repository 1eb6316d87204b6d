// Elasticity of the incremental potential (section 3) with the stable
// Neo-Hookean energy Psi = mu/2 (|F|^2 - 3) - mu (J - 1) + lam/2 (J - 1)^2,
// lam = lambda_Lame + mu (the model is named in the Tab. 2 caption; the
// Lame shift makes the small-strain limit linear elasticity).
//
// Element kernel (one thread per tet): the gradient in FP64 from
// P = mu F + (lam (J - 1) - mu) cof(F); the PSD-projected Hessian of
// section 5.1 from the analytic eigensystem of d2Psi/dF2 in the frame of
// the rotation-variant SVD F = U Sigma V^T.  With a_i' = V^T A_i' (A_i' the
// rows mapping dx_i' to dF), each 3x3 vertex block is U M U^T with
//   M_pp = S_pp a_p b_p + sum_{q != p} c1_pq a_q b_q,
//   M_pq = S_pq a_p b_q + c2_pq a_q b_p          (p != q),
// where S is the PSD-projected 3x3 "scaling" block, and for each axis pair
// (p, q) with third axis k the twist / flip eigenvalues are
// mu +/- (lam (J - 1) - mu) sigma_k, c1 = (w_t+ + w_f+)/2, c2 = (w_f+ - w_t+)/2.
// This is the vertex-block form of section 5.1 with the sparse D_k folded in.
//
// The Neo-Hookean energy (NH, Tab. 2) Psi = mu/2 (|F|^2 - 3) - mu ln J +
// lam/2 (ln J)^2 (lam the Lame constant) has the same structure with
// kappa = (lam ln J - mu) / J in place of lam (J - 1) - mu: P = mu F +
// kappa cof(F), twist / flip eigenvalues mu +/- kappa sigma_k (that is,
// (Psi_p +/- Psi_q) / (sigma_p +/- sigma_q)), and the scaling block
// d2Psi/dsigma_p dsigma_q = lam / (sigma_p sigma_q) + [p = q] (mu +
// (mu - lam ln J) / sigma_p^2).
#include <cuda_runtime.h>

#include <cmath>

#include "bf_device.cuh"
#include "bf_friction.cuh"
#include "bf_internal.cuh"

namespace bf {

template <class T>
__device__ __forceinline__ T my_sqrt(T v);
template <>
__device__ __forceinline__ double my_sqrt<double>(double v) { return sqrt(v); }
template <>
__device__ __forceinline__ float my_sqrt<float>(float v) { return sqrtf(v); }

// cyclic Jacobi on a symmetric 3x3: A = V diag(w) V^T
template <class T>
__device__ void sym3_eig(T a[3][3], T w[3], T V[3][3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? T(1) : T(0);
    const T eps = sizeof(T) == 8 ? T(1e-30) : T(1e-13);
    for (int sweep = 0; sweep < (sizeof(T) == 8 ? 16 : 10); ++sweep) {
        const T off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const T dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= eps * dia || off == T(0)) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
            const T apq = a[p][q];
            if (apq == T(0)) continue;
            const T theta = (a[q][q] - a[p][p]) / (T(2) * apq);
            T t;
            if (fabs((double)theta) > 1e15) t = T(0.5) / theta;
            else t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + my_sqrt<T>(theta * theta + T(1)));
            const T c = T(1) / my_sqrt<T>(t * t + T(1)), s = t * c;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T akp = a[k][p], akq = a[k][q];
                a[k][p] = c * akp - s * akq;
                a[k][q] = s * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T apk = a[p][k], aqk = a[q][k];
                a[p][k] = c * apk - s * aqk;
                a[q][k] = s * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - s * vkq;
                V[k][q] = s * vkp + c * vkq;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) w[i] = a[i][i];
}

// rotation-variant SVD F = U diag(s) V^T with U, V in SO(3); s[2] may be < 0
template <class T>
__device__ void svd3(const T F[3][3], T U[3][3], T s[3], T V[3][3])
{
    T A[3][3], w[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
    sym3_eig<T>(A, w, V);
    // sort eigenvalues descending (columns of V follow)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2 - i; ++j)
            if (w[j] < w[j + 1]) {
                T tw = w[j];
                w[j] = w[j + 1];
                w[j + 1] = tw;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    T tv = V[k][j];
                    V[k][j] = V[k][j + 1];
                    V[k][j + 1] = tv;
                }
            }
    const T detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                   V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
    if (detV < T(0))
#pragma unroll
        for (int k = 0; k < 3; ++k) V[k][2] = -V[k][2];
    T Bc[3][3];  // B = F V, columns b_j
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Bc[i][j] = F[i][0] * V[0][j] + F[i][1] * V[1][j] + F[i][2] * V[2][j];
    const T tiny = sizeof(T) == 8 ? T(1e-150) : T(1e-30);
    // u0
    T n0 = my_sqrt<T>(Bc[0][0] * Bc[0][0] + Bc[1][0] * Bc[1][0] + Bc[2][0] * Bc[2][0]);
    T u0[3];
    if (n0 > tiny) {
        u0[0] = Bc[0][0] / n0; u0[1] = Bc[1][0] / n0; u0[2] = Bc[2][0] / n0;
    } else {
        u0[0] = T(1); u0[1] = T(0); u0[2] = T(0);
    }
    // u1: b1 orthogonalised against u0
    const T pr = u0[0] * Bc[0][1] + u0[1] * Bc[1][1] + u0[2] * Bc[2][1];
    T w1[3] = {Bc[0][1] - pr * u0[0], Bc[1][1] - pr * u0[1], Bc[2][1] - pr * u0[2]};
    T n1 = my_sqrt<T>(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
    T u1[3];
    if (n1 > tiny * (n0 > T(1) ? n0 : T(1))) {
        u1[0] = w1[0] / n1; u1[1] = w1[1] / n1; u1[2] = w1[2] / n1;
    } else {  // any unit vector orthogonal to u0
        T e[3] = {T(0), T(0), T(0)};
        const int m = (fabs(u0[0]) < fabs(u0[1])) ? ((fabs(u0[0]) < fabs(u0[2])) ? 0 : 2) : ((fabs(u0[1]) < fabs(u0[2])) ? 1 : 2);
        e[m] = T(1);
        T c[3] = {u0[1] * e[2] - u0[2] * e[1], u0[2] * e[0] - u0[0] * e[2], u0[0] * e[1] - u0[1] * e[0]};
        T nc = my_sqrt<T>(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        u1[0] = c[0] / nc; u1[1] = c[1] / nc; u1[2] = c[2] / nc;
        n1 = T(0);
    }
    T u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2], u0[0] * u1[1] - u0[1] * u1[0]};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        U[i][0] = u0[i];
        U[i][1] = u1[i];
        U[i][2] = u2[i];
    }
    s[0] = n0;
    s[1] = n1;
    s[2] = u2[0] * Bc[0][2] + u2[1] * Bc[1][2] + u2[2] * Bc[2][2];
}

__device__ __forceinline__ void atomic_add_val(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_val(float *p, double v) { atomicAdd(p, (float)v); }

// Per-tet gradient and PSD Hessian; HT is the Hessian arithmetic type and
// MT the storage type of the block values.  MODEL BF_MODEL_COR: the
// corotated energy Psi = mu |F - R|^2 + lam/2 (tr S - 3)^2 (F = R S, R from
// the rotation-variant SVD), P = 2 mu (F - R) + lam (tr S - 3) R in FP64
// (its own FP64 SVD); in the SVD frame its Hessian has the scaling block
// 2 mu I + lam 1 1^T (PSD for lam >= 0), flip eigenvalues 2 mu and twist
// eigenvalues (Psi_p + Psi_q) / (s_p + s_q) with Psi_p = 2 mu (s_p - 1) +
// lam (tr S - 3), the same assembly as SNH's.
template <class HT, class MT, int MODEL>
__global__ void __launch_bounds__(128) k_elastic(int nt, const int4 *__restrict__ tets, const double *__restrict__ Bm,
                                                 const double *__restrict__ vol, const double *__restrict__ emu,
                                                 const double *__restrict__ elam, const uint8_t *__restrict__ dir,
                                                 const double *__restrict__ xh, double h2, double *__restrict__ grad,
                                                 MT *__restrict__ val, int nnzb, const int *__restrict__ tblk)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt) return;
    const int4 t4 = tets[e];
    const int vid[4] = {t4.x, t4.y, t4.z, t4.w};
    double X[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) X[k][c] = xh[3 * vid[k] + c];
    double B[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) B[k] = Bm[9 * (size_t)e + k];
    const double V0 = vol[e], mu = emu[e], lam = elam[e];
    // F = Ds B, Ds columns x_k - x_0
    double F[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            F[r][c] = (X[1][r] - X[0][r]) * B[c] + (X[2][r] - X[0][r]) * B[3 + c] + (X[3][r] - X[0][r]) * B[6 + c];
    double A[4][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        A[1][c] = B[c];
        A[2][c] = B[3 + c];
        A[3][c] = B[6 + c];
        A[0][c] = -(B[c] + B[3 + c] + B[6 + c]);
    }
    HT Ft[3][3], U[3][3], s[3], V[3][3];
    const HT muT = (HT)mu, lamT = (HT)lam;
    HT c1[3][3], c2[3][3], S3[3][3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            c1[p][q] = HT(0);
            c2[p][q] = HT(0);
        }
    if constexpr (MODEL == BF_MODEL_COR) {
        double Ud[3][3], sd[3], Vd[3][3], R[3][3];
        svd3<double>(F, Ud, sd, Vd);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) R[r][c] = Ud[r][0] * Vd[c][0] + Ud[r][1] * Vd[c][1] + Ud[r][2] * Vd[c][2];
        const double trm3 = sd[0] + sd[1] + sd[2] - 3.0;
        const double sc = h2 * V0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (dir[vid[i]]) continue;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                double g = 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c) g += (2.0 * mu * (F[r][c] - R[r][c]) + lam * trm3 * R[r][c]) * A[i][c];
                atomicAdd(grad + 3 * vid[i] + r, sc * g);
            }
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            s[r] = (HT)sd[r];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                U[r][c] = (HT)Ud[r][c];
                V[r][c] = (HT)Vd[r][c];
            }
        }
        const HT t3 = (HT)trm3;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
            const int p = kk == 0 ? 1 : 0, q = kk == 2 ? 1 : 2;
            const HT den = s[p] + s[q];
            const HT num = HT(2) * muT * (s[p] + s[q] - HT(2)) + HT(2) * lamT * t3;
            HT wt = den > HT(1e-30) || den < HT(-1e-30) ? num / den : HT(0);
            HT wf = HT(2) * muT;
            wt = wt > HT(0) ? wt : HT(0);
            c1[p][q] = c1[q][p] = HT(0.5) * (wt + wf);
            c2[p][q] = c2[q][p] = HT(0.5) * (wf - wt);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) S3[p][q] = lamT + (p == q ? HT(2) * muT : HT(0));
    } else {
    double Jd = 1.0, lnJ = 0.0;  // NH: J and ln J in FP64
    // ---- gradient (FP64) ----
    {
        double C[3][3];  // cofactor: columns f1 x f2, f2 x f0, f0 x f1
        C[0][0] = F[1][1] * F[2][2] - F[2][1] * F[1][2];
        C[1][0] = F[2][1] * F[0][2] - F[0][1] * F[2][2];
        C[2][0] = F[0][1] * F[1][2] - F[1][1] * F[0][2];
        C[0][1] = F[1][2] * F[2][0] - F[2][2] * F[1][0];
        C[1][1] = F[2][2] * F[0][0] - F[0][2] * F[2][0];
        C[2][1] = F[0][2] * F[1][0] - F[1][2] * F[0][0];
        C[0][2] = F[1][0] * F[2][1] - F[2][0] * F[1][1];
        C[1][2] = F[2][0] * F[0][1] - F[0][0] * F[2][1];
        C[2][2] = F[0][0] * F[1][1] - F[1][0] * F[0][1];
        const double J = F[0][0] * C[0][0] + F[1][0] * C[1][0] + F[2][0] * C[2][0];
        if (MODEL == BF_MODEL_NH) {
            Jd = J;
            lnJ = log(J);
        }
        const double k = MODEL == BF_MODEL_NH ? (lam * lnJ - mu) / J : lam * (J - 1.0) - mu;
        const double sc = h2 * V0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (dir[vid[i]]) continue;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double g = (mu * F[r][0] + k * C[r][0]) * A[i][0] + (mu * F[r][1] + k * C[r][1]) * A[i][1] +
                                 (mu * F[r][2] + k * C[r][2]) * A[i][2];
                atomicAdd(grad + 3 * vid[i] + r, sc * g);
            }
        }
    }
    // ---- PSD Hessian in HT ----
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Ft[r][c] = (HT)F[r][c];
    svd3<HT>(Ft, U, s, V);
    const HT J = s[0] * s[1] * s[2];
    const HT kap = MODEL == BF_MODEL_NH ? (HT)((lam * lnJ - mu) / Jd) : lamT * (J - HT(1)) - muT;
    // twist / flip pairs: (0,1) third 2, (0,2) third 1, (1,2) third 0
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        const int p = kk == 0 ? 1 : 0, q = kk == 2 ? 1 : 2;
        HT wt = muT + kap * s[kk], wf = muT - kap * s[kk];
        wt = wt > HT(0) ? wt : HT(0);
        wf = wf > HT(0) ? wf : HT(0);
        c1[p][q] = c1[q][p] = HT(0.5) * (wt + wf);
        c2[p][q] = c2[q][p] = HT(0.5) * (wf - wt);
    }
    // scaling block, PSD-projected: SNH A3 = mu I + kap [[0 s2 s1][s2 0 s0][s1 s0 0]] + lam g g^T;
    // NH A3 = lam r r^T + diag(mu + (mu - lam ln J) r_p^2), r = 1 / s
    {
        HT A3[3][3];
        if (MODEL == BF_MODEL_NH) {
            const HT r[3] = {HT(1) / s[0], HT(1) / s[1], HT(1) / s[2]};
            const HT dl = (HT)(mu - lam * lnJ);
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) A3[p][q] = lamT * r[p] * r[q] + (p == q ? muT + dl * r[p] * r[p] : HT(0));
        } else {
            const HT g[3] = {s[1] * s[2], s[0] * s[2], s[0] * s[1]};
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) A3[p][q] = lamT * g[p] * g[q] + (p == q ? muT : kap * s[3 - p - q]);
        }
        HT w[3], E[3][3];
        sym3_eig<HT>(A3, w, E);
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                HT acc = HT(0);
#pragma unroll
                for (int m = 0; m < 3; ++m) acc += (w[m] > HT(0) ? w[m] : HT(0)) * E[p][m] * E[q][m];
                S3[p][q] = acc;
            }
    }
    }  // model
    // a_i' = V^T A_i'
    HT a[4][3];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int p = 0; p < 3; ++p)
            a[i][p] = V[0][p] * (HT)A[i][0] + V[1][p] * (HT)A[i][1] + V[2][p] * (HT)A[i][2];
    const HT sc = (HT)(h2 * V0);
    int pair = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j, ++pair) {
            if (dir[vid[i]] || dir[vid[j]]) continue;
            HT M[3][3];
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (p == q) {
                        HT acc = S3[p][p] * a[i][p] * a[j][p];
#pragma unroll
                        for (int m = 0; m < 3; ++m)
                            if (m != p) acc += c1[p][m] * a[i][m] * a[j][m];
                        M[p][q] = acc;
                    } else {
                        M[p][q] = S3[p][q] * a[i][p] * a[j][q] + c2[p][q] * a[i][q] * a[j][p];
                    }
                }
            // H = sc * U M U^T
            HT T1[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int q = 0; q < 3; ++q) T1[r][q] = U[r][0] * M[0][q] + U[r][1] * M[1][q] + U[r][2] * M[2][q];
            const int tb = tblk[10 * (size_t)e + pair];
            const int blk = tb & 0x7fffffff;
            const bool tr = (tb >> 31) & 1;
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const HT h = sc * (T1[r][0] * U[c][0] + T1[r][1] * U[c][1] + T1[r][2] * U[c][2]);
                    const int ent = tr ? (3 * c + r) : (3 * r + c);
                    atomic_add_val(val + 9 * (size_t)blk + ent, (double)h);
                }
        }
}

// FP32 copy of the FP64 block sums (mixed precision)
__global__ void k_round_blocks(size_t n, const double *__restrict__ v64, float *__restrict__ v32)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v32[i] = (float)v64[i];
}

void launch_elastic(Scene &S, const double *xhat)
{
    if (S.nt == 0) return;
    const double h2 = S.prm.dt * S.prm.dt;
    ScopedTimer tm(S, T_ELASTIC);
    const int nb = cdiv(S.nt, 128);
    const int m = S.prm.model;
    if (S.prm.precision == BF_PREC_MIXED) {
        // FP32 element Hessians, summed into the blocks in FP64 and stored
        // in FP32: the order of the atomics then moves only the last bits
        // of an FP64 sum, which the FP32 rounding almost always hides, so
        // a step does not depend on the scheduling of its kernels (scenes
        // alone or in a batch take the same steps)
        auto kern = m == BF_MODEL_COR  ? k_elastic<float, double, BF_MODEL_COR>
                    : m == BF_MODEL_NH ? k_elastic<float, double, BF_MODEL_NH>
                                       : k_elastic<float, double, BF_MODEL_SNH>;
        kern<<<nb, 128, 0, S.stream>>>(S.nt, S.tets, S.B, S.vol, S.emu, S.elam, S.dir, xhat, h2, S.grad, S.val,
                                       S.nnzb, S.tblk);
        ++S.n_launch;
        const size_t nval = 9 * (size_t)S.nnzb;
        k_round_blocks<<<cdiv((long long)nval, kThreads), kThreads, 0, S.stream>>>(nval, S.val, S.valf);
    } else {
        auto kern = m == BF_MODEL_COR  ? k_elastic<double, double, BF_MODEL_COR>
                    : m == BF_MODEL_NH ? k_elastic<double, double, BF_MODEL_NH>
                                       : k_elastic<double, double, BF_MODEL_SNH>;
        kern<<<nb, 128, 0, S.stream>>>(S.nt, S.tets, S.B, S.vol, S.emu, S.elam, S.dir, xhat, h2, S.grad, S.val,
                                       S.nnzb, S.tblk);
    }
    ++S.n_launch;
}

// inertia gradient M (xhat - x~) and mass on the diagonal blocks; prescribed
// vertices get a zero gradient and an identity diagonal block
template <class MT>
__global__ void k_vertex_init(int nv, int nnzb, const int *__restrict__ diagblk, const double *__restrict__ mass,
                              const uint8_t *__restrict__ dir, const double *__restrict__ xt,
                              const double *__restrict__ xh, double *__restrict__ grad, MT *__restrict__ val,
                              double *__restrict__ cdiag)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nv) return;
    const int k = diagblk[a];
    const bool d = dir[a];
    const double m = d ? 1.0 : mass[a];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        grad[3 * a + c] = d ? 0.0 : m * (xh[3 * a + c] - xt[3 * a + c]);
        val[9 * (size_t)k + 4 * c] = (MT)m;
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) cdiag[9 * (size_t)a + e] = 0.0;
}

void launch_vertex_init(Scene &S, const double *xtilde, const double *xhat)
{
    const int nb = cdiv(S.nv, kThreads);
    // the blocks are summed in FP64 in both precisions (launch_elastic)
    cudaMemsetAsync(S.val, 0, 9 * (size_t)S.nnzb * sizeof(double), S.stream);
    k_vertex_init<double><<<nb, kThreads, 0, S.stream>>>(S.nv, S.nnzb, S.diagblk, S.mass, S.dir, xtilde, xhat,
                                                         S.grad, S.val, S.cdiag); ++S.n_launch;
}

// max over free DoFs of the diagonal entries (section 5.2 mu_init)
template <class MT>
__global__ void k_max_diag(int nv, int nnzb, const int *__restrict__ diagblk, const uint8_t *__restrict__ dir,
                           const MT *__restrict__ val, double *out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (a < nv && !dir[a]) {
        const int k = diagblk[a];
        for (int c = 0; c < 3; ++c) m = fmax(m, (double)val[9 * (size_t)k + 4 * c]);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomic_max_pos(out, m);
}

double run_mu_max_diag(Scene &S)
{
    cudaMemsetAsync(S.dscal + S_MAXDIAG, 0, sizeof(double), S.stream);
    const int nb = cdiv(S.nv, kThreads);
    if (S.prm.precision == BF_PREC_MIXED)
        {
            k_max_diag<float><<<nb, kThreads, 0, S.stream>>>(S.nv, S.nnzb, S.diagblk, S.dir, S.valf, S.dscal + S_MAXDIAG); ++S.n_launch;
        }
    else
        {
            k_max_diag<double><<<nb, kThreads, 0, S.stream>>>(S.nv, S.nnzb, S.diagblk, S.dir, S.val, S.dscal + S_MAXDIAG); ++S.n_launch;
        }
    if (sync_flags(S)) return -1.0;
    return S.h_scal[S_MAXDIAG];
}

// x~ = x + h v + h^2 g for free vertices (Alg. 1, inertia target); prescribed: x
__global__ void k_xtilde(int nv, const double *__restrict__ x, const double *__restrict__ v,
                         const uint8_t *__restrict__ dir, double h, double gx, double gy, double gz,
                         double *__restrict__ xt)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nv) return;
    const double g[3] = {gx, gy, gz};
#pragma unroll
    for (int c = 0; c < 3; ++c)
        xt[3 * a + c] = dir[a] ? x[3 * a + c] : x[3 * a + c] + h * v[3 * a + c] + h * h * g[c];
}

void launch_xtilde(Scene &S, double *xtilde)
{
    k_xtilde<<<cdiv(S.nv, kThreads), kThreads, 0, S.stream>>>(S.nv, S.x, S.v, S.dir, S.prm.dt, S.prm.gravity[0],
                                                              S.prm.gravity[1], S.prm.gravity[2], xtilde); ++S.n_launch;
}

// ---------------------------------------------------------------------------
// AL energy L of Eq. total-energy (FP64) with the slacks s_i held fixed:
// threads [0, nv) inertia, [nv, nv + nt) h^2 V_e Psi(F_e),
// [nv + nt, nv + nt + nc) gamma (mu/2 (c - s)^2 - lambda (c - s)).
// Reduced deterministically.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_energy(
    int nv, int nt, int nc, int model, const double *__restrict__ mass, const uint8_t *__restrict__ dir,
    const double *__restrict__ xt, const double *__restrict__ xh, const int4 *__restrict__ tets,
    const double *__restrict__ Bm, const double *__restrict__ vol, const double *__restrict__ emu,
    const double *__restrict__ elam, double h2, const int4 *__restrict__ cv, const double *__restrict__ cd,
    const double *__restrict__ cg, const double *__restrict__ clam, const double *__restrict__ cgam,
    const double *__restrict__ cs, const double *__restrict__ xlin, double mu, double delta, int nf,
    const int4 *__restrict__ fv, const double *__restrict__ fw, const double *__restrict__ fn,
    const double *__restrict__ fk, const double *__restrict__ fx0, double eh, double *partials, unsigned *counter,
    double *out)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (tid < nv) {
        const int a = (int)tid;
        if (!dir[a])
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double d = xh[3 * a + c] - xt[3 * a + c];
                e += 0.5 * mass[a] * d * d;
            }
    } else if (tid < (long long)nv + nt) {
        const int t = (int)(tid - nv);
        const int4 t4 = tets[t];
        const int vid[4] = {t4.x, t4.y, t4.z, t4.w};
        double X[4][3];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) X[k][c] = xh[3 * vid[k] + c];
        const double *B = Bm + 9 * (size_t)t;
        double F[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                F[r][c] = (X[1][r] - X[0][r]) * B[c] + (X[2][r] - X[0][r]) * B[3 + c] + (X[3][r] - X[0][r]) * B[6 + c];
        double I2 = 0.0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) I2 += F[r][c] * F[r][c];
        const double J = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                         F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
        const double m = emu[t], l = elam[t];
        if (model == BF_MODEL_COR) {  // singular values from F^T F, the smallest signed by det F
            double C2[3][3], w[3], Q[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) C2[a][b] = F[0][a] * F[0][b] + F[1][a] * F[1][b] + F[2][a] * F[2][b];
            sym3_eig<double>(C2, w, Q);
            double sv[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) sv[a] = sqrt(w[a] > 0.0 ? w[a] : 0.0);
            const int lo = sv[0] <= sv[1] ? (sv[0] <= sv[2] ? 0 : 2) : (sv[1] <= sv[2] ? 1 : 2);
            if (J < 0.0) sv[lo] = -sv[lo];
            const double tr = sv[0] + sv[1] + sv[2];
            e = h2 * vol[t] * (m * ((sv[0] - 1.0) * (sv[0] - 1.0) + (sv[1] - 1.0) * (sv[1] - 1.0) +
                                    (sv[2] - 1.0) * (sv[2] - 1.0)) + 0.5 * l * (tr - 3.0) * (tr - 3.0));
        } else if (model == BF_MODEL_NH) {  // +inf for inverted or flat elements
            const double L = J > 0.0 ? log(J) : 0.0;
            e = J > 0.0 ? h2 * vol[t] * (0.5 * m * (I2 - 3.0) - m * L + 0.5 * l * L * L) : INFINITY;
        } else {
            e = h2 * vol[t] * (0.5 * m * (I2 - 3.0) - m * (J - 1.0) + 0.5 * l * (J - 1.0) * (J - 1.0));
        }
    } else if (tid < (long long)nv + nt + nc) {
        const int i = (int)(tid - nv - nt);
        const int4 v4 = cv[i];
        const int vid[4] = {v4.x, v4.y, v4.z, v4.w};
        const double *g = cg + 12 * (size_t)i;
        double lin = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) lin += g[3 * k + c] * (xh[3 * vid[k] + c] - xlin[3 * vid[k] + c]);
        const double c = cd[i] + lin - delta;
        const double r = c - cs[i];
        e = cgam[i] * (0.5 * mu * r * r - clam[i] * r);
    } else if (tid < (long long)nv + nt + nc + nf) {  // friction (appendix A)
        e = friction_energy_term((int)(tid - nv - nt - nc), fv, fw, fn, fk, fx0, xh, eh);
    }
    double v[1] = {e}, tot[1];
    if (grid_sum<1>(v, partials, counter, tot)) *out = tot[0];
}

void launch_energy(Scene &S, const double *xtilde, const double *xlin, const double *xhat, double *out)
{
    const long long nthr = (long long)S.nv + S.nt + S.nc + S.nf;
    const int nb = cdiv(nthr, kThreads);
    ScopedTimer tm(S, T_ENERGY);
    k_energy<<<nb, kThreads, 0, S.stream>>>(S.nv, S.nt, S.nc, S.prm.model, S.mass, S.dir, xtilde, xhat, S.tets, S.B,
                                            S.vol, S.emu,
                                            S.elam, S.prm.dt * S.prm.dt, S.cv, S.cd, S.cg, S.clam, S.cgam, S.cs, xlin,
                                            S.mu, S.delta, S.nf, S.fv, S.fw, S.fn, S.fk, S.fx0,
                                            S.prm.dt * S.prm.eps_v, S.partials, S.counter, out);
    ++S.n_launch;
}

// ---------------------------------------------------------------------------
// Inversion bound of MaxStepSize (section 4.1, non-invertible materials).
// One thread per element with a free vertex: along x0 + t (x1 - x0),
// F(t) = F0 + t dF and p(t) = det F(t) - s det F0 is a cubic whose
// coefficients follow from the multilinearity of det in the columns (t^k
// collects the determinants with k columns of dF).  Its first root in
// (0, 1] is bracketed on the pieces between the real roots of p' (p is
// monotone on each) and bisected to adjacent doubles, keeping the end with
// p > 0.  The minimum over elements goes to *tmin (non-negative doubles
// compare like their bit patterns).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double det_cols(const double a[3], const double b[3], const double c[3])
{
    return a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
}

__device__ double cubic_first_root01(double c0, double c1, double c2, double c3)
{
    if (!(c0 > 0.0)) return 0.0;
    auto p = [&](double t) { return ((c3 * t + c2) * t + c1) * t + c0; };
    // real roots of p'(t) = 3 c3 t^2 + 2 c2 t + c1 (stable quadratic formula)
    double r[2] = {2.0, 2.0};
    const double qa = 3.0 * c3, qb = 2.0 * c2;
    if (qa != 0.0) {
        const double disc = qb * qb - 4.0 * qa * c1;
        if (disc >= 0.0) {
            const double q = -0.5 * (qb + copysign(sqrt(disc), qb));
            r[0] = q / qa;
            r[1] = q != 0.0 ? c1 / q : r[0];
        }
    } else if (qb != 0.0) {
        r[0] = -c1 / qb;
    }
    if (r[0] > r[1]) {
        const double t = r[0];
        r[0] = r[1];
        r[1] = t;
    }
    double lo = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double hi = k < 2 ? r[k] : 1.0;
        if (!(hi > lo) || hi > 1.0) continue;
        if (p(hi) > 0.0) {
            lo = hi;
            continue;
        }
        double a = lo, b = hi;
        for (int it = 0; it < 1100; ++it) {  // adjacent doubles within [0, 1] after at most ~1075 halvings
            const double m = 0.5 * (a + b);
            if (!(m > a && m < b)) break;
            if (p(m) > 0.0) a = m;
            else b = m;
        }
        return a;
    }
    return 1.0;
}

__global__ void __launch_bounds__(kThreads) k_inversion_bound(int nt, const int4 *__restrict__ tets,
                                                              const double *__restrict__ Bm,
                                                              const uint8_t *__restrict__ dir,
                                                              const double *__restrict__ x0,
                                                              const double *__restrict__ x1, double s, double *tmin)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double t = 1.0;
    if (e < nt) {
        const int4 t4 = tets[e];
        const int vid[4] = {t4.x, t4.y, t4.z, t4.w};
        if (!(dir[vid[0]] && dir[vid[1]] && dir[vid[2]] && dir[vid[3]])) {
            double D0[3][3], D1[3][3];  // Ds at x0 and Ds(x1) - Ds(x0); row r, column k
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const double a = x0[3 * vid[k + 1] + r] - x0[3 * vid[0] + r];
                    D0[r][k] = a;
                    D1[r][k] = (x1[3 * vid[k + 1] + r] - x1[3 * vid[0] + r]) - a;
                }
            const double *B = Bm + 9 * (size_t)e;
            double f[3][3], g[3][3];  // columns of F0 and dF
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    f[c][r] = D0[r][0] * B[c] + D0[r][1] * B[3 + c] + D0[r][2] * B[6 + c];
                    g[c][r] = D1[r][0] * B[c] + D1[r][1] * B[3 + c] + D1[r][2] * B[6 + c];
                }
            const double J0 = det_cols(f[0], f[1], f[2]);
            const double c1 = det_cols(g[0], f[1], f[2]) + det_cols(f[0], g[1], f[2]) + det_cols(f[0], f[1], g[2]);
            const double c2 = det_cols(f[0], g[1], g[2]) + det_cols(g[0], f[1], g[2]) + det_cols(g[0], g[1], f[2]);
            const double c3 = det_cols(g[0], g[1], g[2]);
            t = cubic_first_root01(J0 - s * J0, c1, c2, c3);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
    if ((threadIdx.x & 31) == 0 && t < 1.0) atomic_min_pos(tmin, t);
}

void launch_inversion_bound(Scene &S, const double *x0, const double *x1, double *tmin)
{
    if (S.nt == 0) return;
    k_inversion_bound<<<cdiv(S.nt, kThreads), kThreads, 0, S.stream>>>(S.nt, S.tets, S.B, S.dir, x0, x1,
                                                                       S.prm.s_ccd, tmin);
    ++S.n_launch;
}

double run_energy(Scene &S, const double *xtilde, const double *xlin, const double *xhat)
{
    launch_energy(S, xtilde, xlin, xhat, S.dscal + S_E0);
    if (sync_flags(S)) return NAN;
    return S.h_scal[S_E0];
}

}  // namespace bf
