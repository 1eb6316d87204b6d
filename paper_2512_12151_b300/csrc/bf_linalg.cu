// Linear algebra of the Newton step (section 5.1): symmetric upper
// block-sparse SpMV with the contact terms applied matrix-free, the 3x3
// block-Jacobi preconditioner, and PCG whose scalar recurrences stay on the
// device (each kernel exits early once a device flag says converged).
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "bf_device.cuh"
#include "bf_internal.cuh"

namespace bf {

template <class A, class B>
using wider_t = typename std::conditional<(sizeof(A) >= sizeof(B)), A, B>::type;

// ---------------------------------------------------------------------------
// y += H x.  Threads [0, nnzb) own one stored 3x3 block each; the row part
// is reduced with a
// segmented warp scan (blocks are sorted by row) and the transposed part of
// off-diagonal blocks is scattered with atomics.  Threads
// [nnzb, nnzb + nc) own one contact pair: y_a += mu gamma g_a (g . x) over
// its free vertices.  With with_dot the kernel also reduces p^T H p =
// sum_blocks w x_r^T A x_c (w = 2 off the diagonal) + sum_pairs mu gamma
// (g . x)^2, and the last block sets alpha = rz / pq for PCG.
// ---------------------------------------------------------------------------
template <class MT, class VI, class VO>
__global__ void __launch_bounds__(kThreads) k_spmv(
    int nnzb, const int *__restrict__ rowid, const int *__restrict__ col, const MT *__restrict__ val,
    int nc, const int4 *__restrict__ cv, const double *__restrict__ cg, const double *__restrict__ cw,
    const unsigned char *__restrict__ cmask, const VI *__restrict__ x, VO *__restrict__ y, int with_dot,
    double *partials, unsigned *counter, double *dscal, int *dflag, const int *done)
{
    if (done && *done) return;
    using CT = wider_t<MT, VI>;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double dot = 0.0;
    int r = -1;
    CT yr0 = 0, yr1 = 0, yr2 = 0;
    if (tid < nnzb) {
        r = rowid[tid];
        const int c = col[tid];
        CT a[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) a[e] = (CT)val[9 * (size_t)tid + e];
        const CT xc0 = (CT)x[3 * c], xc1 = (CT)x[3 * c + 1], xc2 = (CT)x[3 * c + 2];
        yr0 = a[0] * xc0 + a[1] * xc1 + a[2] * xc2;
        yr1 = a[3] * xc0 + a[4] * xc1 + a[5] * xc2;
        yr2 = a[6] * xc0 + a[7] * xc1 + a[8] * xc2;
        if (c != r) {
            const CT xr0 = (CT)x[3 * r], xr1 = (CT)x[3 * r + 1], xr2 = (CT)x[3 * r + 2];
            atomicAdd(y + 3 * c, (VO)(a[0] * xr0 + a[3] * xr1 + a[6] * xr2));
            atomicAdd(y + 3 * c + 1, (VO)(a[1] * xr0 + a[4] * xr1 + a[7] * xr2));
            atomicAdd(y + 3 * c + 2, (VO)(a[2] * xr0 + a[5] * xr1 + a[8] * xr2));
            if (with_dot) dot = 2.0 * (double)(xr0 * yr0 + xr1 * yr1 + xr2 * yr2);
        } else if (with_dot) {
            dot = (double)(xc0 * yr0 + xc1 * yr1 + xc2 * yr2);
        }
    } else if (tid < (long long)nnzb + nc) {
        const int i = (int)(tid - nnzb);
        const int4 v = cv[i];
        const unsigned char m = cmask[i];
        const int vid[4] = {v.x, v.y, v.z, v.w};
        const double *g = cg + 12 * (size_t)i;
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (m >> k & 1)
                s += g[3 * k] * (double)x[3 * vid[k]] + g[3 * k + 1] * (double)x[3 * vid[k] + 1] +
                     g[3 * k + 2] * (double)x[3 * vid[k] + 2];
        const double t = cw[i] * s;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (m >> k & 1) {
                atomicAdd(y + 3 * vid[k], (VO)(t * g[3 * k]));
                atomicAdd(y + 3 * vid[k] + 1, (VO)(t * g[3 * k + 1]));
                atomicAdd(y + 3 * vid[k] + 2, (VO)(t * g[3 * k + 2]));
            }
        if (with_dot) dot = t * s;
    }
    // segmented inclusive scan of the row contributions within the warp
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const CT u0 = __shfl_up_sync(0xffffffffu, yr0, o);
        const CT u1 = __shfl_up_sync(0xffffffffu, yr1, o);
        const CT u2 = __shfl_up_sync(0xffffffffu, yr2, o);
        const int ru = __shfl_up_sync(0xffffffffu, r, o);
        if (lane >= o && ru == r) {
            yr0 += u0;
            yr1 += u1;
            yr2 += u2;
        }
    }
    const int rn = __shfl_down_sync(0xffffffffu, r, 1);
    if (r >= 0 && (lane == 31 || rn != r)) {
        atomicAdd(y + 3 * r, (VO)yr0);
        atomicAdd(y + 3 * r + 1, (VO)yr1);
        atomicAdd(y + 3 * r + 2, (VO)yr2);
    }
    if (with_dot) {
        double v[1] = {dot}, tot[1];
        if (grid_sum<1>(v, partials, counter, tot)) {
            dscal[S_PQ] = tot[0];
            if (with_dot == 2) {  // PCG: alpha = rz / pq
                const double pq = tot[0];
                if (!(pq > 0.0) || !isfinite(pq)) {
                    dflag[F_ERR] |= ERR_PQ;
                    dflag[F_DONE] = 1;
                    dscal[S_ALPHA] = 0.0;
                } else {
                    dscal[S_ALPHA] = dscal[S_RZ] / pq;
                }
            }
        }
    }
}

template <class MT, class VI, class VO>
static void spmv_impl(Scene &S, const MT *val, const VI *x, VO *y, int with_dot, const int *done)
{
    const long long nthr = (long long)S.nnzb + n_terms(S);
    const int nb = cdiv(nthr, kThreads);
    ScopedTimer tm(S, T_SPMV);
    k_spmv<MT, VI, VO><<<nb, kThreads, 0, S.stream>>>(S.nnzb, S.rowid, S.col, val, n_terms(S), S.cv, S.cg,
                                                      S.cw, S.cmask, x, y, with_dot, S.partials,
                                                      S.counter, S.dscal, S.dflag, done); ++S.n_launch;
}

void launch_zero(Scene &S, double *p, size_t n) { cudaMemsetAsync(p, 0, n * sizeof(double), S.stream); }

void launch_spmv(Scene &S, const double *x, double *y, bool with_dot, const int *done)
{
    cudaMemsetAsync(y, 0, 3 * (size_t)S.nv * sizeof(double), S.stream);
    if (S.prm.precision == BF_PREC_MIXED)
        spmv_impl<float, double, double>(S, S.valf, x, y, with_dot ? 1 : 0, done);
    else
        spmv_impl<double, double, double>(S, S.val, x, y, with_dot ? 1 : 0, done);
}

// ---------------------------------------------------------------------------
// Block-Jacobi: P_a = (H_aa)^-1 with H_aa = stored diagonal block plus the
// contact contributions accumulated in cdiag (identity for prescribed
// vertices, whose rows are eliminated).
// ---------------------------------------------------------------------------
template <class MT>
__global__ void k_pinv(int nv, int nnzb, const int *__restrict__ diagblk, const MT *__restrict__ val,
                       const double *__restrict__ cdiag, const uint8_t *__restrict__ dir, MT *__restrict__ pinv,
                       int *dflag)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nv) return;
    double m[9];
    if (dir[a]) {
#pragma unroll
        for (int e = 0; e < 9; ++e) m[e] = (e % 4 == 0) ? 1.0 : 0.0;
    } else {
        const int k = diagblk[a];
#pragma unroll
        for (int e = 0; e < 9; ++e) m[e] = (double)val[9 * (size_t)k + e] + cdiag[9 * (size_t)a + e];
    }
    const double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
    const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) {
        atomicOr(dflag + F_ERR, ERR_NONFINITE);
        for (int e = 0; e < 9; ++e) pinv[9 * (size_t)a + e] = (MT)((e % 4 == 0) ? 1.0 : 0.0);
        return;
    }
    const double id = 1.0 / det;
    double o[9];
    o[0] = c00 * id;
    o[1] = (m[2] * m[7] - m[1] * m[8]) * id;
    o[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    o[3] = c01 * id;
    o[4] = (m[0] * m[8] - m[2] * m[6]) * id;
    o[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    o[6] = c02 * id;
    o[7] = (m[1] * m[6] - m[0] * m[7]) * id;
    o[8] = (m[0] * m[4] - m[1] * m[3]) * id;
#pragma unroll
    for (int e = 0; e < 9; ++e) pinv[9 * (size_t)a + e] = (MT)o[e];
}

void launch_pinv(Scene &S)
{
    const int nb = cdiv(S.nv, kThreads);
    if (S.prm.precision == BF_PREC_MIXED)
        {
            k_pinv<float><<<nb, kThreads, 0, S.stream>>>(S.nv, S.nnzb, S.diagblk, S.valf, S.cdiag,
                                                    S.dir, S.pinvf, S.dflag); ++S.n_launch;
        }
    else
        {
            k_pinv<double><<<nb, kThreads, 0, S.stream>>>(S.nv, S.nnzb, S.diagblk, S.val, S.cdiag,
                                                     S.dir, S.pinv, S.dflag); ++S.n_launch;
        }
}

// ---------------------------------------------------------------------------
// PCG.  x and r are FP64; p, q, z have type VT (FP64, or FP32 in mixed
// precision) and the preconditioner type MT.  All dot products accumulate
// in FP64.  Scalars live in dscal, control in dflag.
// ---------------------------------------------------------------------------
template <class MT, class VT>
__global__ void __launch_bounds__(kThreads) k_pcg_init(
    int nv, const double *__restrict__ b, double *__restrict__ x, double *__restrict__ r,
    VT *__restrict__ z, VT *__restrict__ p, VT *__restrict__ q, const MT *__restrict__ pinv, double *partials,
    unsigned *counter, double *dscal, int *dflag)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (a < nv) {
        double rr[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rr[c] = b[3 * a + c];
            r[3 * a + c] = rr[c];
            x[3 * a + c] = 0.0;
            q[3 * a + c] = (VT)0;
        }
        const MT *P = pinv + 9 * (size_t)a;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double zc = (double)P[3 * c] * rr[0] + (double)P[3 * c + 1] * rr[1] + (double)P[3 * c + 2] * rr[2];
            const VT zv = (VT)zc;
            z[3 * a + c] = zv;
            p[3 * a + c] = zv;
            v[0] += rr[c] * (double)zv;
            v[1] += rr[c] * rr[c];
        }
    }
    double tot[2];
    if (grid_sum<2>(v, partials, counter, tot)) {
        dscal[S_RZ] = tot[0];
        dscal[S_BB] = tot[1];
        dscal[S_RR] = tot[1];
        dflag[F_ITERS] = 0;
        dflag[F_MAXIT] = 0;
        const bool bad = !isfinite(tot[0]) || !isfinite(tot[1]);
        if (bad) dflag[F_ERR] |= ERR_NONFINITE;
        dflag[F_DONE] = (tot[1] == 0.0 || bad) ? 1 : 0;
    }
}

template <class MT, class VT>
__global__ void __launch_bounds__(kThreads) k_pcg_update(
    int nv, double *__restrict__ x, double *__restrict__ r, VT *__restrict__ z, const VT *__restrict__ p,
    const VT *__restrict__ q, const MT *__restrict__ pinv, double tol2, int maxit, double *partials,
    unsigned *counter, double *dscal, int *dflag)
{
    if (dflag[F_DONE]) return;
    const double alpha = dscal[S_ALPHA];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (a < nv) {
        double rr[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            x[3 * a + c] += alpha * (double)p[3 * a + c];
            rr[c] = r[3 * a + c] - alpha * (double)q[3 * a + c];
            r[3 * a + c] = rr[c];
        }
        const MT *P = pinv + 9 * (size_t)a;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double zc = (double)P[3 * c] * rr[0] + (double)P[3 * c + 1] * rr[1] + (double)P[3 * c + 2] * rr[2];
            const VT zv = (VT)zc;
            z[3 * a + c] = zv;
            v[0] += rr[c] * (double)zv;
            v[1] += rr[c] * rr[c];
        }
    }
    double tot[2];
    if (grid_sum<2>(v, partials, counter, tot)) {
        const int it = ++dflag[F_ITERS];
        const double rz = tot[0], rr = tot[1];
        dscal[S_BETA] = rz / dscal[S_RZ];
        dscal[S_RZ] = rz;
        dscal[S_RR] = rr;
        if (!isfinite(rr) || !isfinite(rz)) {
            dflag[F_ERR] |= ERR_NONFINITE;
            dflag[F_DONE] = 1;
        } else if (rr <= tol2 * dscal[S_BB]) {
            dflag[F_DONE] = 1;
        } else if (it >= maxit) {
            dflag[F_DONE] = 1;
            dflag[F_MAXIT] = 1;
        }
    }
}

template <class VT>
__global__ void __launch_bounds__(kThreads) k_pcg_dir(int n, const VT *__restrict__ z, VT *__restrict__ p,
                                                     VT *__restrict__ q, const double *dscal, const int *dflag)
{
    if (dflag[F_DONE]) return;
    const VT beta = (VT)dscal[S_BETA];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        p[i] = z[i] + beta * p[i];
        q[i] = (VT)0;
    }
}

// r = b - H x (FP64 vectors), for residual replacement in mixed precision
__global__ void k_sub(int n, const double *__restrict__ b, const double *__restrict__ hx, double *__restrict__ r)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - hx[i];
}

// restart after residual replacement: z = P r, p = z, q = 0, rz = r.z, rr
template <class MT, class VT>
__global__ void __launch_bounds__(kThreads) k_pcg_restart(
    int nv, const double *__restrict__ r, VT *__restrict__ z, VT *__restrict__ p, VT *__restrict__ q,
    const MT *__restrict__ pinv, double tol2, double *partials, unsigned *counter, double *dscal, int *dflag)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (a < nv) {
        const MT *P = pinv + 9 * (size_t)a;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double zc = (double)P[3 * c] * r[3 * a] + (double)P[3 * c + 1] * r[3 * a + 1] +
                              (double)P[3 * c + 2] * r[3 * a + 2];
            const VT zv = (VT)zc;
            z[3 * a + c] = zv;
            p[3 * a + c] = zv;
            q[3 * a + c] = (VT)0;
            v[0] += r[3 * a + c] * (double)zv;
            v[1] += r[3 * a + c] * r[3 * a + c];
        }
    }
    double tot[2];
    if (grid_sum<2>(v, partials, counter, tot)) {
        dscal[S_RZ] = tot[0];
        dscal[S_RR] = tot[1];
        dflag[F_DONE] = (tot[1] <= tol2 * dscal[S_BB]) ? 1 : 0;
    }
}

template <class MT, class VT>
static int pcg_impl(Scene &S, const MT *val, const MT *pinv, VT *p, VT *q, VT *z, const double *b,
                    double *x, double tol, int maxit, int *iters)
{
    const int nv = S.nv, n = 3 * nv;
    const int nbv = cdiv(nv, kThreads), nbn = cdiv(n, kThreads);
    const double tol2 = tol * tol;
    double *r = S.cg_r;
    cudaMemsetAsync(S.dflag + F_ERR, 0, sizeof(int), S.stream);
    k_pcg_init<MT, VT><<<nbv, kThreads, 0, S.stream>>>(nv, b, x, r, z, p, q, pinv, S.partials, S.counter,
                                                       S.dscal, S.dflag); ++S.n_launch;
    const bool mixed = std::is_same<VT, float>::value;
    int total = 0, chunk = 8, replacements = 0;
    for (;;) {
        for (int j = 0; j < chunk; ++j) {
            spmv_impl<MT, VT, VT>(S, val, p, q, 2, S.dflag + F_DONE);
            {
                ScopedTimer tm(S, T_PCG_UPDATE);
                k_pcg_update<MT, VT><<<nbv, kThreads, 0, S.stream>>>(nv, x, r, z, p, q, pinv, tol2, maxit,
                                                                     S.partials, S.counter, S.dscal, S.dflag); ++S.n_launch;
            }
            {
                ScopedTimer tm(S, T_PCG_DIR);
                k_pcg_dir<VT><<<nbn, kThreads, 0, S.stream>>>(n, z, p, q, S.dscal, S.dflag); ++S.n_launch;
            }
        }
        int st = sync_flags(S);
        if (st) return st;
        total = S.h_flag[F_ITERS];
        if (S.h_flag[F_ERR] & (ERR_NONFINITE | ERR_PQ)) {
            if (iters) *iters = total;
            if (S.h_flag[F_ERR] & ERR_PQ && S.h_scal[S_RR] <= tol2 * S.h_scal[S_BB]) return BF_OK;
            return (S.h_flag[F_ERR] & ERR_NONFINITE) ? BF_E_NONFINITE : BF_OK;
        }
        if (S.h_flag[F_DONE]) {
            if (mixed && !S.h_flag[F_MAXIT] && replacements < 4) {
                // residual replacement: recompute r = b - H x in FP64 vectors
                // with the FP32 matrix; continue from it if it is not small
                cudaMemsetAsync(S.cg_q, 0, n * sizeof(double), S.stream);
                spmv_impl<MT, double, double>(S, val, x, S.cg_q, 0, nullptr);
                k_sub<<<nbn, kThreads, 0, S.stream>>>(n, b, S.cg_q, r); ++S.n_launch;
                k_pcg_restart<MT, VT><<<nbv, kThreads, 0, S.stream>>>(nv, r, z, p, q, pinv, tol2, S.partials,
                                                                      S.counter, S.dscal, S.dflag); ++S.n_launch;
                ++replacements;
                st = sync_flags(S);
                if (st) return st;
                if (!S.h_flag[F_DONE]) continue;
            }
            break;
        }
        if (chunk < 32) chunk *= 2;
    }
    if (iters) *iters = total;
    return S.h_flag[F_MAXIT] ? BF_E_CG_MAXIT : BF_OK;
}

int run_pcg(Scene &S, const double *b, double *x, double tol, int maxit, int *iters)
{
    if (S.pcg_mode == 1) return run_pcg_persistent(S, b, x, tol, maxit, iters);
    if (S.prm.precision == BF_PREC_MIXED)
        return pcg_impl<float, float>(S, S.valf, S.pinvf, S.cg_pf, S.cg_qf, S.cg_zf, b, x, tol, maxit, iters);
    return pcg_impl<double, double>(S, S.val, S.pinv, S.cg_p, S.cg_q, S.cg_z, b, x, tol, maxit, iters);
}

// ---------------------------------------------------------------------------
// small vector kernels
// ---------------------------------------------------------------------------
__global__ void k_axpy_to(int n, double *__restrict__ out, const double *__restrict__ a, double r,
                          const double *__restrict__ p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + r * p[i];
}
void launch_axpy_to(Scene &S, double *out, const double *a, double r, const double *p, int n)
{
    k_axpy_to<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, out, a, r, p); ++S.n_launch;
}

__global__ void k_axpy_scaled(int n, double *__restrict__ out, const double *__restrict__ a, double r,
                              const double *__restrict__ p, const double *__restrict__ scale)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + r * (*scale * p[i]);
}
void launch_axpy_scaled(Scene &S, double *out, const double *a, double r, const double *p, const double *scale,
                        int n)
{
    k_axpy_scaled<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, out, a, r, p, scale); ++S.n_launch;
}

// Eq. CCD-clamp: x^[k+1] = (1 - alpha) x^[k] + alpha xhat^[k+1]
__global__ void k_blend(int n, double *__restrict__ xk, const double *__restrict__ xh, double alpha)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xk[i] = (1.0 - alpha) * xk[i] + alpha * xh[i];
}
void launch_blend(Scene &S, double *xk, const double *xh, double alpha, int n)
{
    k_blend<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, xk, xh, alpha); ++S.n_launch;
}

// Alg. 1, end of the time step: v^{t+1} = (x^[k] - x^t) / h, x^{t+1} = x^[k]
__global__ void k_velocity(int n, const double *__restrict__ xk, const double *__restrict__ xt, double h,
                           double *__restrict__ x, double *__restrict__ v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        v[i] = (xk[i] - xt[i]) / h;
        x[i] = xk[i];
    }
}
void launch_velocity(Scene &S)
{
    const int n = 3 * S.nv;
    k_velocity<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, S.xk, S.xt, S.prm.dt, S.x, S.v); ++S.n_launch;
}

}  // namespace bf
