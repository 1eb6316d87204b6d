// Augmented-Lagrangian contact terms (section 4.2, Alg. 2).  For each pair
// i of the active set, linearised at the intersection-free x:
//   c_i(xhat) = d_i(x) + grad d_i(x)^T (xhat - x) - delta,
//   s_i = max(0, c_i - lambda_i / mu),
//   G += mu gamma_i (c_i - lambda_i / mu - s_i) grad d_i(x),
//   H += mu gamma_i grad d_i(x) grad d_i(x)^T.
// The rank-1 Hessian terms are not assembled into the block-sparse matrix:
// the SpMV applies them per pair, and only their diagonal 3x3 blocks are
// accumulated (cdiag) for the block-Jacobi preconditioner.
#include <cuda_runtime.h>

#include "bf_device.cuh"
#include "bf_internal.cuh"

namespace bf {

__device__ __forceinline__ double lin_constraint(int i, const int4 v4, const double *__restrict__ cd,
                                                 const double *__restrict__ cg, const double *__restrict__ xl,
                                                 const double *__restrict__ xh, double delta)
{
    const int vid[4] = {v4.x, v4.y, v4.z, v4.w};
    const double *g = cg + 12 * (size_t)i;
    double lin = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) lin += g[3 * k + c] * (xh[3 * vid[k] + c] - xl[3 * vid[k] + c]);
    return cd[i] + lin - delta;
}

__global__ void k_contact_assemble(int nc, const int4 *__restrict__ cv, const unsigned char *__restrict__ cmask,
                                   const double *__restrict__ cd, const double *__restrict__ cg,
                                   const double *__restrict__ clam, const double *__restrict__ cgam,
                                   const double *__restrict__ xl, const double *__restrict__ xh, double mu,
                                   double delta, double *__restrict__ cs, double *__restrict__ cw,
                                   double *__restrict__ grad, double *__restrict__ cdiag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int4 v4 = cv[i];
    const int vid[4] = {v4.x, v4.y, v4.z, v4.w};
    const double c = lin_constraint(i, v4, cd, cg, xl, xh, delta);
    const double lm = clam[i] / mu;
    double s = c - lm;
    s = s > 0.0 ? s : 0.0;
    cs[i] = s;
    const double w = mu * cgam[i];
    cw[i] = w;
    const double coef = w * (c - lm - s);
    const unsigned char m = cmask[i];
    const double *g = cg + 12 * (size_t)i;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!(m >> k & 1)) continue;
        const double g0 = g[3 * k], g1 = g[3 * k + 1], g2 = g[3 * k + 2];
        if (coef != 0.0) {
            atomicAdd(grad + 3 * vid[k], coef * g0);
            atomicAdd(grad + 3 * vid[k] + 1, coef * g1);
            atomicAdd(grad + 3 * vid[k] + 2, coef * g2);
        }
        double *D = cdiag + 9 * (size_t)vid[k];
        atomicAdd(D + 0, w * g0 * g0);
        atomicAdd(D + 1, w * g0 * g1);
        atomicAdd(D + 2, w * g0 * g2);
        atomicAdd(D + 3, w * g1 * g0);
        atomicAdd(D + 4, w * g1 * g1);
        atomicAdd(D + 5, w * g1 * g2);
        atomicAdd(D + 6, w * g2 * g0);
        atomicAdd(D + 7, w * g2 * g1);
        atomicAdd(D + 8, w * g2 * g2);
    }
}

void launch_contact_assemble(Scene &S, const double *xlin, const double *xhat)
{
    if (S.nc == 0) return;
    ScopedTimer tm(S, T_CONTACT);
    k_contact_assemble<<<cdiv(S.nc, kThreads), kThreads, 0, S.stream>>>(S.nc, S.cv, S.cmask, S.cd, S.cg, S.clam,
                                                                       S.cgam, xlin, xhat, S.mu, S.delta, S.cs,
                                                                       S.cw, S.grad, S.cdiag); ++S.n_launch;
}

// Alg. 2, multiplier and decay update: with s_i = max(0, c_i - lambda_i/mu), s_i = 0 gives
// lambda_i <- lambda_i - mu c_i and gamma_i <- 1, otherwise lambda_i <- 0
// and gamma_i <- Gamma gamma_i.
__global__ void k_multiplier_update(int nc, const int4 *__restrict__ cv, const double *__restrict__ cd,
                                    const double *__restrict__ cg, double *__restrict__ clam,
                                    double *__restrict__ cgam, const double *__restrict__ xl,
                                    const double *__restrict__ xh, double mu, double delta, double Gamma)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double c = lin_constraint(i, cv[i], cd, cg, xl, xh, delta);
    const double lam = clam[i];
    if (c - lam / mu <= 0.0) {
        clam[i] = lam - mu * c;
        cgam[i] = 1.0;
    } else {
        clam[i] = 0.0;
        cgam[i] = Gamma * cgam[i];
    }
}

void launch_multiplier_update(Scene &S, const double *xlin, const double *xhat)
{
    if (S.nc == 0) return;
    {
        k_multiplier_update<<<cdiv(S.nc, kThreads), kThreads, 0, S.stream>>>(S.nc, S.cv, S.cd, S.cg, S.clam, S.cgam,
                                                                        xlin, xhat, S.mu, S.delta,
                                                                        S.prm.gamma_decay); ++S.n_launch;
    }
}

}  // namespace bf
