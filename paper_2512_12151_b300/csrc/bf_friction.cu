// Semi-implicit friction (appendix A; the friction model of IPC, Li et al.
// 2020): U_f = sum_i mu_f F_i f0(|u_i|; h eps_v) over the pairs active at
// the start of the time step, with F_i and the tangent operator fixed
// there.  In the incremental potential the term is
//   k_i f0(|u_i|),  k_i = mu_f mu max(0, lambda_i / mu - c_i(x^t))
// (the h^-2 of F_i cancels the h^2 of the potential; mu, delta and lambda
// as the previous step left them), where u_i is the displacement since x^t
// of the pair's closest points, with their weights w at x^t, projected on
// the plane normal to the pair's unit normal n at x^t.  f0(y) = y from
// y = h eps_v on, and -y^3 / (3 eh^2) + y^2 / eh + eh / 3 below it (C^2).
// The Hessian in u, f0'' t t^T + f0'/y (I - t t^T) with t = u / |u|, is
// PSD as it stands, so each pair adds two weighted rank-one terms,
// f0'' k (w (x) t)(w (x) t)^T and f0'/y k (w (x) b)(w (x) b)^T with
// b = n x t, which go into the contact-term arrays after the
// augmented-Lagrangian pairs: the PCG applies both kinds alike.
#include <cuda_runtime.h>

#include "bf_device.cuh"
#include "bf_friction.cuh"
#include "bf_internal.cuh"

namespace bf {

// From the linearisation at x^t (cd, cg = w_k n per vertex): n is the first
// vertex's block for a point-triangle pair (weight 1) and the sum of the
// first edge's two blocks for an edge pair (weights summing to 1); w_k =
// cg_k . n.  Pairs with k > 0 are appended (any order).
__global__ void k_friction_setup(int nc, const int *__restrict__ ctype, const int4 *__restrict__ cv,
                                 const unsigned char *__restrict__ cmask, const double *__restrict__ cd,
                                 const double *__restrict__ cg, const double *__restrict__ clam, double mu,
                                 double delta, double mu_f, int4 *__restrict__ fv, double *__restrict__ fw,
                                 double *__restrict__ fn, double *__restrict__ fk, unsigned char *__restrict__ fmask,
                                 int *count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double d = cd[i], F = clam[i] / mu - (d - delta);
    if (!(d > 0.0) || !(F > 0.0)) return;
    const double *g = cg + 12 * (size_t)i;
    double n[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) n[c] = ctype[i] == PT ? g[c] : g[c] + g[3 + c];
    const int j = atomicAdd(count, 1);
    fv[j] = cv[i];
    fmask[j] = cmask[i];
    fk[j] = mu_f * mu * F;
#pragma unroll
    for (int c = 0; c < 3; ++c) fn[3 * j + c] = n[c];
#pragma unroll
    for (int k = 0; k < 4; ++k) fw[4 * j + k] = g[3 * k] * n[0] + g[3 * k + 1] * n[1] + g[3 * k + 2] * n[2];
}

// per Newton iteration: gradient, preconditioner blocks, and the two
// rank-one terms of pair j at contact-term slots base + 2j, base + 2j + 1
__global__ void k_friction_assemble(int nf, const int4 *__restrict__ fv, const double *__restrict__ fw,
                                    const double *__restrict__ fn, const double *__restrict__ fk,
                                    const unsigned char *__restrict__ fmask, const double *__restrict__ x0,
                                    const double *__restrict__ xh, double eh, double *__restrict__ grad,
                                    double *__restrict__ cdiag, int base, int4 *__restrict__ cv,
                                    double *__restrict__ cg, double *__restrict__ cw, unsigned char *__restrict__ cmask)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    double ut[3], f1y, f2;
    const double *n;
    int vid[4];
    const double y = fr_slip(j, fv, fw, fn, x0, xh, ut, &n, vid);
    fr_f0(y, eh, &f1y, &f2);
    const double k = fk[j];
    const double *w = fw + 4 * (size_t)j;
    const unsigned char m = fmask[j];
    // slip direction t (any unit vector of the tangent plane when y = 0) and b = n x t
    double t[3];
    if (y > 0.0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) t[c] = ut[c] / y;
    } else {
        const int a = fabs(n[0]) <= fabs(n[1]) ? (fabs(n[0]) <= fabs(n[2]) ? 0 : 2) : (fabs(n[1]) <= fabs(n[2]) ? 1 : 2);
        double e[3] = {0.0, 0.0, 0.0};
        e[a] = 1.0;
        t[0] = n[1] * e[2] - n[2] * e[1];
        t[1] = n[2] * e[0] - n[0] * e[2];
        t[2] = n[0] * e[1] - n[1] * e[0];
        const double l = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) t[c] /= l;
    }
    const double b[3] = {n[1] * t[2] - n[2] * t[1], n[2] * t[0] - n[0] * t[2], n[0] * t[1] - n[1] * t[0]};
    const double s1 = y > 0.0 ? k * f2 : k * f1y, s2 = k * f1y;
    const double gcoef = k * f1y;
    const int p = base + 2 * j;
    cv[p] = cv[p + 1] = fv[j];
    cmask[p] = cmask[p + 1] = m;
    cw[p] = s1;
    cw[p + 1] = s2;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cg[12 * (size_t)p + 3 * q + c] = w[q] * t[c];
            cg[12 * (size_t)(p + 1) + 3 * q + c] = w[q] * b[c];
        }
        if (!(m >> q & 1)) continue;
        double *G = grad + 3 * vid[q];
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(G + c, gcoef * w[q] * ut[c]);
        double *D = cdiag + 9 * (size_t)vid[q];
        const double w2 = w[q] * w[q];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(D + 3 * r + c, w2 * (s1 * t[r] * t[c] + s2 * b[r] * b[c]));
    }
}

int friction_setup(Scene &S)
{
    S.nf = 0;
    if (!(S.prm.mu_f > 0.0) || !(S.mu > 0.0) || S.nc == 0) return BF_OK;
    if (S.fcap < S.nc) {
        void *old[] = {S.fv, S.fw, S.fn, S.fk, S.fmask};
        for (void *p : old)
            if (p) dev_free(S, p);
        S.fcap = S.nc + S.nc / 2;
        S.fv = (int4 *)dev_alloc(S, (size_t)S.fcap * sizeof(int4));
        S.fw = (double *)dev_alloc(S, 4 * (size_t)S.fcap * sizeof(double));
        S.fn = (double *)dev_alloc(S, 3 * (size_t)S.fcap * sizeof(double));
        S.fk = (double *)dev_alloc(S, (size_t)S.fcap * sizeof(double));
        S.fmask = (unsigned char *)dev_alloc(S, (size_t)S.fcap);
        if (!S.fv || !S.fw || !S.fn || !S.fk || !S.fmask) {
            S.fcap = 0;
            return BF_E_OOM;
        }
    }
    if (!S.fx0) {
        S.fx0 = (double *)dev_alloc(S, 3 * (size_t)S.nv * sizeof(double));
        if (!S.fx0) return BF_E_OOM;
    }
    cudaMemcpyAsync(S.fx0, S.x, 3 * (size_t)S.nv * sizeof(double), cudaMemcpyDeviceToDevice, S.stream);
    launch_linearize(S, S.x);  // d and grad d at x^t
    cudaMemsetAsync(S.dflag + F_NFRIC, 0, sizeof(int), S.stream);
    k_friction_setup<<<cdiv(S.nc, kThreads), kThreads, 0, S.stream>>>(S.nc, S.ctype, S.cv, S.cmask, S.cd, S.cg,
                                                                      S.clam, S.mu, S.delta, S.prm.mu_f, S.fv, S.fw,
                                                                      S.fn, S.fk, S.fmask, S.dflag + F_NFRIC);
    ++S.n_launch;
    const int st = sync_flags(S);
    if (st) return st;
    S.nf = S.h_flag[F_NFRIC];
    return BF_OK;
}

int launch_friction_assemble(Scene &S, const double *xhat)
{
    if (S.nf == 0) return BF_OK;
    const int st = active_reserve(S, S.nc + 2 * S.nf);  // room for the rank-one terms after the pairs
    if (st) return st;
    ScopedTimer tm(S, T_CONTACT);
    k_friction_assemble<<<cdiv(S.nf, kThreads), kThreads, 0, S.stream>>>(
        S.nf, S.fv, S.fw, S.fn, S.fk, S.fmask, S.fx0, xhat, S.prm.dt * S.prm.eps_v, S.grad, S.cdiag, S.nc, S.cv,
        S.cg, S.cw, S.cmask);
    ++S.n_launch;
    return BF_OK;
}

}  // namespace bf
