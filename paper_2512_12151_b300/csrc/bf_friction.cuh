// Device helpers of the semi-implicit friction (appendix A), shared by the
// friction kernels and the energy kernel.
#pragma once
#include <cuda_runtime.h>

namespace bf {

// f0(y; eh) and f0'(y) / y (finite at 0) and f0''(y)
__device__ __forceinline__ double fr_f0(double y, double eh, double *f1y, double *f2)
{
    if (y >= eh) {
        *f1y = 1.0 / y;
        *f2 = 0.0;
        return y;
    }
    const double s = y / eh;
    *f1y = (2.0 - s) / eh;
    *f2 = 2.0 * (1.0 - s) / eh;
    return eh * (s * s * (1.0 - s / 3.0) + 1.0 / 3.0);
}

// tangential relative displacement of pair j at xh
__device__ __forceinline__ double fr_slip(int j, const int4 *__restrict__ fv, const double *__restrict__ fw,
                                          const double *__restrict__ fn, const double *__restrict__ x0,
                                          const double *__restrict__ xh, double *ut, const double **nout,
                                          int *vid)
{
    const int4 v = fv[j];
    vid[0] = v.x; vid[1] = v.y; vid[2] = v.z; vid[3] = v.w;
    const double *w = fw + 4 * (size_t)j, *n = fn + 3 * (size_t)j;
    double D[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) D[c] += w[k] * (xh[3 * vid[k] + c] - x0[3 * vid[k] + c]);
    const double dn = D[0] * n[0] + D[1] * n[1] + D[2] * n[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) ut[c] = D[c] - dn * n[c];
    *nout = n;
    return sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
}

__device__ __forceinline__ double friction_energy_term(int j, const int4 *__restrict__ fv, const double *__restrict__ fw,
                                       const double *__restrict__ fn, const double *__restrict__ fk,
                                       const double *__restrict__ x0, const double *__restrict__ xh, double eh)
{
    double ut[3], f1y, f2;
    const double *n;
    int vid[4];
    const double y = fr_slip(j, fv, fw, fn, x0, xh, ut, &n, vid);
    return fk[j] * fr_f0(y, eh, &f1y, &f2);
}

}  // namespace bf
