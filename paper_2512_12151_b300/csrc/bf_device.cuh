// Device helpers: warp / block reductions and a deterministic grid-wide
// reduction (each block writes its partial, the last block to finish sums
// the partials in block order, so results do not depend on scheduling).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bf {

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums K values over the block; the result is valid in thread 0.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K])
{
    __shared__ double sh[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh[k][wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nw ? sh[k][lane] : 0.0;
            v[k] = warp_sum(t);
        }
    }
    __syncthreads();
}

// Grid reduction of K values.  partials must hold K * gridDim.x doubles and
// counter must be zero on entry (it is reset by the last block).  Returns
// true in thread 0 of the last block, with tot[k] = the grid sums.
template <int K>
__device__ __forceinline__ bool grid_sum(double (&v)[K], double *partials, unsigned *counter,
                                         double (&tot)[K])
{
    __shared__ bool last;
    block_sum<K>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) partials[(size_t)k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        s[k] = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
            s[k] += __ldcg(partials + (size_t)k * gridDim.x + i);
    }
    block_sum<K>(s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] = s[k];
        *counter = 0u;
    }
    return threadIdx.x == 0;
}

__device__ __forceinline__ void atomic_max_pos(double *addr, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_pos(double *addr, double v)
{
    atomicMin((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace bf
