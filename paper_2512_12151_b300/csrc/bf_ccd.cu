// Collision detection and the active set (section 5.1, Alg. 3).
//
// This translation unit is compiled with -fmad=false: the unsigned
// distances and the additive CCD below evaluate their FP64 arithmetic in a
// fixed order (products rounded, sums left to right, IEEE division and
// square root), so that a time of impact depends only on its 24 input
// coordinates.
//
// Broad phase: a linear BVH (Karras 2012: Morton codes, radix sort, radix
// tree, bottom-up refit) over the swept boxes of the surface triangles and
// of the surface edges, rebuilt for every CCD pass; vertex boxes query the
// triangle tree, edge boxes the edge tree.  A pair is a candidate when the
// closed swept boxes overlap (box coordinates are exact min/max values), it
// shares no vertex, and not all four of its vertices are prescribed.
// Narrow phase: additive CCD (the ACCD of section 5.1) with thickness 0 and
// target gap s * d(x0).
#include <cub/cub.cuh>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "bf_device.cuh"
#include "bf_internal.cuh"

namespace bf {

// ---------------------------------------------------------------------------
// distances (fixed evaluation order)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dot3(const double *a, const double *b)
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

// squared distance from p to the closed segment [a, b]; *t = parameter
__device__ double seg_d2(const double *p, const double *a, const double *b, double *tout)
{
    double e[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    const double ee = dot3(e, e);
    double t = 0.0;
    if (ee > 0.0) t = dot3(ap, e) / ee;
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    double r[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = p[k] - (a[k] + t * e[k]);
    *tout = t;
    return dot3(r, r);
}

// squared distance from p to the closed triangle (a, b, c); w = weights of
// the closest point
__device__ double tri_d2(const double *p, const double *a, const double *b, const double *c, double *w)
{
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double ac[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    const double d00 = dot3(ab, ab), d01 = dot3(ab, ac), d11 = dot3(ac, ac);
    const double d20 = dot3(ap, ab), d21 = dot3(ap, ac);
    const double den = d00 * d11 - d01 * d01;
    if (den > 0.0) {
        const double v = (d11 * d20 - d01 * d21) / den;
        const double ww = (d00 * d21 - d01 * d20) / den;
        const double u = (1.0 - v) - ww;
        if (u >= 0.0 && v >= 0.0 && ww >= 0.0) {
            double r[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) r[k] = p[k] - ((a[k] + v * ab[k]) + ww * ac[k]);
            w[0] = u;
            w[1] = v;
            w[2] = ww;
            return dot3(r, r);
        }
    }
    double t;
    double best = seg_d2(p, a, b, &t);
    w[0] = 1.0 - t; w[1] = t; w[2] = 0.0;
    double d = seg_d2(p, b, c, &t);
    if (d < best) { best = d; w[0] = 0.0; w[1] = 1.0 - t; w[2] = t; }
    d = seg_d2(p, c, a, &t);
    if (d < best) { best = d; w[0] = t; w[1] = 0.0; w[2] = 1.0 - t; }
    return best;
}

// squared distance between closed segments [a0, a1] and [b0, b1]
__device__ double edge_d2(const double *a0, const double *a1, const double *b0, const double *b1, double *wa,
                          double *wb)
{
    double ea[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
    double eb[3] = {b1[0] - b0[0], b1[1] - b0[1], b1[2] - b0[2]};
    double w[3] = {a0[0] - b0[0], a0[1] - b0[1], a0[2] - b0[2]};
    const double A = dot3(ea, ea), B = dot3(ea, eb), C = dot3(eb, eb), D = dot3(ea, w), E = dot3(eb, w);
    const double den = A * C - B * B;
    double best = INFINITY;
    if (den > 0.0) {
        const double s = (B * E - C * D) / den;
        const double t = (A * E - B * D) / den;
        if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
            double r[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) r[k] = (a0[k] + s * ea[k]) - (b0[k] + t * eb[k]);
            best = dot3(r, r);
            wa[0] = 1.0 - s; wa[1] = s; wb[0] = 1.0 - t; wb[1] = t;
        }
    }
    double t, d;
    d = seg_d2(a0, b0, b1, &t);
    if (d < best) { best = d; wa[0] = 1.0; wa[1] = 0.0; wb[0] = 1.0 - t; wb[1] = t; }
    d = seg_d2(a1, b0, b1, &t);
    if (d < best) { best = d; wa[0] = 0.0; wa[1] = 1.0; wb[0] = 1.0 - t; wb[1] = t; }
    d = seg_d2(b0, a0, a1, &t);
    if (d < best) { best = d; wb[0] = 1.0; wb[1] = 0.0; wa[0] = 1.0 - t; wa[1] = t; }
    d = seg_d2(b1, a0, a1, &t);
    if (d < best) { best = d; wb[0] = 0.0; wb[1] = 1.0; wa[0] = 1.0 - t; wa[1] = t; }
    return best;
}

__device__ __forceinline__ double pair_d2(int type, const double *x)
{
    double w[3], wb[2];
    if (type == PT) return tri_d2(x, x + 3, x + 6, x + 9, w);
    return edge_d2(x, x + 3, x + 6, x + 9, w, wb);
}

// Additive CCD along x0 -> x1 (positions of the pair's 4 vertices).
// Returns true with *toi on a hit at t <= tmax.
__device__ bool accd(int type, const double *x0, const double *x1, double s, double tmax, int max_iter,
                     double *toi)
{
    double p[12], x[12], n[4];
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k] = x1[k] - x0[k];
    double pbar[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) pbar[c] = (((p[c] + p[3 + c]) + p[6 + c]) + p[9 + c]) * 0.25;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) p[3 * k + c] = p[3 * k + c] - pbar[c];
#pragma unroll
    for (int k = 0; k < 4; ++k) n[k] = sqrt(dot3(p + 3 * k, p + 3 * k));
    const double lp = type == PT ? n[0] + fmax(fmax(n[1], n[2]), n[3]) : fmax(n[0], n[1]) + fmax(n[2], n[3]);
    if (lp == 0.0) return false;
#pragma unroll
    for (int k = 0; k < 12; ++k) x[k] = x0[k];
    double d = sqrt(pair_d2(type, x));
    const double g = s * d;
    double t = 0.0;
    double tl = ((1.0 - s) * d) / lp;
    for (int it = 0; it < max_iter; ++it) {
#pragma unroll
        for (int k = 0; k < 12; ++k) x[k] = x[k] + tl * p[k];
        d = sqrt(pair_d2(type, x));
        if (t > 0.0 && d < g) {
            *toi = t;
            return true;
        }
        t = t + tl;
        if (t > tmax) return false;
        tl = (0.9 * d) / lp;
    }
    *toi = t;
    return true;
}

__device__ __forceinline__ int4 pair_vertices(int type, int a, int b, const int *__restrict__ st,
                                              const int *__restrict__ se)
{
    if (type == PT) return make_int4(a, st[3 * b], st[3 * b + 1], st[3 * b + 2]);
    return make_int4(se[2 * a], se[2 * a + 1], se[2 * b], se[2 * b + 1]);
}

__device__ __forceinline__ void gather12(const double *__restrict__ x, int4 v, double *o)
{
    const int id[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) o[3 * k + c] = x[3 * id[k] + c];
}

// ---------------------------------------------------------------------------
// Alg. 2, linearisation: d_i(x), grad d_i(x) (envelope theorem at the closest
// points), and the free-vertex mask of each pair
// ---------------------------------------------------------------------------
__global__ void k_linearize(int nc, const int *__restrict__ ctype, const int4 *__restrict__ cv,
                            const double *__restrict__ x, const uint8_t *__restrict__ dir, double *__restrict__ cd,
                            double *__restrict__ cg, unsigned char *__restrict__ cmask, double *dout, double *gout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int4 v = cv[i];
    double X[12], cw[4];
    gather12(x, v, X);
    double d2;
    if (ctype[i] == PT) {
        double w[3];
        d2 = tri_d2(X, X + 3, X + 6, X + 9, w);
        cw[0] = 1.0; cw[1] = -w[0]; cw[2] = -w[1]; cw[3] = -w[2];
    } else {
        double wa[2], wb[2];
        d2 = edge_d2(X, X + 3, X + 6, X + 9, wa, wb);
        cw[0] = wa[0]; cw[1] = wa[1]; cw[2] = -wb[0]; cw[3] = -wb[1];
    }
    const double d = sqrt(d2);
    double diff[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) diff[c] += cw[k] * X[3 * k + c];
    cd[i] = d;
    if (dout) dout[i] = d;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double gv = d > 0.0 ? cw[k] * diff[c] / d : 0.0;
            cg[12 * (size_t)i + 3 * k + c] = gv;
            if (gout) gout[12 * (size_t)i + 3 * k + c] = gv;
        }
    const int id[4] = {v.x, v.y, v.z, v.w};
    unsigned char m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (!dir[id[k]]) m |= (unsigned char)(1u << k);
    cmask[i] = m;
}

void launch_linearize(Scene &S, const double *xlin)
{
    if (S.nc == 0) return;
    {
        k_linearize<<<cdiv(S.nc, kThreads), kThreads, 0, S.stream>>>(S.nc, S.ctype, S.cv, xlin, S.dir, S.cd, S.cg,
                                                                 S.cmask, nullptr, nullptr); ++S.n_launch;
    }
}

void launch_linearize_out(Scene &S, const double *xlin, double *dout, double *gout)
{
    if (S.nc == 0) return;
    {
        k_linearize<<<cdiv(S.nc, kThreads), kThreads, 0, S.stream>>>(S.nc, S.ctype, S.cv, xlin, S.dir, S.cd, S.cg,
                                                                 S.cmask, dout, gout); ++S.n_launch;
    }
}

// ---------------------------------------------------------------------------
// LBVH
// ---------------------------------------------------------------------------
// box of a primitive over its vertices at x0 and x1 (and x2 unless null)
template <int NV>
__global__ void k_prim_boxes(int n, const int *__restrict__ ids, const double *__restrict__ x0,
                             const double *__restrict__ x1, const double *__restrict__ x2, double *__restrict__ lo,
                             double *__restrict__ hi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int v = ids[NV * (size_t)i + k];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double a = x0[3 * v + c], b = x1[3 * v + c];
            l[c] = fmin(l[c], fmin(a, b));
            h[c] = fmax(h[c], fmax(a, b));
            if (x2) {
                const double e = x2[3 * v + c];
                l[c] = fmin(l[c], e);
                h[c] = fmax(h[c], e);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[3 * (size_t)i + c] = l[c];
        hi[3 * (size_t)i + c] = h[c];
    }
}

__device__ __forceinline__ int f2ord(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_centroid_bounds(int n, const double *__restrict__ lo, const double *__restrict__ hi, int *bnd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (i < n)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float m = (float)(0.5 * (lo[3 * (size_t)i + c] + hi[3 * (size_t)i + c]));
            mn[c] = m;
            mx[c] = m;
        }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicMin(bnd + c, f2ord(mn[c]));
            atomicMax(bnd + 3 + c, f2ord(mx[c]));
        }
}

__device__ __forceinline__ unsigned expand10(unsigned v)
{
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__global__ void k_morton(int n, const double *__restrict__ lo, const double *__restrict__ hi, const int *bnd,
                         unsigned *__restrict__ code, int *__restrict__ prim)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float b0 = ord2f(bnd[c]), b1 = ord2f(bnd[3 + c]);
        const float m = (float)(0.5 * (lo[3 * (size_t)i + c] + hi[3 * (size_t)i + c]));
        float u = b1 > b0 ? (m - b0) / (b1 - b0) : 0.5f;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        q[c] = min((unsigned)(u * 1024.0f), 1023u);
    }
    code[i] = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
    prim[i] = i;
}

// Implicit complete binary tree over the Morton-sorted leaves, padded to
// N = 2^L leaves: heap node h has children 2h and 2h + 1, leaf k is node
// N + k, the root is node 1.  Every node stores its box in FP32 rounded
// outwards (float4 pair: lo.xyz, hi.xyz), so an internal box contains the
// exact FP64 boxes below it; padding leaves are empty boxes.  Leaf boxes are
// also kept exactly (FP64, in leaf order) for the final test.
__global__ void k_leaves(int n, int N, const int *__restrict__ prim, const double *__restrict__ plo,
                         const double *__restrict__ phi, double *__restrict__ llo, double *__restrict__ lhi,
                         float4 *__restrict__ node)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    float l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (k < n) {
        const int p = prim[k];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double a = plo[3 * (size_t)p + c], b = phi[3 * (size_t)p + c];
            llo[3 * (size_t)k + c] = a;
            lhi[3 * (size_t)k + c] = b;
            l[c] = __double2float_rd(a);
            h[c] = __double2float_ru(b);
        }
    }
    node[2 * (size_t)(N + k)] = make_float4(l[0], l[1], l[2], 0.f);
    node[2 * (size_t)(N + k) + 1] = make_float4(h[0], h[1], h[2], 0.f);
}

constexpr int kLevelChunk = 512;  // nodes of one level combined by one block

// Combines `levels` levels upwards: block b takes nodes [cnt + b M, cnt +
// (b + 1) M) of the level whose nodes are [cnt, 2 cnt) (M = chunk) and
// writes their ancestors up to M / 2^levels nodes per block.
__global__ void __launch_bounds__(256) k_levels(int cnt, int M, int levels, float4 *__restrict__ node)
{
    __shared__ float bl[3][kLevelChunk], bh[3][kLevelChunk];
    const int first = cnt + blockIdx.x * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const float4 a = node[2 * (size_t)(first + i)], b = node[2 * (size_t)(first + i) + 1];
        bl[0][i] = a.x; bl[1][i] = a.y; bl[2][i] = a.z;
        bh[0][i] = b.x; bh[1][i] = b.y; bh[2][i] = b.z;
    }
    int base = first, m = M;
    for (int lv = 0; lv < levels; ++lv) {
        __syncthreads();
        m >>= 1;
        base >>= 1;
        float l[3], h[3];
        const int i = threadIdx.x;
        if (i < m)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                l[c] = fminf(bl[c][2 * i], bl[c][2 * i + 1]);
                h[c] = fmaxf(bh[c][2 * i], bh[c][2 * i + 1]);
            }
        __syncthreads();
        if (i < m) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                bl[c][i] = l[c];
                bh[c][i] = h[c];
            }
            node[2 * (size_t)(base + i)] = make_float4(l[0], l[1], l[2], 0.f);
            node[2 * (size_t)(base + i) + 1] = make_float4(h[0], h[1], h[2], 0.f);
        }
    }
}

static void cub_tmp_ensure(Scene &S, size_t bytes)
{
    if (bytes <= S.cub_tmp_bytes) return;
    if (S.cub_tmp) dev_free(S, S.cub_tmp);
    S.cub_tmp_bytes = bytes + bytes / 2;
    S.cub_tmp = dev_alloc(S, S.cub_tmp_bytes);
}

static int bvh_reserve(Scene &S, LBVH &T, int n)
{
    if (n <= T.cap) return BF_OK;
    int cap = std::max(n, 16);
    void *old[] = {T.morton, T.morton_alt, T.prim, T.prim_alt, T.lo, T.hi, T.plo, T.phi, T.node};
    for (void *p : old)
        if (p) dev_free(S, p);
    T.morton = (unsigned *)dev_alloc(S, cap * sizeof(unsigned));
    T.morton_alt = (unsigned *)dev_alloc(S, cap * sizeof(unsigned));
    T.prim = (int *)dev_alloc(S, cap * sizeof(int));
    T.prim_alt = (int *)dev_alloc(S, cap * sizeof(int));
    T.lo = (double *)dev_alloc(S, 3 * (size_t)cap * sizeof(double));
    T.hi = (double *)dev_alloc(S, 3 * (size_t)cap * sizeof(double));
    T.plo = (double *)dev_alloc(S, 3 * (size_t)cap * sizeof(double));
    T.phi = (double *)dev_alloc(S, 3 * (size_t)cap * sizeof(double));
    int np2 = 1;
    while (np2 < cap) np2 <<= 1;
    T.node = (float4 *)dev_alloc(S, 2 * 2 * (size_t)np2 * sizeof(float4));
    if (!T.morton || !T.morton_alt || !T.prim || !T.prim_alt || !T.lo || !T.hi || !T.plo || !T.phi || !T.node)
        return BF_E_OOM;
    T.cap = cap;
    T.topo_valid = 0;
    return BF_OK;
}

// node boxes of the implicit tree from the sorted leaves
static void bvh_fill(Scene &S, LBVH &T)
{
    const int n = T.n, N = T.npad;
    k_leaves<<<cdiv(N, kThreads), kThreads, 0, S.stream>>>(n, N, T.prim, T.plo, T.phi, T.lo, T.hi, T.node);
    ++S.n_launch;
    for (int cnt = N; cnt > 1;) {
        const int M = std::min(cnt, kLevelChunk);
        int lv = 0;
        while ((1 << lv) < M) ++lv;
        k_levels<<<cnt / M, 256, 0, S.stream>>>(cnt, M, lv, T.node);
        ++S.n_launch;
        cnt /= M;
    }
}

// Builds the tree over the swept boxes along x0 -> x1 (or the boxes of the
// vertices at x0, x1 and x2 when x2 is given): Morton order of the
// box centres (radix sort), then the node boxes.  Within one time step, when
// the scene allows it, the leaf order of the step's first build is kept and
// only the boxes are recomputed: any leaf order gives the same candidates.
template <int NV>
static int bvh_build(Scene &S, LBVH &T, int n, const int *ids, const double *x0, const double *x1,
                     const double *x2)
{
    if (T.n != n) T.topo_valid = 0;
    T.n = n;
    if (n == 0) return BF_OK;
    int st = bvh_reserve(S, T, n);
    if (st) return st;
    T.npad = 1;
    while (T.npad < n) T.npad <<= 1;
    ScopedTimer tm(S, T_BVH);
    const int nb = cdiv(n, kThreads);
    k_prim_boxes<NV><<<nb, kThreads, 0, S.stream>>>(n, ids, x0, x1, x2, T.plo, T.phi); ++S.n_launch;
    if (!(S.bvh_reuse && T.topo_valid)) {
        int init[6];
        for (int c = 0; c < 3; ++c) {
            init[c] = 0x7f800000;           // +inf as ordered int
            init[3 + c] = (int)0x807fffff;  // -inf as ordered int
        }
        int *bnd = (int *)S.bounds;
        cudaMemcpyAsync(bnd, init, sizeof(init), cudaMemcpyHostToDevice, S.stream);
        k_centroid_bounds<<<nb, kThreads, 0, S.stream>>>(n, T.plo, T.phi, bnd); ++S.n_launch;
        k_morton<<<nb, kThreads, 0, S.stream>>>(n, T.plo, T.phi, bnd, T.morton, T.prim); ++S.n_launch;
        cub::DoubleBuffer<unsigned> keys(T.morton, T.morton_alt);
        cub::DoubleBuffer<int> vals(T.prim, T.prim_alt);
        size_t bytes = 0;
        cub::DeviceRadixSort::SortPairs(nullptr, bytes, keys, vals, n, 0, 30, S.stream);
        cub_tmp_ensure(S, bytes);
        cub::DeviceRadixSort::SortPairs(S.cub_tmp, bytes, keys, vals, n, 0, 30, S.stream);
        if (keys.Current() != T.morton) {
            std::swap(T.morton, T.morton_alt);
            std::swap(T.prim, T.prim_alt);
        }
        T.topo_valid = 1;
    }
    bvh_fill(S, T);
    return BF_OK;
}

__device__ __forceinline__ bool box_overlap_f(const float *ql, const float *qh, float4 l, float4 h)
{
    return !(ql[0] > h.x || l.x > qh[0] || ql[1] > h.y || l.y > qh[1] || ql[2] > h.z || l.z > qh[2]);
}

constexpr int kQueryThreads = 128;
constexpr int kQueryStack = 32;   // a depth-first stack never holds more than the tree depth + 1 nodes
constexpr int kQuerySplitLog = 5;  // each query is traversed as 32 independent subtree walks

struct QueryTree {
    int nq;              // queries
    const int *qids;     // PT: surface vertex per query; EE: unused (queries are the tree's own leaves)
    int n, N;            // leaves, padded leaf count (power of two)
    const float4 *node;  // FP32 boxes of nodes 2.. (node c at [2c], [2c + 1])
    const int *prim;     // primitive per leaf position
    const double *lo, *hi;  // exact FP64 leaf boxes, leaf order
    int2 *cand;
    int *count;
};

// One sub-walk: query q against the subtree rooted at node h0 (all nodes of
// the tree's level ls are roots of the walks; ls = 0 is the root itself).
// Nodes are culled with their FP32 outward-rounded boxes (both children of
// a node from one 64-byte fetch); a leaf is accepted only by the exact FP64
// closed-box test, so the candidates are exactly the pairs whose swept
// boxes overlap.  Type PT queries a surface vertex against the triangle
// tree; type EE queries an edge leaf against the edge leaves after it in
// leaf order (subtrees whose last leaf is not after the query leaf are
// skipped, so every edge pair is met once).  Candidate slots are reserved
// with one atomic per group of converged lanes.
template <int TYPE>
__device__ __forceinline__ void query_walk(const QueryTree &T, int q, int h0, int ls, const double *__restrict__ x0,
                                           const double *__restrict__ x1, const double *__restrict__ x2,
                                           const int *__restrict__ st,
                                           const int *__restrict__ se, const uint8_t *__restrict__ dir, int cap,
                                           int *dflag, int *stk)
{
    const int N = T.N, L = 31 - __clz(N);  // leaves are nodes [N, 2N)
    if (TYPE == EE) {  // the walk's last leaf must come after q
        const int span = 1 << (L - ls);
        if ((h0 - (1 << ls) + 1) * span - 1 <= q) return;
    }
    double ql[3], qh[3];
    int qa, qv0, qv1 = -1;
    if (TYPE == PT) {
        qa = T.qids[q];
        qv0 = qa;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double a = x0[3 * qa + c], b = x1[3 * qa + c];
            ql[c] = fmin(a, b);
            qh[c] = fmax(a, b);
            if (x2) {
                ql[c] = fmin(ql[c], x2[3 * qa + c]);
                qh[c] = fmax(qh[c], x2[3 * qa + c]);
            }
        }
    } else {
        qa = T.prim[q];
        qv0 = se[2 * qa];
        qv1 = se[2 * qa + 1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ql[c] = T.lo[3 * (size_t)q + c];
            qh[c] = T.hi[3 * (size_t)q + c];
        }
    }
    float fl[3], fh[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        fl[c] = __double2float_rd(ql[c]);
        fh[c] = __double2float_ru(qh[c]);
    }
    const bool qdir = TYPE == PT ? dir[qv0] != 0 : (dir[qv0] && dir[qv1]);
    auto leaf = [&](int k) {
        if (k >= T.n || (TYPE == EE && k <= q)) return;
        const double *l2 = T.lo + 3 * (size_t)k, *h2 = T.hi + 3 * (size_t)k;
        if (ql[0] > h2[0] || l2[0] > qh[0] || ql[1] > h2[1] || l2[1] > qh[1] || ql[2] > h2[2] || l2[2] > qh[2])
            return;
        const int b = T.prim[k];
        bool ok;
        if (TYPE == PT) {
            const int t0 = st[3 * b], t1 = st[3 * b + 1], t2 = st[3 * b + 2];
            ok = qv0 != t0 && qv0 != t1 && qv0 != t2 && !(qdir && dir[t0] && dir[t1] && dir[t2]);
        } else {
            const int e0 = se[2 * b], e1 = se[2 * b + 1];
            ok = e0 != qv0 && e0 != qv1 && e1 != qv0 && e1 != qv1 && !(qdir && dir[e0] && dir[e1]);
        }
        if (ok) {
            const unsigned m = __activemask();
            const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
            int base = 0;
            if (lane == lead) base = atomicAdd(T.count, __popc(m));
            base = __shfl_sync(m, base, lead);
            const int idx = base + __popc(m & ((1u << lane) - 1));
            if (idx < cap) T.cand[idx] = TYPE == PT ? make_int2(qa, b) : make_int2(min(qa, b), max(qa, b));
        }
    };
    if (N == 1) {
        leaf(0);
        return;
    }
    if (ls > 0) {  // the walk's own root box
        const float4 *p = T.node + 2 * (size_t)h0;
        if (!box_overlap_f(fl, fh, __ldg(p), __ldg(p + 1))) return;
    }
    stk[0] = h0;
    int sp = 1;
    for (int visits = 0; sp > 0; ++visits) {
        if (visits > N + 64) {  // the tree has N - 1 internal nodes
            atomicOr(dflag + F_ERR, ERR_CAND_OVERFLOW);
            return;
        }
        const int h = stk[--sp * kQueryThreads];
        const int lc = 32 - __clz(h);  // level of the children (root = level 0)
        const float4 *p = T.node + 4 * (size_t)h;  // children 2h, 2h + 1: 4 consecutive float4
        const float4 l0 = __ldg(p), h0b = __ldg(p + 1), l1 = __ldg(p + 2), h1 = __ldg(p + 3);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int cnode = 2 * h + k;
            if (TYPE == EE) {  // skip subtrees whose last leaf is not after q
                const int span = 1 << (L - lc);
                if ((cnode - (1 << lc) + 1) * span - 1 <= q) continue;
            }
            if (!box_overlap_f(fl, fh, k ? l1 : l0, k ? h1 : h0b)) continue;
            if (lc == L) {
                leaf(cnode - N);
            } else {
                if (sp >= kQueryStack) {
                    atomicOr(dflag + F_ERR, ERR_CAND_OVERFLOW);
                    return;
                }
                stk[sp++ * kQueryThreads] = cnode;
            }
        }
    }
}

// level whose nodes root the sub-walks: kQuerySplitLog, but above the leaves
__host__ __device__ __forceinline__ int query_split_level(int N)
{
    int L = 0;
    while ((1 << L) < N) ++L;
    return L <= 1 ? 0 : (L - 1 < kQuerySplitLog ? L - 1 : kQuerySplitLog);
}

// warps of a query type: each warp takes 32 consecutive queries and one
// sub-walk root, so the lanes of a warp walk the same subtree
__host__ __device__ __forceinline__ int query_warps(int nq, int N)
{
    return nq > 0 && N > 0 ? ((nq + 31) / 32) << query_split_level(N) : 0;
}

// Both query types in one launch (the PT warps first, then the EE warps):
// each alone is too small to fill the device.
__global__ void __launch_bounds__(kQueryThreads) k_query(QueryTree pt, QueryTree ee, int wpt, int wee,
                                                         const double *__restrict__ x0, const double *__restrict__ x1,
                                                         const double *__restrict__ x2,
                                                         const int *__restrict__ st, const int *__restrict__ se,
                                                         const uint8_t *__restrict__ dir, int cap, int *dflag)
{
    __shared__ int stack[kQueryStack * kQueryThreads];
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    int *stk = stack + threadIdx.x;
    if (w < wpt) {
        const int ls = query_split_level(pt.N), j = w & ((1 << ls) - 1), q = (w >> ls) * 32 + lane;
        if (q < pt.nq) query_walk<PT>(pt, q, (1 << ls) + j, ls, x0, x1, x2, st, se, dir, cap, dflag, stk);
    } else if ((w -= wpt) < wee) {
        const int ls = query_split_level(ee.N), j = w & ((1 << ls) - 1), q = (w >> ls) * 32 + lane;
        if (q < ee.nq) query_walk<EE>(ee, q, (1 << ls) + j, ls, x0, x1, x2, st, se, dir, cap, dflag, stk);
    }
}

// narrow phase over candidates; mode 0: min TOI, mode 1: collect hits.
// FILTER: the list is a superset; a pair goes on only if its exact FP64
// swept boxes overlap (the test the broad phase's leaf test makes: point
// against triangle, edge against edge, closed boxes)
template <int TYPE, bool FILTER>
__global__ void k_narrow(int n, const int2 *__restrict__ cand, const int *__restrict__ st, const int *__restrict__ se,
                         const double *__restrict__ x0, const double *__restrict__ x1, double s, int max_iter, int mode,
                         double *toi_min, int *hit_type, int *hit_a, int *hit_b, double *hit_toi, int hit_cap,
                         int *nhit)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 c = cand[i];
    const int4 v = pair_vertices(TYPE, c.x, c.y, st, se);
    double p0[12], p1[12], t;
    gather12(x0, v, p0);
    gather12(x1, v, p1);
    if (FILTER) {
        const int split = TYPE == PT ? 1 : 2;  // vertices [0, split) against [split, 4)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double l1 = INFINITY, h1 = -INFINITY, l2 = INFINITY, h2 = -INFINITY;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double lo = fmin(p0[3 * k + a], p1[3 * k + a]), hi = fmax(p0[3 * k + a], p1[3 * k + a]);
                if (k < split) {
                    l1 = fmin(l1, lo);
                    h1 = fmax(h1, hi);
                } else {
                    l2 = fmin(l2, lo);
                    h2 = fmax(h2, hi);
                }
            }
            if (l1 > h2 || l2 > h1) return;
        }
    }
    if (!accd(TYPE, p0, p1, s, 1.0, max_iter, &t)) return;
    if (mode != 1) atomic_min_pos(toi_min, t);  // mode 0: min TOI, 1: hits, 2: both
    if (mode != 0) {
        const int idx = atomicAdd(nhit, 1);
        if (idx < hit_cap) {
            hit_type[idx] = TYPE;
            hit_a[idx] = c.x;
            hit_b[idx] = c.y;
            hit_toi[idx] = t;
        }
    }
}

__global__ void k_accd_pairs(int type, int n, const double *__restrict__ x0, const double *__restrict__ x1, double s,
                             int max_iter, double *__restrict__ toi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double t;
    toi[i] = accd(type, x0 + 12 * (size_t)i, x1 + 12 * (size_t)i, s, 1.0, max_iter, &t) ? t : INFINITY;
}

int accd_pairs(int type, int n, const double *x0, const double *x1, double s, double *toi, cudaStream_t st)
{
    if (n <= 0) return BF_OK;
    k_accd_pairs<<<cdiv(n, 128), 128, 0, st>>>(type, n, x0, x1, s, kAccdMaxIter, toi);
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Allocation-free narrow phase: alpha = min(1, min_i TOI_i) over explicit
// pairs, for callers that cannot allocate device memory.  Its scratch (the
// per-block minima and the arrival counter of the final reduction) is a
// file-scope device array, so the only device memory the call touches is
// the caller's inputs and output and this array.
// ---------------------------------------------------------------------------
constexpr int kNoAllocThreads = 128;
constexpr int kNoAllocMaxBlocks = 8192;  // -> at most 1,048,576 pairs per call
constexpr int kNoAllocMaxPairs = kNoAllocThreads * kNoAllocMaxBlocks;
// [0, kNoAllocMaxBlocks): per-block minimum TOI (bit pattern of a
// non-negative double); [kNoAllocMaxBlocks]: arrival counter (64 KiB + 256 B)
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocMaxBlocks + 32];

__global__ void __launch_bounds__(kNoAllocThreads) k_min_toi_noalloc(int type, int n, const double *__restrict__ x0,
                                                                     const double *__restrict__ x1, double s,
                                                                     int max_iter, unsigned long long *scratch,
                                                                     double *alpha)
{
    __shared__ unsigned long long smin[kNoAllocThreads / 32];
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double t = 1.0;
    double toi;
    if (i < n) {
        // a pair with a non-finite coordinate allows no step (t = 0): its
        // TOI cannot be trusted, and fmin would drop a NaN
        bool finite = true;
        for (int k = 0; k < 12; ++k)
            finite = finite && isfinite(x0[12 * (size_t)i + k]) && isfinite(x1[12 * (size_t)i + k]);
        if (!finite) t = 0.0;
        else if (accd(type, x0 + 12 * (size_t)i, x1 + 12 * (size_t)i, s, 1.0, max_iter, &toi))
            t = toi == toi ? fmin(t, toi) : 0.0;
    }
    unsigned long long b = (unsigned long long)__double_as_longlong(t);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, b, o);
        b = u < b ? u : b;
    }
    if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kNoAllocThreads / 32; ++w) b = smin[w] < b ? smin[w] : b;
        scratch[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(scratch + kNoAllocMaxBlocks, 1ull) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    unsigned long long m = (unsigned long long)__double_as_longlong(1.0);
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        const unsigned long long u = __ldcg(scratch + k);
        m = u < m ? u : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, m, o);
        m = u < m ? u : m;
    }
    if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kNoAllocThreads / 32; ++w) m = smin[w] < m ? smin[w] : m;
        *alpha = __longlong_as_double((long long)m);
        scratch[kNoAllocMaxBlocks] = 0ull;  // ready for the next call
    }
}

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current) and cached.
static int noalloc_scratch(unsigned long long **out)
{
    static std::mutex mu;
    static unsigned long long *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BF_E_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BF_E_CUDA;
        addr[dev] = (unsigned long long *)p;
    }
    *out = addr[dev];
    return BF_OK;
}

int ccd_reserve(Scene &S, int npt, int nee, int nhit)
{
    const int need = std::max(npt, nee);
    if (need > S.cand_cap) {
        const int cap = std::max(need + need / 2, 1024);
        if (S.cand_pt) dev_free(S, S.cand_pt);
        if (S.cand_ee) dev_free(S, S.cand_ee);
        S.cand_pt = (int2 *)dev_alloc(S, cap * sizeof(int2));
        S.cand_ee = (int2 *)dev_alloc(S, cap * sizeof(int2));
        if (!S.cand_pt || !S.cand_ee) return BF_E_OOM;
        S.cand_cap = cap;
    }
    if (nhit > S.hit_cap) {
        const int cap = std::max(nhit + nhit / 2, 1024);
        void *old[] = {S.hit_type, S.hit_a, S.hit_b, S.hit_toi, S.hit_key, S.hit_key_alt, S.hit_idx, S.hit_idx_alt,
                       S.keep};
        for (void *p : old)
            if (p) dev_free(S, p);
        S.hit_type = (int *)dev_alloc(S, cap * sizeof(int));
        S.hit_a = (int *)dev_alloc(S, cap * sizeof(int));
        S.hit_b = (int *)dev_alloc(S, cap * sizeof(int));
        S.hit_toi = (double *)dev_alloc(S, cap * sizeof(double));
        S.hit_key = (unsigned long long *)dev_alloc(S, cap * sizeof(unsigned long long));
        S.hit_key_alt = (unsigned long long *)dev_alloc(S, cap * sizeof(unsigned long long));
        S.hit_idx = (int *)dev_alloc(S, cap * sizeof(int));
        S.hit_idx_alt = (int *)dev_alloc(S, cap * sizeof(int));
        S.keep = (int *)dev_alloc(S, cap * sizeof(int));
        if (!S.hit_type || !S.hit_a || !S.hit_b || !S.hit_toi || !S.hit_key || !S.hit_key_alt || !S.hit_idx ||
            !S.hit_idx_alt || !S.keep)
            return BF_E_OOM;
        S.hit_cap = cap;
    }
    return BF_OK;
}

// Broad phase: candidates (pairs whose swept boxes along x0 -> x1 overlap;
// with x2, the boxes over x0, x1 and x2) into cand_pt / cand_ee, their
// counts to *npt, *nee.
static int broad_phase(Scene &S, const double *x0, const double *x1, const double *x2, int *npt_out, int *nee_out)
{
    int st = bvh_build<3>(S, S.bvh_tri, S.nst, S.st, x0, x1, x2);
    if (st) return st;
    st = bvh_build<2>(S, S.bvh_edge, S.nse, S.se, x0, x1, x2);
    if (st) return st;
    int npt = 0, nee = 0;
    cudaMemsetAsync(S.dflag + F_ERR, 0, sizeof(int), S.stream);
    for (int attempt = 0; attempt < 3; ++attempt) {
        cudaMemsetAsync(S.dflag + F_NCAND_PT, 0, 2 * sizeof(int), S.stream);
        ScopedTimer tq(S, T_CCD_QUERY);
        const QueryTree pt{S.nst ? S.nsv : 0, S.sv, S.bvh_tri.n, S.bvh_tri.npad, S.bvh_tri.node,
                           S.bvh_tri.prim, S.bvh_tri.lo, S.bvh_tri.hi, S.cand_pt, S.dflag + F_NCAND_PT};
        const QueryTree ee{S.nse > 1 ? S.nse : 0, nullptr, S.bvh_edge.n, S.bvh_edge.npad, S.bvh_edge.node,
                           S.bvh_edge.prim, S.bvh_edge.lo, S.bvh_edge.hi, S.cand_ee, S.dflag + F_NCAND_EE};
        const int wpt = query_warps(pt.nq, pt.N), wee = query_warps(ee.nq, ee.N);
        if (wpt + wee > 0) {
            const int wpb = kQueryThreads / 32;
            k_query<<<cdiv(wpt + wee, wpb), kQueryThreads, 0, S.stream>>>(pt, ee, wpt, wee, x0, x1, x2, S.st,
                                                                        S.se, S.dir, S.cand_cap, S.dflag);
            ++S.n_launch;
        }
        st = sync_flags(S);
        if (st) return st;
        npt = S.h_flag[F_NCAND_PT];
        nee = S.h_flag[F_NCAND_EE];
        if (S.h_flag[F_ERR] & ERR_CAND_OVERFLOW) return BF_E_CAPACITY;
        if (npt <= S.cand_cap && nee <= S.cand_cap) break;
        st = ccd_reserve(S, npt, nee, 0);
        if (st) return st;
    }
    if (npt > S.cand_cap || nee > S.cand_cap) return BF_E_CAPACITY;
    *npt_out = npt;
    *nee_out = nee;
    return BF_OK;
}

// Narrow phase over the listed pairs, mode 0: min TOI (with NH also the
// inversion bound) to *alpha_out; 1: every hit; 2: both in one pass (the
// CCD reuse of the active-set update).  Hits:
// (type, a, b, toi) stored and counted to *nhits_out.  With `filter` the
// lists cover a wider motion: a pair goes on only if its exact swept boxes
// along x0 -> x1 overlap, so exactly the candidates of this motion remain.
static void launch_narrow(Scene &S, const double *x0, const double *x1, int npt, int nee, bool filter, int mode)
{
    const double s = S.prm.s_ccd;
    if (mode != 0) cudaMemsetAsync(S.dflag + F_NHIT, 0, sizeof(int), S.stream);
    if (mode != 1) {
        const double one = 1.0;
        cudaMemcpyAsync(S.dscal + S_TOI, &one, sizeof(double), cudaMemcpyHostToDevice, S.stream);
    }
    ScopedTimer tm(S, T_CCD_NARROW);
    auto launch = [&](auto kern, int n, const int2 *cand) {
        if (!n) return;
        kern<<<cdiv(n, 128), 128, 0, S.stream>>>(n, cand, S.st, S.se, x0, x1, s, kAccdMaxIter, mode,
                                                S.dscal + S_TOI, S.hit_type, S.hit_a, S.hit_b, S.hit_toi, S.hit_cap,
                                                S.dflag + F_NHIT);
        ++S.n_launch;
    };
    if (filter) {
        launch(k_narrow<PT, true>, npt, S.cand_pt);
        launch(k_narrow<EE, true>, nee, S.cand_ee);
    } else {
        launch(k_narrow<PT, false>, npt, S.cand_pt);
        launch(k_narrow<EE, false>, nee, S.cand_ee);
    }
    // NH is not defined for inverted elements: MaxStepSize also keeps every
    // element's volume (section 4.1)
    if (mode != 1 && S.prm.model == BF_MODEL_NH) launch_inversion_bound(S, x0, x1, S.dscal + S_TOI);
}

static int narrow_phase(Scene &S, const double *x0, const double *x1, int npt, int nee, bool filter,
                        bool collect_hits, double *alpha_out, int *nhits_out)
{
    for (int attempt = 0; attempt < 3; ++attempt) {
        launch_narrow(S, x0, x1, npt, nee, filter, collect_hits ? 1 : 0);
        int st = sync_flags(S);
        if (st) return st;
        if (!collect_hits) {
            if (alpha_out) *alpha_out = std::min(1.0, S.h_scal[S_TOI]);
            return BF_OK;
        }
        const int nh = S.h_flag[F_NHIT];
        if (nh <= S.hit_cap) {
            if (nhits_out) *nhits_out = nh;
            return BF_OK;
        }
        st = ccd_reserve(S, 0, 0, nh);
        if (st) return st;
    }
    return BF_E_CAPACITY;
}

// Broad + narrow phase along x0 -> x1.  collect_hits: store every hit
// (type, a, b, toi) and return their count; else *alpha_out = min(1, TOI).
int run_ccd(Scene &S, const double *x0, const double *x1, bool collect_hits, double *alpha_out, int *nhits_out)
{
    int npt = 0, nee = 0;
    const int st = broad_phase(S, x0, x1, nullptr, &npt, &nee);
    if (st) return st;
    return narrow_phase(S, x0, x1, npt, nee, false, collect_hits, alpha_out, nhits_out);
}

// The two CCD passes of an outer iteration start at the same x0: the
// candidates over the boxes of x0, xa and xb contain those of both motions,
// and the exact box test of each narrow pass keeps exactly its own.
int run_ccd_two(Scene &S, const double *x0, const double *xa, const double *xb, int *nhits_a, double *alpha_b)
{
    int npt = 0, nee = 0;
    int st = broad_phase(S, x0, xa, xb, &npt, &nee);
    if (st) return st;
    for (int attempt = 0; attempt < 3; ++attempt) {  // both narrow passes, one synchronisation
        launch_narrow(S, x0, xa, npt, nee, true, 1);
        launch_narrow(S, x0, xb, npt, nee, true, 0);
        st = sync_flags(S);
        if (st) return st;
        const int nh = S.h_flag[F_NHIT];
        if (nh <= S.hit_cap) {
            *nhits_a = nh;
            *alpha_b = std::min(1.0, S.h_scal[S_TOI]);
            return BF_OK;
        }
        st = ccd_reserve(S, 0, 0, nh);
        if (st) return st;
    }
    return BF_E_CAPACITY;
}

// CCD reuse (option ccd_reuse): the MaxStepSize segment x0 -> x1 gives
// both the step bound and the hits of the active-set update, from one
// broad phase over the two position sets and one narrow pass.
int run_ccd_reuse(Scene &S, const double *x0, const double *x1, int *nhits, double *alpha)
{
    int npt = 0, nee = 0;
    int st = broad_phase(S, x0, x1, nullptr, &npt, &nee);
    if (st) return st;
    for (int attempt = 0; attempt < 3; ++attempt) {
        launch_narrow(S, x0, x1, npt, nee, false, 2);
        st = sync_flags(S);
        if (st) return st;
        const int nh = S.h_flag[F_NHIT];
        if (nh <= S.hit_cap) {
            *nhits = nh;
            *alpha = std::min(1.0, S.h_scal[S_TOI]);
            return BF_OK;
        }
        st = ccd_reserve(S, 0, 0, nh);
        if (st) return st;
    }
    return BF_E_CAPACITY;
}

// ---------------------------------------------------------------------------
// Alg. 3 UpdateActiveSet
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long pair_key(int type, int a, int b)
{
    return ((unsigned long long)type << 62) | ((unsigned long long)a << 31) | (unsigned long long)b;
}

__global__ void k_ckeys(int nc, const int *__restrict__ ctype, const int *__restrict__ ca, const int *__restrict__ cb,
                        unsigned long long *__restrict__ key)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) key[i] = pair_key(ctype[i], ca[i], cb[i]);
}

// new pairs (not in C) lower the per-vertex minimum TOI T_v (Alg. 3, per-vertex minimum)
__global__ void k_new_hits(int nh, const int *__restrict__ ht, const int *__restrict__ ha, const int *__restrict__ hb,
                           const double *__restrict__ htoi, const unsigned long long *__restrict__ ck, int nc,
                           const int *__restrict__ st, const int *__restrict__ se, int *__restrict__ isnew,
                           unsigned long long *__restrict__ tv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nh) return;
    const unsigned long long k = pair_key(ht[i], ha[i], hb[i]);
    int lo = 0, hi = nc - 1;
    bool found = false;
    while (lo <= hi) {
        const int m = (lo + hi) >> 1;
        const unsigned long long km = ck[m];
        if (km == k) {
            found = true;
            break;
        }
        if (km < k) lo = m + 1;
        else hi = m - 1;
    }
    isnew[i] = found ? 0 : 1;
    if (found) return;
    const int4 v = pair_vertices(ht[i], ha[i], hb[i], st, se);
    const unsigned long long t = (unsigned long long)__double_as_longlong(htoi[i]);
    atomicMin(tv + v.x, t);
    atomicMin(tv + v.y, t);
    atomicMin(tv + v.z, t);
    atomicMin(tv + v.w, t);
}

// keep a new pair whose TOI equals T_v of one of its vertices (Alg. 3, filter)
__global__ void k_keep(int nh, const int *__restrict__ ht, const int *__restrict__ ha, const int *__restrict__ hb,
                       const double *__restrict__ htoi, const int *__restrict__ isnew, const int *__restrict__ st,
                       const int *__restrict__ se, const unsigned long long *__restrict__ tv,
                       unsigned long long *__restrict__ kkey, int *__restrict__ kidx, int *nkeep)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nh || !isnew[i]) return;
    const int4 v = pair_vertices(ht[i], ha[i], hb[i], st, se);
    const unsigned long long t = (unsigned long long)__double_as_longlong(htoi[i]);
    if (tv[v.x] == t || tv[v.y] == t || tv[v.z] == t || tv[v.w] == t) {
        const int j = atomicAdd(nkeep, 1);
        kkey[j] = pair_key(ht[i], ha[i], hb[i]);
        kidx[j] = i;
    }
}

__global__ void k_append(int nk, int nc, const int *__restrict__ kidx, const int *__restrict__ ht,
                         const int *__restrict__ ha, const int *__restrict__ hb, const int *__restrict__ st,
                         const int *__restrict__ se, int *ctype, int *ca, int *cb, int4 *cv, double *clam, double *cgam)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nk) return;
    const int i = kidx[j];
    const int o = nc + j;
    ctype[o] = ht[i];
    ca[o] = ha[i];
    cb[o] = hb[i];
    cv[o] = pair_vertices(ht[i], ha[i], hb[i], st, se);
    clam[o] = 0.0;
    cgam[o] = 1.0;
}

// prune gamma < 0.01 (Alg. 3, decay pruning): stable compaction in place via a scan
__global__ void k_prune_flags(int nc, const double *__restrict__ cgam, int *__restrict__ flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) flag[i] = cgam[i] < 0.01 ? 0 : 1;
}

template <class T>
__global__ void k_scatter(int nc, const int *__restrict__ flag, const int *__restrict__ pos, const T *__restrict__ in,
                          T *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc && flag[i]) out[pos[i]] = in[i];
}

int active_reserve(Scene &S, int n);

template <class T>
static void compact_array(Scene &S, int nc, const int *flag, const int *pos, T *&arr, void *scratch)
{
    k_scatter<T><<<cdiv(nc, kThreads), kThreads, 0, S.stream>>>(nc, flag, pos, arr, (T *)scratch); ++S.n_launch;
    cudaMemcpyAsync(arr, scratch, nc * sizeof(T), cudaMemcpyDeviceToDevice, S.stream);
}

int run_update_active_set(Scene &S, const double *x, const double *xhat)
{
    int nh = 0;
    const int st = run_ccd(S, x, xhat, true, nullptr, &nh);
    if (st) return st;
    return apply_active_set_hits(S, nh);
}

int apply_active_set_hits(Scene &S, int nh)
{
    int st = BF_OK;
    if (nh > 0) {
        // sorted keys of C for the membership test
        size_t bytes = 0;
        if (S.nc > 0) {
            k_ckeys<<<cdiv(S.nc, kThreads), kThreads, 0, S.stream>>>(S.nc, S.ctype, S.ca, S.cb, S.ckey); ++S.n_launch;
            cub::DeviceRadixSort::SortKeys(nullptr, bytes, S.ckey, S.ckey_sorted, S.nc, 0, 64, S.stream);
            cub_tmp_ensure(S, bytes);
            cub::DeviceRadixSort::SortKeys(S.cub_tmp, bytes, S.ckey, S.ckey_sorted, S.nc, 0, 64, S.stream);
        }
        cudaMemsetAsync(S.tv, 0x7f, (size_t)S.nv * sizeof(unsigned long long), S.stream);
        k_new_hits<<<cdiv(nh, kThreads), kThreads, 0, S.stream>>>(nh, S.hit_type, S.hit_a, S.hit_b, S.hit_toi,
                                                                  S.ckey_sorted, S.nc, S.st, S.se, S.keep, S.tv); ++S.n_launch;
        cudaMemsetAsync(S.dflag + F_NKEEP, 0, sizeof(int), S.stream);
        k_keep<<<cdiv(nh, kThreads), kThreads, 0, S.stream>>>(nh, S.hit_type, S.hit_a, S.hit_b, S.hit_toi, S.keep,
                                                             S.st, S.se, S.tv, S.hit_key, S.hit_idx,
                                                             S.dflag + F_NKEEP); ++S.n_launch;
        st = sync_flags(S);
        if (st) return st;
        const int nk = S.h_flag[F_NKEEP];
        if (nk > 0) {
            // deterministic order: sort the kept pairs by key
            cub::DoubleBuffer<unsigned long long> kb(S.hit_key, S.hit_key_alt);
            cub::DoubleBuffer<int> vb(S.hit_idx, S.hit_idx_alt);
            bytes = 0;
            cub::DeviceRadixSort::SortPairs(nullptr, bytes, kb, vb, nk, 0, 64, S.stream);
            cub_tmp_ensure(S, bytes);
            cub::DeviceRadixSort::SortPairs(S.cub_tmp, bytes, kb, vb, nk, 0, 64, S.stream);
            st = active_reserve(S, S.nc + nk);
            if (st) return st;
            {
                k_append<<<cdiv(nk, kThreads), kThreads, 0, S.stream>>>(nk, S.nc, vb.Current(), S.hit_type, S.hit_a,
                                                                   S.hit_b, S.st, S.se, S.ctype, S.ca, S.cb, S.cv,
                                                                   S.clam, S.cgam); ++S.n_launch;
            }
            S.nc += nk;
        }
    }
    if (S.nc == 0) return BF_OK;
    // prune
    int *flag = (int *)S.ckey;  // reuse scratch (>= nc ints)
    int *pos = (int *)S.ckey_sorted;
    k_prune_flags<<<cdiv(S.nc, kThreads), kThreads, 0, S.stream>>>(S.nc, S.cgam, flag); ++S.n_launch;
    size_t bytes = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, bytes, flag, pos, S.nc, S.stream);
    cub_tmp_ensure(S, bytes);
    cub::DeviceScan::ExclusiveSum(S.cub_tmp, bytes, flag, pos, S.nc, S.stream);
    int lastflag = 0, lastpos = 0;
    cudaMemcpyAsync(&lastflag, flag + S.nc - 1, sizeof(int), cudaMemcpyDeviceToHost, S.stream);
    cudaMemcpyAsync(&lastpos, pos + S.nc - 1, sizeof(int), cudaMemcpyDeviceToHost, S.stream);
    st = check_cuda(cudaStreamSynchronize(S.stream));
    if (st) return st;
    const int keep = lastpos + lastflag;
    if (keep == S.nc) return BF_OK;
    void *scratch = S.cw;  // nc doubles of scratch (recomputed every Newton iteration)
    void *scratch16 = S.cg; // 12 nc doubles
    compact_array<int>(S, S.nc, flag, pos, S.ctype, scratch);
    compact_array<int>(S, S.nc, flag, pos, S.ca, scratch);
    compact_array<int>(S, S.nc, flag, pos, S.cb, scratch);
    compact_array<double>(S, S.nc, flag, pos, S.clam, scratch);
    compact_array<double>(S, S.nc, flag, pos, S.cgam, scratch);
    compact_array<int4>(S, S.nc, flag, pos, S.cv, scratch16);
    S.nc = keep;
    return check_cuda(cudaGetLastError());
}

}  // namespace bf

extern "C" int bf_max_step_size_pairs_noalloc(int32_t type, int32_t n, const double *x0, const double *x1, double s,
                                              double *alpha, void *stream)
{
    using namespace bf;
    if ((type != PT && type != EE) || n < 0 || !alpha || !(s > 0 && s < 1)) return BF_E_ARG;
    if (n > kNoAllocMaxPairs) return BF_E_ARG;
    if (n > 0 && (!x0 || !x1)) return BF_E_ARG;
    unsigned long long *scratch = nullptr;
    int st = noalloc_scratch(&scratch);
    if (st) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    // the arrival counter must start at zero (a failed earlier call may have
    // left it set); no other scratch needs clearing: every block writes its
    // own minimum before it is read
    if (cudaMemsetAsync(scratch + kNoAllocMaxBlocks, 0, sizeof(unsigned long long), cs) != cudaSuccess)
        return BF_E_CUDA;
    const int blocks = std::max(1, cdiv(n, kNoAllocThreads));
    k_min_toi_noalloc<<<blocks, kNoAllocThreads, 0, cs>>>(type, n, x0, x1, s, kAccdMaxIter, scratch, alpha);
    if (cudaGetLastError() != cudaSuccess) return BF_E_CUDA;
    return check_cuda(cudaStreamSynchronize(cs));
}
