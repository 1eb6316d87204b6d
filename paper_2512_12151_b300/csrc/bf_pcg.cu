// Persistent block-Jacobi PCG (section 5.1): one cooperative launch per
// linear solve, one CTA per SM, all CTAs co-resident.
//
// Work split: CTA c owns the contiguous vertex rows [part[c], part[c+1]),
// balanced by block count.  It keeps x, r, the row sums q = (H p) and the
// 3x3 preconditioner of its rows in shared memory for the whole solve and,
// when they fit in the combined shared memory of the GPU (the "resident"
// variant), also the blocks of its rows (full-row view: upper blocks and
// the transposed lower ones), row after row, with its neighbours as 16-bit
// offsets into the CTA's vertex window, which covers every neighbour of its
// rows.  The direction p over that window also stays in shared memory: each
// iteration updates it in place, p = z + beta p, from the z values of the
// window (16 bytes per vertex), so every CTA holds bit-identical copies of p
// on the vertices it shares with others.  Each thread then takes a run of
// consecutive blocks (stored interleaved, so that a warp reads consecutive
// 9-word blocks: no bank conflicts), sums them per row in registers and adds
// each row piece to shared memory once, so the SpMV needs no global atomics.
//
// Contact pairs (rank one: mu gamma g g^T) are dealt round-robin to the
// CTAs (pair i -> CTA i % gridDim.x), so that each CTA carries an equal share
// however the pairs cluster on the mesh.  A CTA caches its pairs' gradient,
// weight and ids in shared memory for the solve, fetches the p values at
// their vertices together with its window, and adds mu gamma g (g . p) to a
// global contact vector with atomics; the owners of the rows read (and
// clear) that vector after the next grid-wide reduction.
//
// Two grid-wide reductions per iteration double as the grid barriers:
//   A: q = H p (p updated in place first; contact part to the contact
//      vector); reduce p.q -> alpha
//   B: x += alpha p, r -= alpha q, z = P r; reduce r.z and r.r -> beta,
//      convergence test.
// Thread 0 of every CTA reads the reduced values and derives the scalars
// (alpha, beta, the next state) once for its CTA; every CTA reads the same
// reduced bits, so all take the same decisions.  Every spin has an
// iteration limit (ERR_BARRIER).
//
// Mixed precision runs the iterations in FP32 (p, q, z, r and the increment
// of x).  Dot products are accumulated without loss beyond FP64-like
// accuracy: per CTA as compensated FP32 sums (every rounding error of the
// additions is kept exactly by Knuth's TwoSum and summed separately, the
// cascaded summation of Ogita, Rump and Oishi, "Accurate sum and dot
// product", 2005), across CTAs in FP64.  Reliable updates: whenever |r| has
// dropped by 10x since the last one, or the recurrence signals convergence,
// x is folded into its FP64 value and r is recomputed as b - H x with FP64
// vectors (FP32 matrix); convergence is decided on that residual.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <mutex>
#include <type_traits>
#include <vector>

#include "bf_device.cuh"
#include "bf_internal.cuh"

namespace bf {

constexpr int kPcgThreads = 512;  // threads per CTA at one CTA per SM
constexpr int kPcgMaxWarps = kPcgThreads / 32;
constexpr int kPcgMaxCached = 256;  // contact pairs per CTA cached in shared memory
constexpr int kPcgMaxGrid = 1024;  // CTAs of one launch
constexpr int kPcgEntriesPerCta = 3072;  // target full-row blocks per CTA for small systems

struct PcgArgs {
    int nv, nc;
    const int *part, *win, *frowptr;
    const unsigned short *eslot;     // shared-memory slot of every full-row entry (resident variant)
    const void *jval;                // global variant: blocks in jagged order, 9 planes of nfull values
    const unsigned short *jnbr;      // global variant: window offset of each jagged slot
    unsigned char *gvec;             // global variant: per-CTA x, x_l, r, q (gvec_stride bytes each)
    size_t gvec_stride;
    int nfull;
    const int *rinfo, *lvl, *lvlptr;  // rows by decreasing length; level offsets per CTA
    const int *fnbr, *fblk;
    const void *val;
    const int4 *cv;
    const double *cg, *cw;
    const unsigned char *cmask;
    const void *pinv;
    const double *b;
    double *x;
    void *z, *p0, *p1;
    double *qd;               // FP64 contact part of H x (reliable updates)
    double *res;
    unsigned *bar;
    const unsigned *bar_poll;  // the word the barrier spins on (bar, or an idle word in the failure test)
    double tol2;
    int maxit, max_replace, max_rows, max_ent, max_win, max_len, kc;
    double *dscal;
    int *dflag;
    // symmetric variant: the upper blocks in consumption order (chunks of 9
    // FP32 planes and 16-bit neighbour offsets; chunk table in lvl, its
    // per-CTA start in lvlptr) and the accumulation vector of transposed
    // products and contact terms
    const void *uval;
    float4 *yq;
    // single-reduction variant: published row sums, FP64 contact parts,
    // owners' (r, s), FP64 H x of the reliable updates
    void *cwq, *crs, *cpp;
    double *cqc, *chx;
    unsigned char *cfl;
    float4 *z4;  // symmetric variant: z = P r, one float4 per vertex
};

enum { PCG_RUN = 0, PCG_DONE, PCG_MAXIT, PCG_BAD, PCG_FOLD, PCG_ABORT };

// scalar state of the recurrence, maintained by thread 0 of each CTA
// (rr_done = tol^2 |b|^2 and rr_fold, the |r|^2 of the next reliable update,
// are formed once, not in every reduction)
struct PcgCtl {
    double alpha, beta, rz, rz_old, rr, rr_done, rr_fold, bb;
    float al, bt;
    int it, folds, state;
};

// num / den rounded to FP32, for the scalars that only reach FP32 vector
// updates: an FP32 division of the rounded operands when both lie within
// [2^-100, 2^100] in magnitude (short: this GPU's FP64 pipe is narrow and
// an FP64 division sits on the path through every grid-wide reduction),
// else the FP64 quotient rounded.  Every CTA computes the same bits.
__device__ __forceinline__ float div_to_f32(double num, double den)
{
    const int en = (__double2hiint(num) >> 20) & 0x7ff, ed = (__double2hiint(den) >> 20) & 0x7ff;
    if (en > 923 && en < 1123 && ed > 923 && ed < 1123)
        return __fdiv_rn(__double2float_rn(num), __double2float_rn(den));
    return __double2float_rn(num / den);
}

// Finiteness and order tests on IEEE-754 bit patterns with integer
// operations, for the scalar steps on the path through a grid-wide reduction
// (this GPU's FP64 pipe is narrow): finite; 0 < x < inf; a <= b for a, b in
// [+0, inf].
__device__ __forceinline__ bool finite_b(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff; }
__device__ __forceinline__ bool pos_b(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool le_nonneg_b(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Knuth's TwoSum: s = fl(a + b) and the exact rounding error e = a + b - s
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bv = s - a;
    e = (a - (s - bv)) + (b - bv);
}

// compensated FP32 accumulator: the value is s + c
struct AccF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        float e;
        two_sum(s, v, s, e);
        c += e;
    }
    __device__ __forceinline__ void add(double v)  // an FP64 value as two FP32 parts
    {
        const float hi = (float)v;
        add(hi);
        add((float)(v - (double)hi));
    }
};

__device__ __forceinline__ void acc_add(AccF &a, float v) { a.add(v); }
__device__ __forceinline__ void acc_add(AccF &a, double v) { a.add(v); }
__device__ __forceinline__ void acc_add(double &a, double v) { a += v; }

// butterfly sum of compensated pairs over a warp (the same result in every
// lane: TwoSum is exact whatever the operand order)
__device__ __forceinline__ void warp_sum2(float &s, float &c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, s, o);
        const float co = __shfl_xor_sync(0xffffffffu, c, o);
        float e;
        two_sum(s, so, s, e);
        c = (c + co) + e;
    }
}

// block sum of K compensated accumulators; the FP64 result is valid in warp 0
template <int K>
__device__ __forceinline__ void block_sum(AccF (&a)[K], double (&out)[K], float2 *sh)
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        warp_sum2(a[k].s, a[k].c);
        if (lane == 0) sh[k * kPcgMaxWarps + w] = make_float2(a[k].s, a[k].c);
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 v = lane < nw ? sh[k * kPcgMaxWarps + lane] : make_float2(0.f, 0.f);
            float s = v.x, c = v.y;
            warp_sum2(s, c);
            out[k] = (double)s + (double)c;
        }
    }
}

// block sum of K FP64 values: every thread parks its values in shared
// memory (sh: K x blockDim.x), up to four warps each add a share (strided,
// then shuffles) and thread 0 adds the shares; valid in thread 0
template <int K>
__device__ __forceinline__ void block_sum(double (&a)[K], double (&out)[K], double *sh, double *q4)
{
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * blockDim.x + threadIdx.x] = a[k];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = min(4, (int)(blockDim.x + 31) >> 5);
    const int share = ((int)blockDim.x + nw - 1) / nw;
    if (w < nw) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = 0.0;
            for (int i = lane; i < share; i += 32) {
                const int j = w * share + i;
                if (j < (int)blockDim.x) t += sh[k * blockDim.x + j];
            }
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) q4[4 * k + w] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = q4[4 * k];
            for (int i = 1; i < nw; ++i) t += q4[4 * k + i];
            out[k] = t;
        }
}

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s: far beyond any legitimate wait

// Grid-wide sum of K block sums (called by thread 0 of every CTA) that
// doubles as the grid barrier.  Reduction: each CTA adds its block sum to
// accumulator slot (n % 3) with an FP64 atomic add, n = the count of
// reductions so far in this launch; CTA 0 zeroes slot (n + 1) % 3 before it
// arrives (that slot was last read before the previous barrier and is next
// written after this one).  Barrier: one arrival counter whose top bit
// flips when every CTA has arrived (CTA 0 adds 0x80000000 - (gridDim.x - 1),
// the others 1, so the sum of one barrier's arrivals is 0x80000000), with a
// release on the arrival and acquire loads of `poll` while spinning
// (bounded: ERR_BARRIER and false on timeout).  `poll` is `bar` except in the
// failure-detection test, which polls a word no CTA increments.
template <int K>
__device__ __forceinline__ bool grid_total(const double (&v)[K], double *acc, unsigned n, unsigned *bar,
                                           const unsigned *poll, int *dflag, double (&tot)[K])
{
    const unsigned slot = n % 3u, next = (n + 1u) % 3u;
#pragma unroll
    for (int k = 0; k < K; ++k) atomicAdd(acc + 8 * slot + k, v[k]);
    if (blockIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[8 * next + k] = 0.0;
    // the top bit of the counter is (n + 1) & 1 once barrier n is complete
    // (it flips at the last arrival of every barrier), so the arrival needs
    // no returned value and the polling starts at once
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(add) : "memory");
    const unsigned want = ((n + 1u) & 1u) << 31;
    unsigned spins = 0;
    unsigned long long t_start = 0;
    while ((ld_acquire_gpu(poll) & 0x80000000u) != want) {
        if ((++spins & 255u) == 0u) {  // give up after kBarrierTimeoutNs
            const unsigned long long t = globaltimer();
            if (t_start == 0) t_start = t;
            else if (t - t_start > kBarrierTimeoutNs) {
                atomicOr(dflag + F_ERR, ERR_BARRIER);
                return false;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = __ldcg(acc + 8 * slot + k);
    return true;
}

// Row sums of H u over the CTA's rows, stored into s_q (component-major,
// s_q[c * ldq + row]).  One thread per row; rows are taken in the CTA's
// order of decreasing length, so the threads of a warp run loops of about
// the same length.  rinfo[t] = (local row << 8) | row length of the t-th
// row in that order; ent(t, row, j, a) loads the 9 values of the row's j-th
// block and returns the neighbour's window offset; getu(v_rel, out) loads u
// there.  Every row is written, so s_q needs no clearing.
template <int UNROLL, class CT, class GetU, class Ent>
__device__ __forceinline__ void row_sums(int nr, const int *rinfo, GetU getu, Ent ent, CT *s_q, int ldq)
{
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
        const int info = rinfo[t];
        const int row = info >> 8, len = info & 255;
        CT y0 = CT(0), y1 = CT(0), y2 = CT(0);
#pragma unroll UNROLL
        for (int j = 0; j < len; ++j) {
            CT a[9], u[3];
            getu(ent(t, row, j, a), u);
            y0 += a[0] * u[0] + a[1] * u[1] + a[2] * u[2];
            y1 += a[3] * u[0] + a[4] * u[1] + a[5] * u[2];
            y2 += a[6] * u[0] + a[7] * u[1] + a[8] * u[2];
        }
        s_q[row] = y0;
        s_q[ldq + row] = y1;
        s_q[2 * ldq + row] = y2;
    }
}

template <class T>
__device__ __forceinline__ void load3v(const T *src, T *u)
{
    if (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(src);
        u[0] = q.x; u[1] = q.y; u[2] = q.z;
    } else {
        u[0] = src[0]; u[1] = src[1]; u[2] = src[2];
    }
}

// the direction update p = z + beta p_old, written once so that every CTA
// rounds it the same way
__device__ __forceinline__ float dir_update(float z, float bt, float p) { return fmaf(bt, p, z); }
__device__ __forceinline__ double dir_update(double z, double bt, double p) { return fma(bt, p, z); }

// Shared-memory layout of the persistent PCG (byte offsets, 16-byte aligned
// sections), shared by the kernel and the host-side sizing.
struct PcgLayout {
    size_t x, xl, r, q, pinv, p4, val, nbr, rinfo, lvl, cg, cp, cw, cv, cm, total;
};

// Modes: 0 = blocks read from the BSR values through the full-row map,
// vectors in shared memory; 1 = blocks resident in shared memory; 2 = blocks
// streamed from a jagged copy in global memory (coalesced), per-row vectors
// in global memory (systems whose rows do not fit in shared memory); 3 =
// upper blocks only streamed from a jagged copy, transposed products
// accumulated in global memory (mixed precision; k_pcg_sym below); 4 =
// blocks resident in shared memory, one grid-wide reduction per iteration
// (k_pcg_cg1 below).
enum { PCG_STREAM = 0, PCG_RESIDENT = 1, PCG_GLOBAL = 2, PCG_SYM = 3, PCG_CG1 = 4 };

__host__ __device__ inline PcgLayout pcg_layout(bool mixed, int ct, int mt, int max_rows, int max_win, int max_ent,
                                                int max_len, int mode, int kc)
{
    const bool res = mode == PCG_RESIDENT, vec = mode != PCG_GLOBAL;
    PcgLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    const int rt = mixed ? 4 : 8;
    L.x = take(vec ? 3 * (size_t)max_rows * 8 : 0);
    L.xl = take(vec && mixed ? 3 * (size_t)max_rows * rt : 0);
    L.r = take(vec ? 3 * (size_t)max_rows * rt : 0);
    L.q = take(vec ? 3 * (size_t)max_rows * (mixed ? 8 : ct) : 0);  // FP64 H x of the reliable updates reuses it
    L.pinv = take(vec ? 9 * (size_t)max_rows * mt : 0);
    L.p4 = take(4 * (size_t)max_win * ct);
    L.val = take(res ? 9 * (size_t)max_ent * mt : 0);
    L.nbr = take(res ? (size_t)max_ent * 2 : 0);
    L.rinfo = take((size_t)max_rows * 4);
    L.lvl = take(((size_t)max_len + 1) * 4);
    L.cg = take(12 * (size_t)kc * ct);
    L.cp = take(12 * (size_t)kc * ct);
    L.cw = take((size_t)kc * ct);
    L.cv = take((size_t)kc * 16);
    L.cm = take((size_t)kc * 4);
    L.total = o;
    return L;
}

// the per-CTA vector region of the global variant (same offsets scheme)
__host__ __device__ inline PcgLayout pcg_vec_layout(bool mixed, int ct, int max_rows)
{
    PcgLayout L = pcg_layout(mixed, ct, 4, max_rows, 0, 0, 0, PCG_STREAM, 0);
    L.total = L.pinv;  // x, x_l, r, q only
    return L;
}

// bytes of one cached contact pair (gradient, p at its vertices, weight, ids, flags)
inline size_t pcg_contact_bytes(int ct) { return 25 * (size_t)ct + 20; }

template <class MT, class VT, int MODE>
__global__ void __launch_bounds__(kPcgThreads, 1) k_pcg_persistent(PcgArgs A)
{
    constexpr bool RES = MODE == PCG_RESIDENT, GV = MODE == PCG_GLOBAL;
    using CT = typename std::conditional<(sizeof(MT) >= sizeof(VT)), MT, VT>::type;
    constexpr bool mixed = sizeof(VT) == 4;
    using RT = typename std::conditional<mixed, float, double>::type;  // r and the iteration part of x
    using Acc = typename std::conditional<mixed, AccF, double>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PcgCtl ctl;
    __shared__ float2 red_f[2 * kPcgMaxWarps];
    __shared__ double red_d[mixed ? 1 : 2 * kPcgThreads];
    __shared__ double red_q4[8];
    const MT *__restrict__ gval = (const MT *)A.val;
    const MT *__restrict__ gpinv = (const MT *)A.pinv;
    VT *__restrict__ z = (VT *)A.z;
    VT *pb[2] = {(VT *)A.p0, (VT *)A.p1};
    // contact part of H p, accumulated in FP64 in both precisions (the order
    // of the atomics then changes only the last bits of an FP64 sum)
    double *__restrict__ qcd = A.qd;
    const int c = blockIdx.x;
    const int r0 = A.part[c], r1 = A.part[c + 1], nr = r1 - r0;
    const int wlo = A.win[2 * c], whi = A.win[2 * c + 1], nwin = whi - wlo;
    const int E0 = A.frowptr[r0], ne = A.frowptr[r1] - E0;  // the CTA's full-row entries
    const int nco = A.nc > c ? (A.nc - c + (int)gridDim.x - 1) / (int)gridDim.x : 0;  // pairs c + k grid
    const int ncached = min(nco, A.kc);
    const PcgLayout L =
        pcg_layout(mixed, sizeof(CT), sizeof(MT), A.max_rows, A.max_win, A.max_ent, A.max_len, MODE, A.kc);
    const PcgLayout Lv = GV ? pcg_vec_layout(mixed, sizeof(CT), A.max_rows) : L;
    unsigned char *vb = GV ? A.gvec + (size_t)c * A.gvec_stride : smem;  // per-row vectors
    const int ld = A.max_rows;  // per-row arrays are component-major: a[c * ld + row]
    double *s_x = (double *)(vb + Lv.x);
    RT *s_xl = (RT *)(vb + Lv.xl);
    RT *s_r = (RT *)(vb + Lv.r);
    CT *s_q = (CT *)(vb + Lv.q);
    double *s_hx = (double *)(vb + Lv.q);
    const MT *s_pinv = GV ? gpinv + 9 * (size_t)r0 : (const MT *)(smem + L.pinv);
    CT *s_p4 = (CT *)(smem + L.p4);
    MT *s_val = (MT *)(smem + L.val);
    unsigned short *s_nbr = (unsigned short *)(smem + L.nbr);
    int *s_rinfo = (int *)(smem + L.rinfo);
    int *s_lvl = (int *)(smem + L.lvl);
    CT *s_cg = (CT *)(smem + L.cg);
    CT *s_cp = (CT *)(smem + L.cp);
    CT *s_cw = (CT *)(smem + L.cw);
    int4 *s_cv = (int4 *)(smem + L.cv);
    int *s_cm = (int *)(smem + L.cm);
    if (!GV)
        for (int i = threadIdx.x; i < 9 * nr; i += blockDim.x) ((MT *)(smem + L.pinv))[i] = gpinv[9 * (size_t)r0 + i];
    if (RES) {
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            const int fe = E0 + e;
            const int fb = A.fblk[fe];
            const int slot = A.eslot[fe];
            const MT *src = gval + 9 * (size_t)(fb & 0x7fffffff);
            MT *dst = s_val + 9 * slot;
            if (fb < 0) {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) dst[3 * i + j] = src[3 * j + i];
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) dst[i] = src[i];
            }
            s_nbr[slot] = (unsigned short)(A.fnbr[fe] - wlo);
        }
    }
    if (RES || GV)
        for (int j = threadIdx.x; j < A.lvlptr[c + 1] - A.lvlptr[c]; j += blockDim.x) s_lvl[j] = A.lvl[A.lvlptr[c] + j];
    for (int t = threadIdx.x; t < nr; t += blockDim.x) s_rinfo[t] = A.rinfo[r0 + t];
    for (int k = threadIdx.x; k < ncached; k += blockDim.x) {
        const int i = c + k * (int)gridDim.x;
        s_cv[k] = A.cv[i];
        s_cm[k] = A.cmask[i];
        s_cw[k] = (CT)A.cw[i];
#pragma unroll
        for (int j = 0; j < 12; ++j) s_cg[12 * k + j] = (CT)A.cg[12 * (size_t)i + j];
    }
    for (int i = threadIdx.x; i < 4 * nwin; i += blockDim.x) s_p4[i] = CT(0);  // p_old = 0
    // values of the j-th block of local row `row` (row-major, lower blocks
    // transposed; in shared memory at level j, position t of the row order);
    // returns the neighbour's window offset
    auto ent = [&](int t, int row, int j, CT *a) -> int {
        if (RES) {
            const int slot = s_lvl[j] + t;
            const MT *v = s_val + 9 * slot;
#pragma unroll
            for (int i = 0; i < 9; ++i) a[i] = (CT)v[i];
            return s_nbr[slot];
        } else if (GV) {  // 9 coalesced planes, streamed past the caches
            const size_t slot = (size_t)E0 + s_lvl[j] + t;
            const MT *v = (const MT *)A.jval + slot;
#pragma unroll
            for (int i = 0; i < 9; ++i) a[i] = (CT)__ldcs(v + (size_t)i * A.nfull);
            return __ldcs(A.jnbr + slot);
        } else {
            const int fe = __ldg(A.frowptr + r0 + row) + j;
            const int fb = __ldg(A.fblk + fe);
            const MT *src = gval + 9 * (size_t)(fb & 0x7fffffff);
            if (fb < 0) {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) a[3 * i + j] = (CT)__ldg(src + 3 * j + i);
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) a[i] = (CT)__ldg(src + i);
            }
            return __ldg(A.fnbr + fe) - wlo;
        }
    };
    // z = P r for row i (written to global memory); returns the row's r.z
    auto precond = [&](int i, const RT *rv) -> CT {
        const int a = r0 + i;
        const MT *P = s_pinv + 9 * i;
        CT zc[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            zc[k] = (CT)P[3 * k] * (CT)rv[0] + (CT)P[3 * k + 1] * (CT)rv[1] + (CT)P[3 * k + 2] * (CT)rv[2];
            z[3 * a + k] = (VT)zc[k];
        }
        return ((CT)rv[0] * zc[0] + (CT)rv[1] * zc[1]) + (CT)rv[2] * zc[2];
    };
    unsigned nred = 0;  // reductions so far (selects the accumulator slot)
    // block sum then grid sum; thread 0 runs on_total(tot) (or marks the
    // CTA aborted), then the CTA synchronises
    auto reduce = [&](auto &acc, auto on_total) {
        constexpr int K = (int)std::extent<std::remove_reference_t<decltype(acc)>>::value;
        double blk[K], tot[K];
        if constexpr (mixed) block_sum<K>(acc, blk, red_f);
        else block_sum<K>(acc, blk, red_d, red_q4);
        if (threadIdx.x == 0) {
            if (grid_total<K>(blk, A.res, nred, A.bar, A.bar_poll, A.dflag, tot)) on_total(tot);
            else ctl.state = PCG_ABORT;
        }
        ++nred;
        __syncthreads();
    };
    unsigned long long tA = 0, tA2 = 0, tB = 0, tB2 = 0, t0 = 0, tS = 0, tR = 0, tC = 0;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    __syncthreads();
    // ---- init: r = b, x = 0, z = P r, p_old = 0 ------------------------------
    {
        Acc acc[2] = {};
        for (int i = threadIdx.x; i < nr; i += blockDim.x) {
            const int a = r0 + i;
            RT rv[3];
            double bb = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double bk = A.b[3 * a + k];
                rv[k] = (RT)bk;
                s_r[k * ld + i] = rv[k];
                s_x[k * ld + i] = 0.0;
                if (mixed) s_xl[k * ld + i] = RT(0);
                qcd[3 * a + k] = 0.0;
                if (A.nc > 0) pb[0][3 * a + k] = VT(0);
                bb += bk * bk;  // |b|^2 in FP64
            }
            acc_add(acc[0], precond(i, rv));
            acc_add(acc[1], bb);
        }
        reduce(acc, [&](const double *t) {
            ctl.rz = t[0];
            ctl.bb = t[1];
            ctl.rr = t[1];
            ctl.rr_done = A.tol2 * t[1];
            ctl.rr_fold = 0.01 * t[1];
            ctl.beta = 0.0;
            ctl.bt = 0.f;
            ctl.it = 0;
            ctl.folds = 0;
            if (pos_b(t[1]) && finite_b(t[0]) && finite_b(t[1])) ctl.state = PCG_RUN;
            else ctl.state = t[1] == 0.0 ? PCG_DONE : PCG_BAD;
        });
    }
    int parity = 0;
    while (ctl.state == PCG_RUN) {
        VT *pold = pb[parity], *pnew = pb[parity ^ 1];
        // ---- phase A: p = z + beta p over the window, q = H p ----------------
        {
            if (timer) t0 = globaltimer();
            const CT bt = mixed ? (CT)ctl.bt : (CT)ctl.beta;
            {  // window z and the contacts' p: coalesced loads issued together
                const int nf = 3 * nwin, ncf = 12 * ncached, ntot = nf + ncf;
                const VT *zw = z + 3 * wlo;
                for (int f0 = threadIdx.x; f0 < ntot; f0 += 8 * blockDim.x) {
                    VT zz[8], pp[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int f = f0 + k * blockDim.x;
                        zz[k] = VT(0);
                        pp[k] = VT(0);
                        if (f < nf) {
                            zz[k] = __ldcg(zw + f);
                        } else if (f < ntot) {
                            const int g = f - nf, kk = g / 12, q = (g % 12) / 3, j = g % 3;
                            if (s_cm[kk] >> q & 1) {
                                const int v = (&s_cv[kk].x)[q];
                                zz[k] = __ldcg(z + 3 * v + j);
                                pp[k] = __ldcg(pold + 3 * v + j);
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int f = f0 + k * blockDim.x;
                        if (f < nf) {
                            CT *d = s_p4 + 4 * (f / 3) + f % 3;
                            *d = dir_update((CT)zz[k], bt, *d);
                        } else if (f < ntot) {
                            s_cp[f - nf] = dir_update((CT)zz[k], bt, (CT)pp[k]);
                        }
                    }
                }
            }
            __syncthreads();
            if (timer) tS += globaltimer() - t0;
            auto getp = [&](int vr, CT *o) { load3v(s_p4 + 4 * vr, o); };
            row_sums<2, CT>(nr, s_rinfo, getp, ent, s_q, ld);
            if (timer) tR += globaltimer() - t0;
            // this CTA's contact pairs: y += mu gamma g (g . p) into qcd
            CT cdot = CT(0);
            for (int k = threadIdx.x; k < nco; k += blockDim.x) {
                CT g[12], u[12], w;
                int vid[4], m;
                if (k < ncached) {
                    const int4 v = s_cv[k];
                    vid[0] = v.x; vid[1] = v.y; vid[2] = v.z; vid[3] = v.w;
                    m = s_cm[k];
                    w = s_cw[k];
#pragma unroll
                    for (int j = 0; j < 12; ++j) {
                        g[j] = s_cg[12 * k + j];
                        u[j] = s_cp[12 * k + j];
                    }
                } else {
                    const int i = c + k * (int)gridDim.x;
                    const int4 v = A.cv[i];
                    vid[0] = v.x; vid[1] = v.y; vid[2] = v.z; vid[3] = v.w;
                    m = A.cmask[i];
                    w = (CT)A.cw[i];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            g[3 * q + j] = (CT)A.cg[12 * (size_t)i + 3 * q + j];
                            u[3 * q + j] = (m >> q & 1) ? dir_update((CT)__ldcg(z + 3 * vid[q] + j), bt,
                                                                     (CT)__ldcg(pold + 3 * vid[q] + j))
                                                        : CT(0);
                        }
                }
                CT s = CT(0);
#pragma unroll
                for (int j = 0; j < 12; ++j) s += g[j] * u[j];
                const CT t = w * s;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (m >> q & 1)
#pragma unroll
                        for (int j = 0; j < 3; ++j) atomicAdd(qcd + 3 * vid[q] + j, (double)(t * g[3 * q + j]));
                cdot += t * s;
            }
            __syncthreads();
            if (timer) tC += globaltimer() - t0;
            Acc acc[1] = {};
            acc_add(acc[0], cdot);  // p^T H_c p of this CTA's pairs
            for (int i = threadIdx.x; i < nr; i += blockDim.x) {
                const int a = r0 + i;
                CT p[3];
                load3v(s_p4 + 4 * (a - wlo), p);
                if (A.nc > 0)
#pragma unroll
                    for (int k = 0; k < 3; ++k) pnew[3 * a + k] = (VT)p[k];  // read by other CTAs' pairs
                acc_add(acc[0], (p[0] * s_q[i] + p[1] * s_q[ld + i]) + p[2] * s_q[2 * ld + i]);
            }
            if (timer) {
                const unsigned long long t1 = globaltimer();
                tA += t1 - t0;
                t0 = t1;
            }
            reduce(acc, [&](const double *t) {
                const double pq = t[0];
                if (!finite_b(pq)) {
                    ctl.state = PCG_BAD;
                } else if (!pos_b(pq)) {
                    // no curvature left along p: stop with the current x, as the
                    // per-phase solver does, and let the line search judge it
                    ctl.state = PCG_DONE;
                } else if (mixed) {
                    ctl.al = div_to_f32(ctl.rz, pq);
                    ctl.alpha = (double)ctl.al;
                } else {
                    ctl.alpha = ctl.rz / pq;
                    ctl.al = (float)ctl.alpha;
                }
            });
            if (timer) {
                const unsigned long long t1 = globaltimer();
                tA2 += t1 - t0;
                t0 = t1;
            }
        }
        if (ctl.state != PCG_RUN) break;
        // ---- phase B: x, r, z updates ---------------------------------------
        {
            const double alpha = ctl.alpha;
            const RT al = mixed ? (RT)ctl.al : (RT)alpha;
            Acc acc[2] = {};
#pragma unroll 2
            for (int i = threadIdx.x; i < nr; i += blockDim.x) {
                const int a = r0 + i;
                VT qg[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) qg[k] = (VT)__ldcg(qcd + 3 * a + k);
                CT pc[3];
                load3v(s_p4 + 4 * (a - wlo), pc);
                RT rv[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    if (mixed) s_xl[k * ld + i] += al * (RT)pc[k];
                    else s_x[k * ld + i] += alpha * (double)pc[k];
                    rv[k] = s_r[k * ld + i] - al * ((RT)s_q[k * ld + i] + (RT)qg[k]);
                    s_r[k * ld + i] = rv[k];
                    qcd[3 * a + k] = 0.0;
                }
                acc_add(acc[0], precond(i, rv));
                acc_add(acc[1], ((CT)rv[0] * (CT)rv[0] + (CT)rv[1] * (CT)rv[1]) + (CT)rv[2] * (CT)rv[2]);
            }
            if (timer) {
                const unsigned long long t1 = globaltimer();
                tB += t1 - t0;
                t0 = t1;
            }
            reduce(acc, [&](const double *t) {
                ++ctl.it;
                ctl.rz_old = ctl.rz;
                if (mixed) {
                    ctl.bt = div_to_f32(t[0], ctl.rz_old);
                    ctl.beta = (double)ctl.bt;
                } else {
                    ctl.beta = t[0] / ctl.rz_old;
                    ctl.bt = (float)ctl.beta;
                }
                ctl.rz = t[0];
                ctl.rr = t[1];
                if (!finite_b(t[0]) || !finite_b(t[1])) {
                    ctl.state = PCG_BAD;
                    return;
                }
                const bool done = le_nonneg_b(ctl.rr, ctl.rr_done);  // rr, rr_done, rr_fold >= 0
                if (mixed && ctl.folds < A.max_replace && (done || le_nonneg_b(ctl.rr, ctl.rr_fold)))
                    ctl.state = PCG_FOLD;
                else if (done)
                    ctl.state = PCG_DONE;
                else if (ctl.it >= A.maxit)
                    ctl.state = PCG_MAXIT;
            });
            if (timer) tB2 += globaltimer() - t0;
        }
        parity ^= 1;
        if constexpr (mixed) {
        if (ctl.state == PCG_FOLD) {
            // reliable update: x += x_l in FP64, then r = b - H x with FP64
            // vectors (FP32 matrix); the direction p is kept and beta rescaled
            for (int i = threadIdx.x; i < nr; i += blockDim.x)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double xv = s_x[k * ld + i] + (double)s_xl[k * ld + i];
                    s_x[k * ld + i] = xv;
                    s_xl[k * ld + i] = RT(0);
                    A.x[3 * (r0 + i) + k] = xv;
                }
            {
                AccF none[1];
                reduce(none, [&](const double *) {});  // x visible to every CTA
            }
            if (ctl.state == PCG_ABORT) break;
            auto getx = [&](int vr, double *o) {
#pragma unroll
                for (int k = 0; k < 3; ++k) o[k] = __ldcg(A.x + 3 * (wlo + vr) + k);
            };
            auto ent64 = [&](int t, int row, int j, double *a) -> int {
                CT tv[9];
                const int v = ent(t, row, j, tv);
#pragma unroll
                for (int k = 0; k < 9; ++k) a[k] = (double)tv[k];
                return v;
            };
            row_sums<2, double>(nr, s_rinfo, getx, ent64, s_hx, ld);
            for (int k = threadIdx.x; k < nco; k += blockDim.x) {
                const int i = c + k * (int)gridDim.x;
                const int4 v = A.cv[i];
                const int mk = A.cmask[i];
                const int vid[4] = {v.x, v.y, v.z, v.w};
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (mk >> q & 1)
#pragma unroll
                        for (int j = 0; j < 3; ++j) s += A.cg[12 * (size_t)i + 3 * q + j] * __ldcg(A.x + 3 * vid[q] + j);
                const double t = A.cw[i] * s;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (mk >> q & 1)
#pragma unroll
                        for (int j = 0; j < 3; ++j) atomicAdd(A.qd + 3 * vid[q] + j, t * A.cg[12 * (size_t)i + 3 * q + j]);
            }
            {
                AccF none[1];
                reduce(none, [&](const double *) {});  // contact parts complete
            }
            if (ctl.state == PCG_ABORT) break;
            AccF acc[2];
            for (int i = threadIdx.x; i < nr; i += blockDim.x) {
                const int a = r0 + i;
                RT rv[3];
                double rr = 0.0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double rh = A.b[3 * a + k] - s_hx[k * ld + i] - __ldcg(A.qd + 3 * a + k);
                    A.qd[3 * a + k] = 0.0;
                    rr += rh * rh;
                    rv[k] = (RT)rh;
                    s_r[k * ld + i] = rv[k];
                }
                acc_add(acc[0], (float)precond(i, rv));
                acc_add(acc[1], rr);
            }
            reduce(acc, [&](const double *t) {
                ++ctl.folds;
                ctl.bt = div_to_f32(t[0], ctl.rz_old);
                ctl.beta = (double)ctl.bt;
                ctl.rz = t[0];
                ctl.rr = t[1];
                ctl.rr_fold = 0.01 * t[1];
                if (!finite_b(t[0]) || !finite_b(t[1])) ctl.state = PCG_BAD;
                else if (le_nonneg_b(ctl.rr, ctl.rr_done)) ctl.state = PCG_DONE;
                else if (ctl.it >= A.maxit) ctl.state = PCG_MAXIT;
                else ctl.state = PCG_RUN;
            });
        }
        }
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            A.x[3 * (r0 + i) + k] = s_x[k * ld + i] + (mixed ? (double)s_xl[k * ld + i] : 0.0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.dflag[F_ITERS] = ctl.it;
        A.dflag[F_MAXIT] = ctl.state == PCG_MAXIT;
        A.dflag[F_DONE] = 1;
        if (ctl.state == PCG_BAD) A.dflag[F_ERR] |= ERR_NONFINITE;
        A.dscal[S_RR] = ctl.rr;
        A.dscal[S_BB] = ctl.bb;
        A.dscal[S_RZ] = ctl.rz;
        A.dscal[S_T_SPMV] = 1e-6 * (double)tA;
        A.dscal[S_T_RED1] = 1e-6 * (double)tA2;
        A.dscal[S_T_UPD] = 1e-6 * (double)tB;
        A.dscal[S_T_RED2] = 1e-6 * (double)tB2;
        A.dscal[S_T_STAGE] = 1e-6 * (double)tS;
        A.dscal[S_T_ROWS] = 1e-6 * (double)tR;
        A.dscal[S_T_CONTACT] = 1e-6 * (double)tC;
    }
}

// ---------------------------------------------------------------------------
// Single-reduction variant of the resident PCG: the recurrence of Chronopoulos
// and Gear ("s-step iterative methods for symmetric linear systems", J.
// Comput. Appl. Math. 25, 1989), which gives the iterates of the
// two-reduction form in exact arithmetic with one grid-wide reduction per
// iteration.  Iteration k:
//   u = P r, w = H u; gamma = r.u, delta = u.w, |r|^2   (one reduction)
//   beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
//   p = u + beta p, s = w + beta s (s = H p by recurrence), x += alpha p,
//   r -= alpha s.
// The product needs u on the CTA's whole vertex window, so every CTA runs the
// recurrences of s and r, and u = P r, on its window itself: the same
// operations (explicitly rounded, no contraction left to the compiler) on the
// same bits give every CTA bit-identical copies of the values the owner of a
// row holds.  What crosses CTAs is only w: each owner publishes the full-row
// sums of its rows (double-buffered by iteration parity) and the contact
// pairs add their part in FP64 (triple-buffered: written in iteration k, read
// after the reduction of k, cleared by the owners in k + 2).  The vertices of
// a CTA's contact pairs may lie outside its window: there it takes r and s of
// the previous iteration from the owners' published copy (double-buffered)
// and applies the same update.  Blocks stay in shared memory as in the
// resident variant, and so does the upper triangle of P over the window (P
// is the inverse of a symmetric block; every CTA applies the same symmetric
// form).  The row sums and contact parts are read from component planes in
// global memory (L2), so a warp's loads are coalesced, the contact part only
// at the vertices of a pair (flagged per vertex at the start of the solve).
//
// Mixed precision: s, r, u, p and the increment of x in FP32, dot products
// compensated (AccF) and summed across CTAs in FP64, x in FP64.  Reliable
// updates as in the two-reduction form (|r| down 10x, or convergence): x is
// folded, r = b - H x is recomputed with FP64 vectors, and the product of the
// same iteration is redone from the new r; the recurrences of s and p carry
// on.
// ---------------------------------------------------------------------------
struct PcgCg1Layout {
    size_t x, xl, pd, wq, u4, sw, rw, pw, val, nbr, rinfo, lvl, cg, cu, cw, cv, cm, fl, total;
};

__host__ __device__ inline PcgCg1Layout pcg_cg1_layout(bool mixed, int ct, int mt, int max_rows, int max_win,
                                                       int max_ent, int max_len, int kc)
{
    PcgCg1Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    L.x = take(3 * (size_t)max_rows * 8);
    L.xl = take(mixed ? 3 * (size_t)max_rows * ct : 0);
    L.pd = take(3 * (size_t)max_rows * ct);
    L.wq = take(3 * (size_t)max_rows * ct);
    L.u4 = take(4 * (size_t)max_win * ct);
    L.sw = take(3 * (size_t)max_win * ct);
    L.rw = take(3 * (size_t)max_win * ct);
    L.pw = take(6 * (size_t)max_win * ct);
    L.val = take(9 * (size_t)max_ent * mt);
    L.nbr = take((size_t)max_ent * 2);
    L.rinfo = take((size_t)max_rows * 4);
    L.lvl = take(((size_t)max_len + 1) * 4);
    L.cg = take(12 * (size_t)kc * ct);
    L.cu = take(12 * (size_t)kc * ct);
    L.cw = take((size_t)kc * ct);
    L.cv = take((size_t)kc * 16);
    L.cm = take((size_t)kc * 4);
    L.fl = take((size_t)max_win);
    L.total = o;
    return L;
}

// Global buffers of the single-reduction variant, in this order (byte
// offsets as multiples of nv): row sums w (2 parities x 3 planes, 6 ct),
// FP64 contact parts (3 buffers x 3 planes, 72), the owners' (r, s) (2
// parities, 8 values per vertex, 16 ct), FP64 H x of the reliable updates
// (24), the upper triangle of P (6 planes, 6 ct), a byte per vertex that
// flags the vertices of contact pairs (zero between solves).
struct PcgCg1Buf {
    size_t wq, qc, rs, hx, pp, fl, total;
};

inline PcgCg1Buf pcg_cg1_buf(int nv_, int ct)
{
    const size_t nv = (size_t)nv_;
    PcgCg1Buf B;
    B.wq = 0;
    B.qc = B.wq + 6 * nv * ct;
    B.rs = B.qc + 72 * nv;
    B.hx = B.rs + 16 * nv * ct;
    B.pp = B.hx + 24 * nv;
    B.fl = B.pp + 6 * nv * ct;
    B.total = B.fl + ((nv + 15) & ~(size_t)15);
    return B;
}

// scalar state of the single-reduction recurrence (thread 0 of each CTA;
// the reciprocals of gamma_old and alpha_old are formed by another thread
// during the product, off the path through the reduction: an FP64 division
// is long on this GPU, whose FP64 pipe is narrow)
struct PcgCg1Ctl {
    double alpha, beta, gam_old, inv_gam_old, c_old, rr, rr_done, rr_fold, bb;  // c_old = 1 / (gamma_old alpha_old)
    float al, bt;
    int it, folds, state, skip;
};


// explicitly rounded operations, so that every CTA computes the window
// recurrences to the same bits whatever code the compiler emits around them
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float to_ct(double v, float) { return __double2float_rn(v); }
__device__ __forceinline__ double to_ct(double v, double) { return v; }

// u = P r for one vertex, P symmetric given by its upper triangle
// (p00, p01, p02, p11, p12, p22)
template <class CT>
__device__ __forceinline__ void prec3(const CT (&P)[6], const CT (&r)[3], CT (&u)[3])
{
    u[0] = fma_rn(P[2], r[2], fma_rn(P[1], r[1], mul_rn(P[0], r[0])));
    u[1] = fma_rn(P[4], r[2], fma_rn(P[3], r[1], mul_rn(P[1], r[0])));
    u[2] = fma_rn(P[5], r[2], fma_rn(P[4], r[1], mul_rn(P[2], r[0])));
}

// row-major index of upper-triangle entry i of a 3x3 block: 0, 1, 2, 4, 5, 8
__host__ __device__ constexpr int upper3(int i) { return i < 3 ? i : (i < 5 ? i + 1 : 8); }

template <class MT, class VT>
__global__ void __launch_bounds__(kPcgThreads, 1) k_pcg_cg1(PcgArgs A)
{
    using CT = typename std::conditional<(sizeof(MT) >= sizeof(VT)), MT, VT>::type;
    constexpr bool mixed = sizeof(VT) == 4;
    using Acc = typename std::conditional<mixed, AccF, double>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PcgCg1Ctl ctl;
    __shared__ float2 red_f[3 * kPcgMaxWarps];
    __shared__ double red_d[mixed ? 1 : 3 * kPcgThreads];
    __shared__ double red_q4[12];
    __shared__ unsigned long long tm[8];  // A, A2, -, -, t0, S, R, C
    const MT *__restrict__ gval = (const MT *)A.val;
    const MT *__restrict__ gpinv = (const MT *)A.pinv;
    const int c = blockIdx.x;
    const int r0 = A.part[c], r1 = A.part[c + 1], nr = r1 - r0;
    const int wlo = A.win[2 * c], whi = A.win[2 * c + 1], nwin = whi - wlo;
    const int E0 = A.frowptr[r0], ne = A.frowptr[r1] - E0;
    const int nco = A.nc > c ? (A.nc - c + (int)gridDim.x - 1) / (int)gridDim.x : 0;  // pairs c + k grid
    const int ncached = min(nco, A.kc);
    const PcgCg1Layout L =
        pcg_cg1_layout(mixed, sizeof(CT), sizeof(MT), A.max_rows, A.max_win, A.max_ent, A.max_len, A.kc);
    const int ld = A.max_rows, lw = A.max_win;  // component-major: own rows a[k ld + i], window a[k lw + j]
    double *s_x = (double *)(smem + L.x);
    CT *s_xl = (CT *)(smem + L.xl);
    CT *s_pd = (CT *)(smem + L.pd);
    CT *s_wq = (CT *)(smem + L.wq);
    CT *s_u4 = (CT *)(smem + L.u4);
    CT *s_sw = (CT *)(smem + L.sw);
    CT *s_rw = (CT *)(smem + L.rw);
    CT *s_pw = (CT *)(smem + L.pw);
    MT *s_val = (MT *)(smem + L.val);
    unsigned short *s_nbr = (unsigned short *)(smem + L.nbr);
    int *s_rinfo = (int *)(smem + L.rinfo);
    int *s_lvl = (int *)(smem + L.lvl);
    CT *s_cg = (CT *)(smem + L.cg);
    CT *s_cu = (CT *)(smem + L.cu);
    CT *s_cw = (CT *)(smem + L.cw);
    int4 *s_cv = (int4 *)(smem + L.cv);
    int *s_cm = (int *)(smem + L.cm);
    unsigned char *s_fl = smem + L.fl;
    const size_t nv = (size_t)A.nv;
    CT *const wqb = (CT *)A.cwq;   // row sums of w: parity m, component q at wqb + nv (3 m + q)
    double *const qcb = A.cqc;    // contact part of w: buffer m, component q at qcb + nv (3 m + q)
    CT *const rsb = (CT *)A.crs;   // owners' (r, s): parity m at rsb + 8 nv m, 8 values per vertex
    CT *const ppl = (CT *)A.cpp;   // P: upper-triangle entry i of vertex a at ppl[i nv + a]
    unsigned char *const gfl = A.cfl;  // vertices of contact pairs
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const int fe = E0 + e;
        const int fb = A.fblk[fe];
        const int slot = A.eslot[fe];
        const MT *src = gval + 9 * (size_t)(fb & 0x7fffffff);
        MT *dst = s_val + 9 * slot;
        if (fb < 0) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) dst[3 * i + j] = src[3 * j + i];
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) dst[i] = src[i];
        }
        s_nbr[slot] = (unsigned short)(A.fnbr[fe] - wlo);
    }
    for (int j = threadIdx.x; j < A.lvlptr[c + 1] - A.lvlptr[c]; j += blockDim.x) s_lvl[j] = A.lvl[A.lvlptr[c] + j];
    for (int t = threadIdx.x; t < nr; t += blockDim.x) s_rinfo[t] = A.rinfo[r0 + t];
    for (int k = threadIdx.x; k < ncached; k += blockDim.x) {
        const int i = c + k * (int)gridDim.x;
        s_cv[k] = A.cv[i];
        s_cm[k] = A.cmask[i];
        s_cw[k] = (CT)A.cw[i];
#pragma unroll
        for (int j = 0; j < 12; ++j) s_cg[12 * k + j] = (CT)A.cg[12 * (size_t)i + j];
    }
    for (int i = threadIdx.x; i < 3 * lw; i += blockDim.x) s_sw[i] = CT(0);
    // the upper triangle of P of the own rows into the planes, and the flags
    // of this CTA's pairs' vertices (read by other CTAs after the first
    // reduction)
    for (int e = threadIdx.x; e < 6 * nr; e += blockDim.x) {
        const int i = e / nr, row = e - i * nr;
        const size_t a = (size_t)(r0 + row);
        ppl[(size_t)i * nv + a] = (CT)gpinv[9 * a + upper3(i)];
    }
    for (int kk = threadIdx.x; kk < nco; kk += blockDim.x) {
        const int i = c + kk * (int)gridDim.x;
        const int4 v = A.cv[i];
        const int m = A.cmask[i];
        if (m & 1) gfl[v.x] = 1;
        if (m & 2) gfl[v.y] = 1;
        if (m & 4) gfl[v.z] = 1;
        if (m & 8) gfl[v.w] = 1;
    }
    auto load_p = [&](size_t a, CT (&P)[6]) {
#pragma unroll
        for (int i = 0; i < 6; ++i) P[i] = __ldcg(ppl + (size_t)i * nv + a);
    };
    // w of vertex a from the product of iteration m >= 0: the row sum plus,
    // where the vertex belongs to a pair, the contact part rounded to CT (no
    // FP64 arithmetic per window row: the FP64 pipe is narrow)
    auto load_w = [&](size_t a, int m, bool in_pair, CT (&w)[3]) {
        const CT *wq = wqb + 3 * nv * (size_t)(m & 1) + a;
        const double *qc = qcb + 3 * nv * (size_t)(m % 3) + a;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            w[q] = __ldcg(wq + q * nv);
            if (in_pair) w[q] = add_rn(w[q], to_ct(__ldcg(qc + q * nv), CT()));
        }
    };
    // r of vertex a as its owner published it: values 0..2 (r) or 4..6 (s) of parity m
    auto load_rs = [&](size_t a, int m, int off, CT (&v)[3]) {
        const CT *p = rsb + 8 * nv * (size_t)(m & 1) + 8 * a + off;
        if (mixed) {
            const float4 f = __ldcg(reinterpret_cast<const float4 *>(p));
            v[0] = f.x; v[1] = f.y; v[2] = f.z;
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q) v[q] = __ldcg(p + q);
        }
    };
    unsigned nred = 0;
    auto reduce = [&](auto &acc, auto on_total) {
        constexpr int K = (int)std::extent<std::remove_reference_t<decltype(acc)>>::value;
        double blk[K], tot[K];
        if constexpr (mixed) block_sum<K>(acc, blk, red_f);
        else block_sum<K>(acc, blk, red_d, red_q4);
        if (threadIdx.x == 0) {
            if (grid_total<K>(blk, A.res, nred, A.bar, A.bar_poll, A.dflag, tot)) on_total(tot);
            else ctl.state = PCG_ABORT;
        }
        ++nred;
        __syncthreads();
    };
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < 8; ++i) tm[i] = 0;
    __syncthreads();
    // ---- init: x = 0, p = s = 0, r = b (published for iteration 0) --------
    {
        Acc acc[1] = {};
        for (int i = threadIdx.x; i < nr; i += blockDim.x) {
            const size_t a = (size_t)(r0 + i);
            double bb = 0.0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const double bk = A.b[3 * a + q];
                s_x[q * ld + i] = 0.0;
                if (mixed) s_xl[q * ld + i] = CT(0);
                s_pd[q * ld + i] = CT(0);
#pragma unroll
                for (int m = 0; m < 3; ++m) qcb[nv * (3 * m + q) + a] = 0.0;
                A.qd[3 * a + q] = 0.0;
                rsb[8 * a + q] = to_ct(bk, CT());
                rsb[8 * a + 4 + q] = CT(0);
                bb += bk * bk;
            }
            acc_add(acc[0], bb);
        }
        reduce(acc, [&](const double *t) {
            ctl.bb = t[0];
            ctl.rr = t[0];
            ctl.rr_done = A.tol2 * t[0];
            ctl.rr_fold = 0.01 * t[0];
            ctl.alpha = ctl.beta = ctl.gam_old = ctl.inv_gam_old = ctl.c_old = 0.0;
            ctl.al = ctl.bt = 0.f;
            ctl.it = 0;
            ctl.folds = 0;
            ctl.skip = 1;
            if (pos_b(t[0])) ctl.state = PCG_RUN;
            else ctl.state = t[0] == 0.0 ? PCG_DONE : PCG_BAD;
        });
    }
    if (ctl.state == PCG_RUN) {  // P and the pair flags over the window
        for (int e = threadIdx.x; e < 6 * nwin; e += blockDim.x) {
            const int i = e / nwin, j = e - i * nwin;
            s_pw[i * lw + j] = __ldcg(ppl + (size_t)i * nv + wlo + j);
        }
        for (int j = threadIdx.x; j < nwin; j += blockDim.x) s_fl[j] = __ldcg(gfl + wlo + j);
        __syncthreads();
    }
    while (ctl.state == PCG_RUN) {
        const int k = ctl.it;
        const bool upd = !ctl.skip;
        const CT al = mixed ? (CT)ctl.al : (CT)ctl.alpha, bt = mixed ? (CT)ctl.bt : (CT)ctl.beta;
        const double alpha = ctl.alpha;  // FP64 only
        if (timer) tm[4] = globaltimer();
        Acc acc[3] = {};  // gamma = r.u, delta = u.H u, |r|^2
        // ---- stage: the recurrences over the window and at the vertices of
        // the cached contact pairs (items nwin + 4 pair + vertex), u = P r ----
        {
            CT *rsc = rsb + 8 * nv * (size_t)(k & 1);
            double *qcn = qcb + 3 * nv * (size_t)((k + 1) % 3);  // product k - 2: read before the reduction of k - 1
            const int nitem = nwin + 4 * ncached;
            constexpr int RB = mixed ? 2 : 1;  // items per thread whose loads are issued together
            for (int i0 = threadIdx.x; i0 < nitem; i0 += RB * blockDim.x) {
                CT P[RB][6], w[RB][3], ro[RB][3], so[RB][3];
                int av[RB];
#pragma unroll
                for (int v = 0; v < RB; ++v) {
                    const int e = i0 + v * (int)blockDim.x;
                    av[v] = -1;
                    if (e < nwin) {
                        av[v] = wlo + e;
                    } else if (e < nitem) {
                        const int kk = (e - nwin) >> 2, q = (e - nwin) & 3;
                        if (s_cm[kk] >> q & 1) av[v] = (&s_cv[kk].x)[q];
                    }
                    if (av[v] >= 0) {
                        const size_t a = (size_t)av[v];
                        if (e < nwin) {
#pragma unroll
                            for (int i = 0; i < 6; ++i) P[v][i] = s_pw[i * lw + e];
                        } else {
                            load_p(a, P[v]);
                        }
                        if (upd) load_w(a, k - 1, e >= nwin || s_fl[e], w[v]);
                        if (e >= nwin && upd) {  // a pair's vertex: (r, s) of iteration k - 1
                            load_rs(a, k - 1, 0, ro[v]);
                            load_rs(a, k - 1, 4, so[v]);
                        } else if (!upd) {
                            load_rs(a, k, 0, ro[v]);  // r published for iteration k
                        }
                    }
                }
#pragma unroll
                for (int v = 0; v < RB; ++v) {
                    const int e = i0 + v * (int)blockDim.x;
                    if (e >= nitem) continue;
                    CT r[3], s[3], u[3];
                    if (e >= nwin) {  // u at a pair's vertex (zero where the pair has no vertex)
                        const int kk = (e - nwin) >> 2, q = (e - nwin) & 3;
                        if (av[v] >= 0) {
#pragma unroll
                            for (int j = 0; j < 3; ++j) {
                                if (upd) {
                                    s[j] = fma_rn(bt, so[v][j], w[v][j]);
                                    r[j] = fma_rn(-al, s[j], ro[v][j]);
                                } else {
                                    r[j] = ro[v][j];
                                }
                            }
                            prec3(P[v], r, u);
                        } else {
                            u[0] = u[1] = u[2] = CT(0);
                        }
#pragma unroll
                        for (int j = 0; j < 3; ++j) s_cu[12 * kk + 3 * q + j] = u[j];
                        continue;
                    }
                    const int j = e, a = wlo + j, i = a - r0;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (upd) {
                            s[q] = fma_rn(bt, s_sw[q * lw + j], w[v][q]);
                            r[q] = fma_rn(-al, s[q], s_rw[q * lw + j]);
                            s_sw[q * lw + j] = s[q];
                        } else {
                            r[q] = ro[v][q];
                        }
                        s_rw[q * lw + j] = r[q];
                    }
                    prec3(P[v], r, u);
                    if (i >= 0 && i < nr) {  // own row
                        if (upd) {
                            CT uo[3];
                            load3v(s_u4 + 4 * j, uo);  // u of iteration k - 1
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const CT p = fma_rn(bt, s_pd[q * ld + i], uo[q]);
                                s_pd[q * ld + i] = p;
                                if (mixed) s_xl[q * ld + i] += al * p;
                                else s_x[q * ld + i] += alpha * (double)p;
                                qcn[(size_t)q * nv + a] = 0.0;
                            }
                            if (A.nc > 0) {
                                if (mixed) {
                                    float4 *d = reinterpret_cast<float4 *>(rsc + 8 * (size_t)a);
                                    d[0] = make_float4((float)r[0], (float)r[1], (float)r[2], 0.f);
                                    d[1] = make_float4((float)s[0], (float)s[1], (float)s[2], 0.f);
                                } else {
#pragma unroll
                                    for (int q = 0; q < 3; ++q) {
                                        rsc[8 * (size_t)a + q] = r[q];
                                        rsc[8 * (size_t)a + 4 + q] = s[q];
                                    }
                                }
                            }
                        }
                        acc_add(acc[0], (r[0] * u[0] + r[1] * u[1]) + r[2] * u[2]);
                        acc_add(acc[2], (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]);
                    }
                    if (mixed) *reinterpret_cast<float4 *>(s_u4 + 4 * j) = make_float4((float)u[0], (float)u[1], (float)u[2], 0.f);
                    else
#pragma unroll
                        for (int q = 0; q < 3; ++q) s_u4[4 * j + q] = u[q];
                }
            }
        }
        __syncthreads();
        if (timer) tm[5] += globaltimer() - tm[4];
        // ---- product: w = H u on the own rows (published), contact part ------
        {
            // rows are taken in order of decreasing length: their sums go to
            // shared memory first and out to the planes in row order, so the
            // global stores are coalesced.  Warps without a row (fewer rows
            // than threads) take the contact pairs meanwhile; otherwise every
            // thread sums rows, then takes pairs.
            CT *wqc = wqb + 3 * nv * (size_t)(k & 1);
            double *qck = qcb + 3 * nv * (size_t)(k % 3);
            const int nrw = (nr + 31) & ~31;
            const bool split = nrw < (int)blockDim.x;
            const int c0 = split ? nrw : 0, cstep = split ? (int)blockDim.x - nrw : (int)blockDim.x;
            CT cdot = CT(0);
            if (!split || (int)threadIdx.x < nrw) {
                for (int t = threadIdx.x; t < nr; t += blockDim.x) {
                    const int info = s_rinfo[t];
                    const int row = info >> 8, len = info & 255;
                    CT y0 = CT(0), y1 = CT(0), y2 = CT(0);
#pragma unroll 4
                    for (int j = 0; j < len; ++j) {
                        const int slot = s_lvl[j] + t;
                        const MT *v = s_val + 9 * slot;
                        CT a[9], u[3];
#pragma unroll
                        for (int i = 0; i < 9; ++i) a[i] = (CT)v[i];
                        load3v(s_u4 + 4 * s_nbr[slot], u);
                        y0 += a[0] * u[0] + a[1] * u[1] + a[2] * u[2];
                        y1 += a[3] * u[0] + a[4] * u[1] + a[5] * u[2];
                        y2 += a[6] * u[0] + a[7] * u[1] + a[8] * u[2];
                    }
                    s_wq[row] = y0;
                    s_wq[ld + row] = y1;
                    s_wq[2 * ld + row] = y2;
                    CT ui[3];
                    load3v(s_u4 + 4 * (r0 + row - wlo), ui);
                    acc_add(acc[1], (ui[0] * y0 + ui[1] * y1) + ui[2] * y2);
                }
            }
            if (timer) tm[6] += globaltimer() - tm[4];
            if (threadIdx.x == blockDim.x - 1 && k > 0) {  // for the reduction below (read after its block sum)
                ctl.inv_gam_old = 1.0 / ctl.gam_old;
                ctl.c_old = ctl.inv_gam_old / (mixed ? (double)ctl.al : ctl.alpha);
            }
            if (!split || (int)threadIdx.x >= nrw) {
                for (int kk = (int)threadIdx.x - c0; kk < nco; kk += cstep) {
                    CT g[12], u[12], w;
                    int vid[4], m;
                    if (kk < ncached) {
                        const int4 v = s_cv[kk];
                        vid[0] = v.x; vid[1] = v.y; vid[2] = v.z; vid[3] = v.w;
                        m = s_cm[kk];
                        w = s_cw[kk];
#pragma unroll
                        for (int j = 0; j < 12; ++j) {
                            g[j] = s_cg[12 * kk + j];
                            u[j] = s_cu[12 * kk + j];
                        }
                    } else {  // beyond the cache: the same update at the pair's vertices
                        const int i = c + kk * (int)gridDim.x;
                        const int4 v = A.cv[i];
                        vid[0] = v.x; vid[1] = v.y; vid[2] = v.z; vid[3] = v.w;
                        m = A.cmask[i];
                        w = (CT)A.cw[i];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            CT uq[3] = {CT(0), CT(0), CT(0)};
                            if (m >> q & 1) {
                                const size_t a = (size_t)vid[q];
                                CT P[6], r[3];
                                load_p(a, P);
                                if (upd) {
                                    CT wv[3], ro[3], so[3];
                                    load_w(a, k - 1, true, wv);
                                    load_rs(a, k - 1, 0, ro);
                                    load_rs(a, k - 1, 4, so);
#pragma unroll
                                    for (int j = 0; j < 3; ++j) r[j] = fma_rn(-al, fma_rn(bt, so[j], wv[j]), ro[j]);
                                } else {
                                    load_rs(a, k, 0, r);
                                }
                                prec3(P, r, uq);
                            }
#pragma unroll
                            for (int j = 0; j < 3; ++j) {
                                g[3 * q + j] = (CT)A.cg[12 * (size_t)i + 3 * q + j];
                                u[3 * q + j] = uq[j];
                            }
                        }
                    }
                    CT s = CT(0);
#pragma unroll
                    for (int j = 0; j < 12; ++j) s += g[j] * u[j];
                    const CT t = w * s;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (m >> q & 1)
#pragma unroll
                            for (int j = 0; j < 3; ++j) atomicAdd(qck + (size_t)j * nv + vid[q], (double)(t * g[3 * q + j]));
                    cdot += t * s;
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nr; i += blockDim.x)
#pragma unroll
                for (int q = 0; q < 3; ++q) wqc[(size_t)q * nv + r0 + i] = s_wq[q * ld + i];
            acc_add(acc[1], cdot);
            if (timer) {
                tm[7] += globaltimer() - tm[4];
                const unsigned long long t1 = globaltimer();
                tm[0] += t1 - tm[4];
                tm[4] = t1;
            }
        }
        reduce(acc, [&](const double *t) {
            const double gam = t[0], del = t[1], rr = t[2];
            ctl.rr = rr;
            if (!finite_b(gam) || !finite_b(del) || !finite_b(rr)) {
                ctl.state = PCG_BAD;
                return;
            }
            const bool done = le_nonneg_b(rr, ctl.rr_done);  // rr, rr_done, rr_fold >= 0
            if (mixed && ctl.folds < A.max_replace && (done || le_nonneg_b(rr, ctl.rr_fold))) {
                ctl.state = PCG_FOLD;
                return;
            }
            if (done) {
                ctl.state = PCG_DONE;
                return;
            }
            if (ctl.it >= A.maxit) {
                ctl.state = PCG_MAXIT;
                return;
            }
            // p.Hp = delta - beta gamma / alpha_old = delta - gamma^2 / (gamma_old alpha_old)
            const double den = ctl.it > 0 ? fma(-(gam * gam), ctl.c_old, del) : del;
            if (!pos_b(den) || !pos_b(gam)) {  // no curvature left: stop with the current x
                ctl.state = PCG_DONE;
                return;
            }
            if (mixed) {
                // the FP32 updates use alpha and beta rounded to FP32: alpha
                // by an FP32 division of the FP64 quantities (short on this
                // GPU), carried as exactly that value in the recurrence
                ctl.al = div_to_f32(gam, den);
                ctl.bt = ctl.it > 0 ? __double2float_rn(gam * ctl.inv_gam_old) : 0.f;
            } else {
                ctl.alpha = gam / den;
                ctl.beta = ctl.it > 0 ? gam * ctl.inv_gam_old : 0.0;
            }
            ctl.gam_old = gam;
            ++ctl.it;
            ctl.skip = 0;
        });
        if (timer) tm[1] += globaltimer() - tm[4];
        if constexpr (mixed) {
        if (ctl.state == PCG_FOLD) {
            // reliable update: x += x_l in FP64; the contact part of this
            // iteration's product is dropped (the product is redone)
            double *qck = qcb + 3 * nv * (size_t)(k % 3);
            for (int i = threadIdx.x; i < nr; i += blockDim.x)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const double xv = s_x[q * ld + i] + (double)s_xl[q * ld + i];
                    s_x[q * ld + i] = xv;
                    s_xl[q * ld + i] = CT(0);
                    A.x[3 * (size_t)(r0 + i) + q] = xv;
                    qck[(size_t)q * nv + r0 + i] = 0.0;
                }
            {
                AccF none[1];
                reduce(none, [&](const double *) {});  // x visible to every CTA
            }
            if (ctl.state == PCG_ABORT) break;
            // H x with FP64 vectors (FP32 blocks): own full rows, then the
            // contact part into qd
            for (int t = threadIdx.x; t < nr; t += blockDim.x) {
                const int info = s_rinfo[t];
                const int row = info >> 8, len = info & 255;
                double h[3] = {0.0, 0.0, 0.0};
                for (int j = 0; j < len; ++j) {
                    const int slot = s_lvl[j] + t;
                    const MT *v = s_val + 9 * slot;
                    const size_t b = 3 * (size_t)(wlo + s_nbr[slot]);
                    double xj[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) xj[q] = __ldcg(A.x + b + q);
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        h[q] += (double)v[3 * q] * xj[0] + (double)v[3 * q + 1] * xj[1] + (double)v[3 * q + 2] * xj[2];
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) A.chx[3 * (size_t)(r0 + row) + q] = h[q];
            }
            for (int kk = threadIdx.x; kk < nco; kk += blockDim.x) {
                const int i = c + kk * (int)gridDim.x;
                const int4 v = A.cv[i];
                const int mk = A.cmask[i];
                const int vid[4] = {v.x, v.y, v.z, v.w};
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (mk >> q & 1)
#pragma unroll
                        for (int j = 0; j < 3; ++j) s += A.cg[12 * (size_t)i + 3 * q + j] * __ldcg(A.x + 3 * vid[q] + j);
                const double t = A.cw[i] * s;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (mk >> q & 1)
#pragma unroll
                        for (int j = 0; j < 3; ++j) atomicAdd(A.qd + 3 * vid[q] + j, t * A.cg[12 * (size_t)i + 3 * q + j]);
            }
            {
                AccF none[1];
                reduce(none, [&](const double *) {});  // contact part complete
            }
            if (ctl.state == PCG_ABORT) break;
            // r = b - H x, published for the redone product of iteration k
            CT *rsk = rsb + 8 * nv * (size_t)(k & 1);
            AccF acc1[1];
            for (int i = threadIdx.x; i < nr; i += blockDim.x) {
                const size_t a = (size_t)(r0 + i);
                double rr = 0.0;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const double rh = A.b[3 * a + q] - __ldcg(A.chx + 3 * a + q) - __ldcg(A.qd + 3 * a + q);
                    A.qd[3 * a + q] = 0.0;
                    rr += rh * rh;
                    rsk[8 * a + q] = to_ct(rh, CT());
                }
                acc1[0].add(rr);
            }
            reduce(acc1, [&](const double *t) {
                ++ctl.folds;
                ctl.rr = t[0];
                ctl.rr_fold = 0.01 * t[0];
                if (!finite_b(t[0])) ctl.state = PCG_BAD;
                else if (le_nonneg_b(t[0], ctl.rr_done)) ctl.state = PCG_DONE;
                else {
                    ctl.state = PCG_RUN;
                    ctl.skip = 1;
                }
            });
        }
        }
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < 3; ++q)
            A.x[3 * (size_t)(r0 + i) + q] = s_x[q * ld + i] + (mixed ? (double)s_xl[q * ld + i] : 0.0);
    // clear the pair flags (every CTA has copied its window's flags before
    // the first product, and none reads them after its last reduction)
    for (int kk = threadIdx.x; kk < nco; kk += blockDim.x) {
        const int i = c + kk * (int)gridDim.x;
        const int4 v = A.cv[i];
        const int m = A.cmask[i];
        if (m & 1) gfl[v.x] = 0;
        if (m & 2) gfl[v.y] = 0;
        if (m & 4) gfl[v.z] = 0;
        if (m & 8) gfl[v.w] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.dflag[F_ITERS] = ctl.it;
        A.dflag[F_MAXIT] = ctl.state == PCG_MAXIT;
        A.dflag[F_DONE] = 1;
        if (ctl.state == PCG_BAD) A.dflag[F_ERR] |= ERR_NONFINITE;
        A.dscal[S_RR] = ctl.rr;
        A.dscal[S_BB] = ctl.bb;
        A.dscal[S_RZ] = ctl.gam_old;
        A.dscal[S_T_SPMV] = 1e-6 * (double)tm[0];
        A.dscal[S_T_RED1] = 1e-6 * (double)tm[1];
        A.dscal[S_T_UPD] = 0.0;
        A.dscal[S_T_RED2] = 0.0;
        A.dscal[S_T_STAGE] = 1e-6 * (double)tm[5];
        A.dscal[S_T_ROWS] = 1e-6 * (double)tm[6];
        A.dscal[S_T_CONTACT] = 1e-6 * (double)tm[7];
    }
}

// ---------------------------------------------------------------------------
// Symmetric variant for systems whose rows do not fit in shared memory
// (mixed precision).  The matrix is symmetric (section 5.1 stores its upper
// triangle), so each upper block B_ij (i < j) is streamed once and used
// twice: B_ij p_j joins row i's sum in registers, and B_ij^T p_i goes to
// row j through a vector reduction (red.global.add.v4.f32) into the
// accumulation vector yq, which the owner of row j reads (and clears) after
// the grid-wide reduction that ends the product.  Each row's own sum and the
// contact terms add into yq the same way, so yq holds q = H p complete.  The
// product p.Hp needs no complete q: with D_i the diagonal blocks, p.Hp =
// sum_i p_i.D_i p_i + 2 sum_{i<j} p_i.B_ij p_j, which each row's thread
// forms from its own blocks.
//
// Per CTA: rows [part[c], part[c+1]) in order of decreasing upper length,
// taken in rounds of blockDim.x rows (one per thread); the blocks stream in
// the order they are consumed (round, then level; level 0 is the diagonal
// block) and each round is prefetched into L2 while the previous one is
// summed, the first during the reductions before the product; the window
// of p over [part[c], last upper neighbour] in shared memory (16-bit
// offsets); r and the FP32 increment of x per row in shared memory; z = P r
// as one float4 per vertex and P as six planes of its upper triangle in
// global memory; FP64 x and H x of the reliable updates in a per-CTA global
// vector (L2-resident).
// ---------------------------------------------------------------------------
struct PcgSymLayout {
    size_t p4, r, xl, rinfo, lvl, cg, cp, cw, cv, cm, total;
};

__host__ __device__ inline PcgSymLayout pcg_sym_layout(int max_rows, int max_win, int max_len, int kc)
{
    PcgSymLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    L.p4 = take(16 * (size_t)max_win);
    L.r = take(12 * (size_t)max_rows);
    L.xl = take(12 * (size_t)max_rows);
    L.rinfo = take(4 * (size_t)max_rows);
    L.lvl = take(8 * (size_t)max_len);  // chunk table: max_len = entries per CTA
    L.cg = take(48 * (size_t)kc);
    L.cp = take(48 * (size_t)kc);
    L.cw = take(4 * (size_t)kc);
    L.cv = take(16 * (size_t)kc);
    L.cm = take(4 * (size_t)kc);
    L.total = o;
    return L;
}

// per-CTA global vector of the symmetric variant: FP64 x and H x (3 per row each)
inline size_t pcg_sym_vec_bytes(int max_rows) { return ((48 * (size_t)max_rows) + 255) & ~(size_t)255; }

constexpr int kSymRowBatch = 2;  // rows per thread whose update-phase loads are issued together
constexpr int kSymStageBatch = 8;  // window vertices per thread whose staging loads are issued together
constexpr int kSymPrefetchBytes = 32768;  // bytes per bulk L2 prefetch instruction

// bulk prefetch of [p, p + bytes) into L2 (16-byte aligned, a multiple of
// 16 bytes; a hint: nothing waits for it)
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void red_add4(float4 *dst, float a, float b, float c)
{
    atomicAdd(dst, make_float4(a, b, c, 0.f));  // vector reduction at L2 (sm_90+)
}

__global__ void __launch_bounds__(kPcgThreads, 1) k_pcg_sym(PcgArgs A)
{
    using CT = float;
    using VT = float;
    using RT = float;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PcgCtl ctl;
    __shared__ float2 red_f[2 * kPcgMaxWarps];
    const float *__restrict__ gpinv = (const float *)A.pinv;
    float4 *__restrict__ z4 = A.z4;  // z = P r, one float4 per vertex (one vector load each in the staging)
    VT *pb[2] = {(VT *)A.p0, (VT *)A.p1};
    float4 *__restrict__ yq = A.yq;
    const unsigned char *__restrict__ ub = (const unsigned char *)A.uval;
    const int c = blockIdx.x;
    const int r0 = A.part[c], r1 = A.part[c + 1], nr = r1 - r0;
    const int wlo = A.win[2 * c], whi = A.win[2 * c + 1], nwin = whi - wlo;  // wlo == r0
    const int ntab = A.lvlptr[c + 1] - A.lvlptr[c];  // chunk-table entries
    const int rounds = (nr + (int)blockDim.x - 1) / (int)blockDim.x;
    const int lm = rounds > 0 ? (ntab - 1) / rounds : 0;  // levels per round
    const int nco = A.nc > c ? (A.nc - c + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const int ncached = min(nco, A.kc);
    const PcgSymLayout L = pcg_sym_layout(A.max_rows, A.max_win, A.max_len, A.kc);
    const int ld = A.max_rows;  // per-row arrays are component-major: a[k * ld + row]
    double *g_x = (double *)(A.gvec + (size_t)c * A.gvec_stride);
    double *g_hx = g_x + 3 * (size_t)ld;
    CT *s_p4 = (CT *)(smem + L.p4);
    RT *s_r = (RT *)(smem + L.r);
    RT *s_xl = (RT *)(smem + L.xl);
    int *s_rinfo = (int *)(smem + L.rinfo);
    int2 *s_tab = (int2 *)(smem + L.lvl);
    CT *s_cg = (CT *)(smem + L.cg);
    CT *s_cp = (CT *)(smem + L.cp);
    CT *s_cw = (CT *)(smem + L.cw);
    int4 *s_cv = (int4 *)(smem + L.cv);
    int *s_cm = (int *)(smem + L.cm);
    for (int j = threadIdx.x; j < ntab; j += blockDim.x) s_tab[j] = ((const int2 *)A.lvl)[A.lvlptr[c] + j];
    // round q of the CTA's blocks: bytes [tab[q lm], tab[(q + 1) lm]); the
    // first round goes to L2 now, each later one while the previous is used
    auto prefetch_round = [&](int q) {
        if (q < rounds) {
            const int b0 = ((const int2 *)A.lvl)[A.lvlptr[c] + q * lm].x;
            const int b1 = ((const int2 *)A.lvl)[A.lvlptr[c] + (q + 1) * lm].x;
            for (int o = b0; o < b1; o += kSymPrefetchBytes)
                prefetch_l2(ub + o, (unsigned)min(kSymPrefetchBytes, b1 - o));
        }
    };
    if (threadIdx.x == 0) prefetch_round(0);
    for (int t = threadIdx.x; t < nr; t += blockDim.x) s_rinfo[t] = A.rinfo[r0 + t];
    for (int k = threadIdx.x; k < ncached; k += blockDim.x) {
        const int i = c + k * (int)gridDim.x;
        s_cv[k] = A.cv[i];
        s_cm[k] = A.cmask[i];
        s_cw[k] = (CT)A.cw[i];
#pragma unroll
        for (int j = 0; j < 12; ++j) s_cg[12 * k + j] = (CT)A.cg[12 * (size_t)i + j];
    }
    for (int i = threadIdx.x; i < 4 * nwin; i += blockDim.x) s_p4[i] = CT(0);  // p_old = 0
    // P of the own rows as six planes of its upper triangle (P inverts a
    // symmetric block): the update phase then loads them coalesced, six
    // words per row instead of nine at a 36-byte stride
    const size_t nvs = (size_t)A.nv;
    float *const ppl = (float *)A.cpp;
    for (int e = threadIdx.x; e < 6 * nr; e += blockDim.x) {
        const int i = e / nr, row = e - i * nr;
        const size_t a = (size_t)(r0 + row);
        ppl[(size_t)i * nvs + a] = gpinv[9 * a + upper3(i)];
    }
    // z = P r of a row from its upper-triangle entries (p00 p01 p02 p11 p12 p22)
    auto apply_p = [&](const float (&P)[6], const RT *rv, CT (&zc)[3]) {
        zc[0] = P[0] * rv[0] + P[1] * rv[1] + P[2] * rv[2];
        zc[1] = P[1] * rv[0] + P[3] * rv[1] + P[4] * rv[2];
        zc[2] = P[2] * rv[0] + P[4] * rv[1] + P[5] * rv[2];
    };
    // z = P r for local row `row` (written to global memory); returns r.z
    auto precond = [&](int row, const RT *rv) -> CT {
        const size_t a = (size_t)(r0 + row);
        float P[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) P[i] = __ldcg(ppl + (size_t)i * nvs + a);
        CT zc[3];
        apply_p(P, rv, zc);
        z4[a] = make_float4(zc[0], zc[1], zc[2], 0.f);
        return (rv[0] * zc[0] + rv[1] * zc[1]) + rv[2] * zc[2];
    };
    unsigned nred = 0;
    auto reduce = [&](auto &acc, auto on_total) {
        constexpr int K = (int)std::extent<std::remove_reference_t<decltype(acc)>>::value;
        double blk[K], tot[K];
        block_sum<K>(acc, blk, red_f);
        if (threadIdx.x == 0) {
            if (grid_total<K>(blk, A.res, nred, A.bar, A.bar_poll, A.dflag, tot)) on_total(tot);
            else ctl.state = PCG_ABORT;
        }
        ++nred;
        __syncthreads();
    };
    // per-phase device time seen by thread 0 of CTA 0 (kept in shared
    // memory: 64-bit counters in registers would cost the hot loops 16)
    __shared__ unsigned long long tm[8];  // A, A2, B, B2, t0, S, R, C
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < 8; ++i) tm[i] = 0;
    __syncthreads();
    // ---- init: r = b, x = 0, z = P r, p_old = 0, yq = 0 on the own rows ----
    {
        AccF acc[2] = {};
        for (int i = threadIdx.x; i < nr; i += blockDim.x) {
            const int a = r0 + i;
            RT rv[3];
            double bb = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double bk = A.b[3 * a + k];
                rv[k] = (RT)bk;
                s_r[k * ld + i] = rv[k];
                s_xl[k * ld + i] = RT(0);
                g_x[k * ld + i] = 0.0;
                A.qd[3 * a + k] = 0.0;
                if (A.nc > 0) pb[0][3 * a + k] = VT(0);
                bb += bk * bk;
            }
            yq[a] = make_float4(0.f, 0.f, 0.f, 0.f);
            acc[0].add(precond(i, rv));
            acc[1].add(bb);
        }
        reduce(acc, [&](const double *t) {
            ctl.rz = t[0];
            ctl.bb = t[1];
            ctl.rr = t[1];
            ctl.rr_done = A.tol2 * t[1];
            ctl.rr_fold = 0.01 * t[1];
            ctl.beta = 0.0;
            ctl.bt = 0.f;
            ctl.it = 0;
            ctl.folds = 0;
            if (pos_b(t[1]) && finite_b(t[0]) && finite_b(t[1])) ctl.state = PCG_RUN;
            else ctl.state = t[1] == 0.0 ? PCG_DONE : PCG_BAD;
        });
    }
    int parity = 0;
    while (ctl.state == PCG_RUN) {
        VT *pold = pb[parity], *pnew = pb[parity ^ 1];
        // ---- phase A: p = z + beta p over the window, row sums, transposes ---
        {
            if (timer) tm[4] = globaltimer();
            const CT bt = (CT)ctl.bt;
            {
                // items: the window's vertices (z as one vector load each),
                // then the components of the cached pairs' vertices
                const int ncf = 12 * ncached, ntot = nwin + ncf;
                const float *zs = (const float *)z4;
                for (int f0 = threadIdx.x; f0 < ntot; f0 += kSymStageBatch * blockDim.x) {
                    float4 zz[kSymStageBatch];
                    VT pp[kSymStageBatch];
#pragma unroll
                    for (int k = 0; k < kSymStageBatch; ++k) {
                        const int f = f0 + k * blockDim.x;
                        zz[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                        pp[k] = VT(0);
                        if (f < nwin) {
                            zz[k] = __ldcg(z4 + wlo + f);
                        } else if (f < ntot) {
                            const int g = f - nwin, kk = g / 12, q = (g % 12) / 3, j = g % 3;
                            if (s_cm[kk] >> q & 1) {
                                const int v = (&s_cv[kk].x)[q];
                                zz[k].x = __ldcg(zs + 4 * (size_t)v + j);
                                pp[k] = __ldcg(pold + 3 * v + j);
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kSymStageBatch; ++k) {
                        const int f = f0 + k * blockDim.x;
                        if (f < nwin) {
                            float4 *d = reinterpret_cast<float4 *>(s_p4 + 4 * f);
                            float4 pv = *d;
                            pv.x = dir_update(zz[k].x, bt, pv.x);
                            pv.y = dir_update(zz[k].y, bt, pv.y);
                            pv.z = dir_update(zz[k].z, bt, pv.z);
                            *d = pv;
                        } else if (f < ntot) {
                            s_cp[f - nwin] = dir_update(zz[k].x, bt, pp[k]);
                        }
                    }
                }
            }
            __syncthreads();
            if (timer) tm[5] += globaltimer() - tm[4];
            // Row sums in batches of four levels: the loads of a batch are
            // issued together, before its products and vector reductions (a
            // reduction keeps the loads that follow it behind it).
            AccF acc[1] = {};
            for (int q = 0; q < rounds; ++q) {
                if (threadIdx.x == 0) prefetch_round(q + 1);
                const int u = threadIdx.x, t = q * (int)blockDim.x + u;
                if (t >= nr) continue;
                const int info = s_rinfo[t];
                const int row = info >> 8, len = info & 255;
                const int2 *tq = s_tab + q * lm;
                CT pi[3];
                load3v(s_p4 + 4 * row, pi);
                CT yd[3] = {0.f, 0.f, 0.f}, yo[3] = {0.f, 0.f, 0.f};
                for (int j0 = 0; j0 < len; j0 += 4) {
                    CT a[4][9];
                    int vr[4];
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        vr[w] = -1;
                        if (j0 + w < len) {
                            const int2 e = tq[j0 + w];  // chunk of level j0 + w: offset, padded row count
                            const float *pl = (const float *)(ub + e.x) + u;
#pragma unroll
                            for (int i = 0; i < 9; ++i) a[w][i] = __ldcs(pl + (size_t)i * e.y);
                            // level 0: the row itself (diagonal block)
                            vr[w] = __ldcs((const unsigned short *)(ub + e.x + 36 * (size_t)e.y) + u);
                        }
                    }
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        if (vr[w] >= 0) {
                            CT pj[3];
                            load3v(s_p4 + 4 * vr[w], pj);
                            const CT s0 = a[w][0] * pj[0] + a[w][1] * pj[1] + a[w][2] * pj[2];
                            const CT s1 = a[w][3] * pj[0] + a[w][4] * pj[1] + a[w][5] * pj[2];
                            const CT s2 = a[w][6] * pj[0] + a[w][7] * pj[1] + a[w][8] * pj[2];
                            if (j0 + w == 0) {
                                yd[0] = s0; yd[1] = s1; yd[2] = s2;
                            } else {
                                yo[0] += s0; yo[1] += s1; yo[2] += s2;
                                red_add4(yq + wlo + vr[w], a[w][0] * pi[0] + a[w][3] * pi[1] + a[w][6] * pi[2],
                                         a[w][1] * pi[0] + a[w][4] * pi[1] + a[w][7] * pi[2],
                                         a[w][2] * pi[0] + a[w][5] * pi[1] + a[w][8] * pi[2]);
                            }
                        }
                    }
                }
                red_add4(yq + r0 + row, yd[0] + yo[0], yd[1] + yo[1], yd[2] + yo[2]);  // q complete in yq
                acc[0].add((pi[0] * yd[0] + pi[1] * yd[1]) + pi[2] * yd[2]);
                acc[0].add(2.f * ((pi[0] * yo[0] + pi[1] * yo[1]) + pi[2] * yo[2]));
            }
            if (threadIdx.x == 0) prefetch_round(0);  // the next product's first round, during the reductions
            if (timer) tm[6] += globaltimer() - tm[4];
            // this CTA's contact pairs: yq += mu gamma g (g . p)
            CT cdot = CT(0);
            for (int k = threadIdx.x; k < nco; k += blockDim.x) {
                CT g[12], u[12], w;
                int vid[4], m;
                if (k < ncached) {
                    const int4 v = s_cv[k];
                    vid[0] = v.x; vid[1] = v.y; vid[2] = v.z; vid[3] = v.w;
                    m = s_cm[k];
                    w = s_cw[k];
#pragma unroll
                    for (int j = 0; j < 12; ++j) {
                        g[j] = s_cg[12 * k + j];
                        u[j] = s_cp[12 * k + j];
                    }
                } else {
                    const int i = c + k * (int)gridDim.x;
                    const int4 v = A.cv[i];
                    vid[0] = v.x; vid[1] = v.y; vid[2] = v.z; vid[3] = v.w;
                    m = A.cmask[i];
                    w = (CT)A.cw[i];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            g[3 * q + j] = (CT)A.cg[12 * (size_t)i + 3 * q + j];
                            u[3 * q + j] = (m >> q & 1) ? dir_update(__ldcg((const float *)z4 + 4 * (size_t)vid[q] + j), bt,
                                                                     __ldcg(pold + 3 * vid[q] + j))
                                                        : CT(0);
                        }
                }
                CT s = CT(0);
#pragma unroll
                for (int j = 0; j < 12; ++j) s += g[j] * u[j];
                const CT t = w * s;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (m >> q & 1) red_add4(yq + vid[q], t * g[3 * q], t * g[3 * q + 1], t * g[3 * q + 2]);
                cdot += t * s;
            }
            if (timer) tm[7] += globaltimer() - tm[4];
            acc[0].add(cdot);
            if (A.nc > 0)
                for (int i = threadIdx.x; i < nr; i += blockDim.x) {  // read by other CTAs' pairs
                    CT p[3];
                    load3v(s_p4 + 4 * i, p);
#pragma unroll
                    for (int k = 0; k < 3; ++k) pnew[3 * (r0 + i) + k] = p[k];
                }
            if (timer) {
                const unsigned long long t1 = globaltimer();
                tm[0] += t1 - tm[4];
                tm[4] = t1;
            }
            reduce(acc, [&](const double *t) {
                const double pq = t[0];
                if (!finite_b(pq)) ctl.state = PCG_BAD;
                else if (!pos_b(pq)) ctl.state = PCG_DONE;
                else {
                    ctl.al = div_to_f32(ctl.rz, pq);
                    ctl.alpha = (double)ctl.al;
                }
            });
            if (timer) {
                const unsigned long long t1 = globaltimer();
                tm[1] += t1 - tm[4];
                tm[4] = t1;
            }
        }
        if (ctl.state != PCG_RUN) break;
        // ---- phase B: x, r, z updates ---------------------------------------
        {
            const RT al = ctl.al;
            AccF acc[2] = {};
            // kSymRowBatch rows per thread at a time, their global loads issued together
            for (int row0 = threadIdx.x; row0 < nr; row0 += kSymRowBatch * blockDim.x) {
                float4 yg[kSymRowBatch];
                float P[kSymRowBatch][6];
#pragma unroll
                for (int u = 0; u < kSymRowBatch; ++u) {
                    const int row = row0 + u * blockDim.x;
                    if (row < nr) {
                        const int a = r0 + row;
                        yg[u] = __ldcg(yq + a);

#pragma unroll
                        for (int i = 0; i < 6; ++i) P[u][i] = __ldcg(ppl + (size_t)i * nvs + a);
                    }
                }
#pragma unroll
                for (int u = 0; u < kSymRowBatch; ++u) {
                    const int row = row0 + u * blockDim.x;
                    if (row < nr) {
                        const int a = r0 + row;
                        yq[a] = make_float4(0.f, 0.f, 0.f, 0.f);
                        CT pc[3];
                        load3v(s_p4 + 4 * row, pc);
                        const float qk[3] = {yg[u].x, yg[u].y, yg[u].z};
                        RT rv[3];
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            s_xl[k * ld + row] += al * pc[k];
                            rv[k] = s_r[k * ld + row] - al * qk[k];
                            s_r[k * ld + row] = rv[k];
                        }
                        CT zc[3];
                        apply_p(P[u], rv, zc);
                        z4[a] = make_float4(zc[0], zc[1], zc[2], 0.f);
                        acc[0].add((rv[0] * zc[0] + rv[1] * zc[1]) + rv[2] * zc[2]);
                        acc[1].add((rv[0] * rv[0] + rv[1] * rv[1]) + rv[2] * rv[2]);
                    }
                }
            }
            if (timer) {
                const unsigned long long t1 = globaltimer();
                tm[2] += t1 - tm[4];
                tm[4] = t1;
            }
            reduce(acc, [&](const double *t) {
                ++ctl.it;
                ctl.rz_old = ctl.rz;
                ctl.bt = div_to_f32(t[0], ctl.rz_old);
                ctl.beta = (double)ctl.bt;
                ctl.rz = t[0];
                ctl.rr = t[1];
                if (!finite_b(t[0]) || !finite_b(t[1])) {
                    ctl.state = PCG_BAD;
                    return;
                }
                const bool done = le_nonneg_b(ctl.rr, ctl.rr_done);  // rr, rr_done, rr_fold >= 0
                if (ctl.folds < A.max_replace && (done || le_nonneg_b(ctl.rr, ctl.rr_fold))) ctl.state = PCG_FOLD;
                else if (done) ctl.state = PCG_DONE;
                else if (ctl.it >= A.maxit) ctl.state = PCG_MAXIT;
            });
            if (timer) tm[3] += globaltimer() - tm[4];
        }
        parity ^= 1;
        if (ctl.state == PCG_FOLD) {
            // reliable update: x += x_l in FP64, then r = b - H x with FP64
            // vectors (FP32 matrix, the transposed products by FP64 atomics
            // into qd); the direction p is kept and beta rescaled
            for (int i = threadIdx.x; i < nr; i += blockDim.x)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double xv = g_x[k * ld + i] + (double)s_xl[k * ld + i];
                    g_x[k * ld + i] = xv;
                    s_xl[k * ld + i] = RT(0);
                    A.x[3 * (r0 + i) + k] = xv;
                }
            {
                AccF none[1];
                reduce(none, [&](const double *) {});  // x visible to every CTA
            }
            if (ctl.state == PCG_ABORT) break;
            for (int t = threadIdx.x; t < nr; t += blockDim.x) {
                const int info = s_rinfo[t];
                const int row = info >> 8, len = info & 255;
                const int q = t / (int)blockDim.x, u = t - q * (int)blockDim.x;
                double xi[3], h[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int k = 0; k < 3; ++k) xi[k] = __ldcg(A.x + 3 * (r0 + row) + k);
                for (int j = 0; j < len; ++j) {
                    const int2 e = s_tab[q * lm + j];
                    const float *pl = (const float *)(ub + e.x) + u;
                    double a[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) a[i] = (double)__ldcs(pl + (size_t)i * e.y);
                    const int vr = j == 0 ? row : (int)__ldcs((const unsigned short *)(ub + e.x + 36 * (size_t)e.y) + u);
                    double xj[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) xj[k] = __ldcg(A.x + 3 * (wlo + vr) + k);
#pragma unroll
                    for (int k = 0; k < 3; ++k) h[k] += a[3 * k] * xj[0] + a[3 * k + 1] * xj[1] + a[3 * k + 2] * xj[2];
                    if (j > 0)
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            atomicAdd(A.qd + 3 * (wlo + vr) + k, a[k] * xi[0] + a[3 + k] * xi[1] + a[6 + k] * xi[2]);
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) g_hx[k * ld + row] = h[k];
            }
            for (int k = threadIdx.x; k < nco; k += blockDim.x) {
                const int i = c + k * (int)gridDim.x;
                const int4 v = A.cv[i];
                const int mk = A.cmask[i];
                const int vid[4] = {v.x, v.y, v.z, v.w};
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (mk >> q & 1)
#pragma unroll
                        for (int j = 0; j < 3; ++j) s += A.cg[12 * (size_t)i + 3 * q + j] * __ldcg(A.x + 3 * vid[q] + j);
                const double t = A.cw[i] * s;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (mk >> q & 1)
#pragma unroll
                        for (int j = 0; j < 3; ++j) atomicAdd(A.qd + 3 * vid[q] + j, t * A.cg[12 * (size_t)i + 3 * q + j]);
            }
            {
                AccF none[1];
                reduce(none, [&](const double *) {});  // transposed and contact parts complete
            }
            if (ctl.state == PCG_ABORT) break;
            AccF acc[2];
            for (int i = threadIdx.x; i < nr; i += blockDim.x) {
                const int a = r0 + i;
                RT rv[3];
                double rr = 0.0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double rh = A.b[3 * a + k] - g_hx[k * ld + i] - __ldcg(A.qd + 3 * a + k);
                    A.qd[3 * a + k] = 0.0;
                    rr += rh * rh;
                    rv[k] = (RT)rh;
                    s_r[k * ld + i] = rv[k];
                }
                acc[0].add(precond(i, rv));
                acc[1].add(rr);
            }
            reduce(acc, [&](const double *t) {
                ++ctl.folds;
                ctl.bt = div_to_f32(t[0], ctl.rz_old);
                ctl.beta = (double)ctl.bt;
                ctl.rz = t[0];
                ctl.rr = t[1];
                ctl.rr_fold = 0.01 * t[1];
                if (!finite_b(t[0]) || !finite_b(t[1])) ctl.state = PCG_BAD;
                else if (le_nonneg_b(ctl.rr, ctl.rr_done)) ctl.state = PCG_DONE;
                else if (ctl.it >= A.maxit) ctl.state = PCG_MAXIT;
                else ctl.state = PCG_RUN;
            });
        }
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < 3; ++k) A.x[3 * (r0 + i) + k] = g_x[k * ld + i] + (double)s_xl[k * ld + i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.dflag[F_ITERS] = ctl.it;
        A.dflag[F_MAXIT] = ctl.state == PCG_MAXIT;
        A.dflag[F_DONE] = 1;
        if (ctl.state == PCG_BAD) A.dflag[F_ERR] |= ERR_NONFINITE;
        A.dscal[S_RR] = ctl.rr;
        A.dscal[S_BB] = ctl.bb;
        A.dscal[S_RZ] = ctl.rz;
        A.dscal[S_T_SPMV] = 1e-6 * (double)tm[0];
        A.dscal[S_T_RED1] = 1e-6 * (double)tm[1];
        A.dscal[S_T_UPD] = 1e-6 * (double)tm[2];
        A.dscal[S_T_RED2] = 1e-6 * (double)tm[3];
        A.dscal[S_T_STAGE] = 1e-6 * (double)tm[5];
        A.dscal[S_T_ROWS] = 1e-6 * (double)tm[6];
        A.dscal[S_T_CONTACT] = 1e-6 * (double)tm[7];
    }
}

// Row ranges of the CTAs (about equal block counts), each CTA's vertex
// window (its rows and all their neighbours), and the jagged shared-memory
// layout of each CTA's blocks: rows in order of decreasing length (ties by
// row), level j holding the j-th block of every row longer than j, so the
// j-th block of the t-th row sits at slot lvl[j] + t.
static int make_partition(Scene &S, int grid, int *max_rows, int *max_ent, int *max_win, int *max_len)
{
    const std::vector<int> &fr = S.h_frowptr;
    const std::vector<int> &fn = S.h_fnbr;
    std::vector<int> part(grid + 1, S.nv);
    part[0] = 0;
    const double per = (double)S.nfull / grid;
    int r = 0;
    for (int c = 1; c < grid; ++c) {
        const double target = per * c;
        while (r < S.nv && fr[r] < target) ++r;
        part[c] = std::max(part[c - 1], r);
    }
    part[grid] = S.nv;
    std::vector<int> win(2 * grid), rinfo(S.nv), lvl, lvlptr(grid + 1, 0);
    std::vector<unsigned short> eslot(S.nfull), jnbr(S.nfull);
    std::vector<int> edst(S.nfull);
    int mr = 0, me = 0, mw = 0, ml = 0;
    std::vector<int> order;
    for (int c = 0; c < grid; ++c) {
        const int a = part[c], b = part[c + 1];
        if (b - a > 65535 || fr[b] - fr[a] > 65535) return BF_E_CAPACITY;
        int lo = a, hi = b;
        for (int v = a; v < b; ++v)
            for (int e = fr[v]; e < fr[v + 1]; ++e) {
                lo = std::min(lo, fn[e]);
                hi = std::max(hi, fn[e] + 1);
            }
        if (hi - lo > 65535) return BF_E_CAPACITY;
        win[2 * c] = lo;
        win[2 * c + 1] = hi;
        order.resize(b - a);
        for (int v = a; v < b; ++v) order[v - a] = v;
        auto len = [&](int v) { return fr[v + 1] - fr[v]; };
        std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return len(u) > len(v); });
        const int lmax = b > a ? len(order[0]) : 0;
        if (lmax > 255) return BF_E_CAPACITY;
        std::vector<int> at(lmax + 1, 0);  // level offsets
        for (int j = 0; j < lmax; ++j) {
            int n = 0;
            while (n < b - a && len(order[n]) > j) ++n;
            at[j + 1] = at[j] + n;
        }
        for (int t = 0; t < b - a; ++t) {
            const int v = order[t];
            rinfo[a + t] = (v - a) << 8 | len(v);
            for (int j = 0; j < len(v); ++j) {
                const int fe = fr[v] + j, slot = at[j] + t;
                eslot[fe] = (unsigned short)slot;
                edst[fe] = fr[a] + slot;  // jagged position in global memory
                jnbr[fr[a] + slot] = (unsigned short)(fn[fe] - lo);
            }
        }
        lvl.insert(lvl.end(), at.begin(), at.end());
        lvlptr[c + 1] = (int)lvl.size();
        mr = std::max(mr, b - a);
        me = std::max(me, fr[b] - fr[a]);
        mw = std::max(mw, hi - lo);
        ml = std::max(ml, lmax);
    }
    auto put = [&](auto *&dst, const auto &host) -> int {
        using T = std::remove_reference_t<decltype(*dst)>;
        if (dst) dev_free(S, dst);
        dst = (T *)dev_alloc(S, std::max<size_t>(host.size(), 1) * sizeof(T));
        if (!dst) return BF_E_OOM;
        if (!host.empty())
            cudaMemcpyAsync(dst, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, S.stream);
        return BF_OK;
    };
    int st = put(S.part, part);
    if (!st) st = put(S.win, win);
    if (!st) st = put(S.pcg_eslot, eslot);
    if (!st) st = put(S.pcg_rinfo, rinfo);
    if (!st) st = put(S.pcg_lvl, lvl);
    if (!st) st = put(S.pcg_lvlptr, lvlptr);
    if (!st) st = put(S.pcg_edst, edst);
    if (!st) st = put(S.pcg_jnbr, jnbr);
    if (st) return st;
    *max_rows = mr;
    *max_ent = me;
    *max_win = mw;
    *max_len = ml;
    return check_cuda(cudaStreamSynchronize(S.stream));
}

// Partition of the symmetric variant: row ranges of equal length; each
// CTA's window runs from its first row to its last upper neighbour.  A
// CTA's rows are ordered by decreasing upper length (ties by row) and
// taken in rounds of `block` rows, thread t of the CTA owning row
// r * block + t of that order in round r.  The upper blocks are stored in
// the order the CTA consumes them: round by round, and within a round level
// by level (level 0 is every row's diagonal block, first in its upper row;
// level j the j-th upper block of the rows longer than j, a prefix of the
// round), each (round, level) chunk as 9 planes of FP32 values followed by
// the 16-bit window offsets of the neighbours, its row count padded to 32
// and its start aligned to 128 bytes.  A CTA's chunks are contiguous, so a
// round can be prefetched into L2 as one range.  The chunk table of CTA c
// (byte offset and padded count per round and level, then the end of its
// last round) starts at entry tabptr[c].
static int make_partition_sym(Scene &S, int grid, int block, int *max_rows, int *max_win, int *max_len,
                              int *max_tab, size_t *bytes)
{
    const std::vector<int> &rp = S.h_rowptr;
    const std::vector<int> &col = S.h_col;
    std::vector<int> part(grid + 1, S.nv);
    part[0] = 0;
    // equal row counts: a thread's work is the sum of its rows' lengths over
    // the rounds, so equal rounds per CTA balance the CTAs (balancing block
    // counts gave a few CTAs 7 or 8 rounds of short rows against 6: 48.2 ->
    // 43.6 us per iteration on the spiky-ball system)
    for (int c = 1; c < grid; ++c) part[c] = (int)((long long)S.nv * c / grid);
    part[grid] = S.nv;
    std::vector<int> win(2 * grid), rinfo(S.nv), tab, tabptr(grid + 1, 0), uedst(2 * (size_t)S.nnzb);
    std::vector<unsigned short> unbr(S.nnzb);
    int mr = 0, mw = 0, ml = 0, mt = 0;
    size_t off = 0;
    std::vector<int> order;
    for (int c = 0; c < grid; ++c) {
        const int a = part[c], b = part[c + 1], nr = b - a;
        int hi = b;
        for (int v = a; v < b; ++v) {
            if (rp[v + 1] == rp[v] || col[rp[v]] != v) return BF_E_CAPACITY;  // diagonal block first
            hi = std::max(hi, col[rp[v + 1] - 1] + 1);
        }
        if (hi - a > 65535) return BF_E_CAPACITY;
        win[2 * c] = a;
        win[2 * c + 1] = hi;
        order.resize(nr);
        for (int v = a; v < b; ++v) order[v - a] = v;
        auto len = [&](int v) { return rp[v + 1] - rp[v]; };
        std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return len(u) > len(v); });
        const int lmax = nr > 0 ? len(order[0]) : 0;
        if (lmax > 255) return BF_E_CAPACITY;
        const int rounds = cdiv(nr, block);
        const size_t tab0 = tab.size();
        tab.resize(tab0 + 2 * ((size_t)rounds * lmax + 1));
        for (int q = 0; q < rounds; ++q) {
            const int t0 = q * block, t1 = std::min(nr, t0 + block);
            for (int j = 0; j < lmax; ++j) {
                int n = 0;
                while (t0 + n < t1 && len(order[t0 + n]) > j) ++n;
                const int np = (n + 31) & ~31;
                off = (off + 127) & ~(size_t)127;
                if (off + 38 * (size_t)np > 0x7fffffffu) return BF_E_CAPACITY;
                tab[tab0 + 2 * ((size_t)q * lmax + j)] = (int)off;
                tab[tab0 + 2 * ((size_t)q * lmax + j) + 1] = np;
                for (int u = 0; u < n; ++u) {
                    const int v = order[t0 + u], k = rp[v] + j;
                    uedst[2 * (size_t)k] = (int)off;
                    uedst[2 * (size_t)k + 1] = np << 16 | u;
                    unbr[k] = (unsigned short)(col[k] - a);
                }
                off += 38 * (size_t)np;
            }
        }
        off = (off + 127) & ~(size_t)127;
        tab[tab.size() - 2] = (int)off;  // end of the CTA's last round
        tab[tab.size() - 1] = 0;
        tabptr[c + 1] = (int)(tab.size() / 2);
        for (int t = 0; t < nr; ++t) rinfo[a + t] = (order[t] - a) << 8 | len(order[t]);
        mr = std::max(mr, nr);
        mw = std::max(mw, hi - a);
        ml = std::max(ml, lmax);
        mt = std::max(mt, rounds * lmax + 1);
    }
    auto put = [&](auto *&dst, const auto &host) -> int {
        using T = std::remove_reference_t<decltype(*dst)>;
        if (dst) dev_free(S, dst);
        dst = (T *)dev_alloc(S, std::max<size_t>(host.size(), 1) * sizeof(T));
        if (!dst) return BF_E_OOM;
        if (!host.empty())
            cudaMemcpyAsync(dst, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, S.stream);
        return BF_OK;
    };
    int st = put(S.part, part);
    if (!st) st = put(S.win, win);
    if (!st) st = put(S.pcg_rinfo, rinfo);
    if (!st) st = put(S.pcg_lvl, tab);
    if (!st) st = put(S.pcg_lvlptr, tabptr);
    if (!st) st = put(S.pcg_uedst, uedst);
    if (!st) st = put(S.pcg_unbr, unbr);
    if (st) return st;
    *max_rows = mr;
    *max_win = mw;
    *max_len = ml;
    *max_tab = mt;
    *bytes = off;
    return check_cuda(cudaStreamSynchronize(S.stream));
}

// symmetric variant: the upper blocks (9 FP32 planes) and their neighbour
// offsets into the chunks of the consumption order
__global__ void k_jagged_gather_upper(int nnzb, const int2 *__restrict__ uedst, const unsigned short *__restrict__ unbr,
                                      const float *__restrict__ val, unsigned char *__restrict__ ubuf)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnzb) return;
    const int2 e = uedst[k];
    const int np = e.y >> 16, u = e.y & 0xffff;
    float *pl = (float *)(ubuf + e.x) + u;
#pragma unroll
    for (int i = 0; i < 9; ++i) pl[(size_t)i * np] = val[9 * (size_t)k + i];
    ((unsigned short *)(ubuf + e.x + 36 * (size_t)np))[u] = unbr[k];
}

// Sets up the symmetric variant at `cps` CTAs per SM, if it fits.
static int setup_sym(Scene &S, int nsm, int cps, size_t smem_optin)
{
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_pcg_sym) != cudaSuccess) return BF_E_CUDA;
    const int grid = std::max(1, std::min(nsm * cps, cdiv(S.nnzb, kPcgEntriesPerCta / 2)));
    if (grid > kPcgMaxGrid) return BF_E_CAPACITY;
    const int block = (kPcgThreads / cps) & ~31;
    int mr = 0, mw = 0, ml = 0, mt = 0;
    size_t ubytes = 0;
    int st = make_partition_sym(S, grid, block, &mr, &mw, &ml, &mt, &ubytes);
    if (st) return st;
    const size_t avail = smem_optin - fa.sharedSizeBytes;
    const PcgSymLayout L0 = pcg_sym_layout(mr, mw, mt, 0);
    if (L0.total > avail) return BF_E_CAPACITY;
    int kc = S.pcg_no_cache ? 0 : (int)std::min<size_t>(kPcgMaxCached, (avail - L0.total) / pcg_contact_bytes(4));
    while (kc > 0 && pcg_sym_layout(mr, mw, mt, kc).total > avail) --kc;
    const PcgSymLayout L = pcg_sym_layout(mr, mw, mt, kc);
    cudaFuncSetAttribute(k_pcg_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)avail);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg_sym, block, L.total);
    if (occ < cps) return BF_E_CAPACITY;
    const size_t stride = pcg_sym_vec_bytes(mr);
    if (S.pcg_gvec) dev_free(S, S.pcg_gvec);
    if (S.pcg_uval) dev_free(S, S.pcg_uval);
    if (S.pcg_yq) dev_free(S, S.pcg_yq);
    if (S.pcg_pp) dev_free(S, S.pcg_pp);
    if (S.pcg_z4) dev_free(S, S.pcg_z4);
    S.pcg_gvec = (unsigned char *)dev_alloc(S, stride * grid);
    S.pcg_uval = (float *)dev_alloc(S, std::max<size_t>(ubytes, 128));
    S.pcg_yq = (float4 *)dev_alloc(S, (size_t)S.nv * sizeof(float4));
    S.pcg_pp = (float *)dev_alloc(S, 6 * (size_t)S.nv * sizeof(float));
    S.pcg_z4 = (float4 *)dev_alloc(S, (size_t)S.nv * sizeof(float4));
    if (!S.pcg_gvec || !S.pcg_uval || !S.pcg_yq || !S.pcg_pp || !S.pcg_z4) return BF_E_OOM;
    S.pcg_gvec_stride = stride;
    S.pcg_grid = grid;
    S.pcg_block = block;
    S.pcg_smem = (int)L.total;
    S.pcg_resident = PCG_SYM;
    S.pcg_max_rows = mr;
    S.pcg_max_ent = S.nnzb;
    S.pcg_max_win = mw;
    S.pcg_max_len = mt;  // chunk-table entries per CTA (rounds x levels + 1)
    S.pcg_kc = kc;
    return BF_OK;
}


// Chooses the launch: the resident variant when the blocks fit in shared
// memory at the requested CTAs per SM (falling back to fewer CTAs per SM),
// else the variant that streams the blocks from global memory.  Shared
// memory left over caches contact pairs (up to kPcgMaxCached per CTA).
template <class MT, class VT>
static int setup_persistent(Scene &S)
{
    using CT = typename std::conditional<(sizeof(MT) >= sizeof(VT)), MT, VT>::type;
    constexpr bool mixed = sizeof(VT) == 4;
    int dev = 0, nsm = 0, coop = 0, smem_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) return BF_E_CUDA;
    const int per_sm = std::min(4, std::max(1, S.pcg_ctas_per_sm));
    const int modes[5] = {PCG_CG1, PCG_RESIDENT, PCG_STREAM, PCG_SYM, PCG_GLOBAL};
    for (int mode : modes) {
        if (mode == PCG_CG1 && !S.pcg_cg1) continue;
        if ((mode == PCG_RESIDENT || mode == PCG_CG1) && !S.pcg_allow_resident) continue;
        if ((mode == PCG_RESIDENT || mode == PCG_CG1 || mode == PCG_STREAM) && S.pcg_force_global) continue;
        if (mode == PCG_SYM) {  // mixed precision only (FP32 blocks and vector reductions)
            if constexpr (mixed && std::is_same<MT, float>::value) {
                if (S.pcg_no_sym) continue;
                for (int cps = per_sm; cps >= 1; --cps) {
                    const int st = setup_sym(S, nsm, cps, (size_t)smem_optin);
                    if (st == BF_OK) return BF_OK;
                    if (st != BF_E_CAPACITY) return st;
                }
            }
            continue;
        }
        const void *kern = mode == PCG_CG1        ? (const void *)k_pcg_cg1<MT, VT>
                           : mode == PCG_RESIDENT ? (const void *)k_pcg_persistent<MT, VT, PCG_RESIDENT>
                           : mode == PCG_STREAM   ? (const void *)k_pcg_persistent<MT, VT, PCG_STREAM>
                                                  : (const void *)k_pcg_persistent<MT, VT, PCG_GLOBAL>;
        // shared-memory bytes at kc cached contact pairs
        auto layout_bytes = [&](int mr, int mw, int me, int ml, int kc) -> size_t {
            if (mode == PCG_CG1) return pcg_cg1_layout(mixed, sizeof(CT), sizeof(MT), mr, mw, me, ml, kc).total;
            return pcg_layout(mixed, sizeof(CT), sizeof(MT), mr, mw, me, ml, mode, kc).total;
        };
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return BF_E_CUDA;
        for (int cps = per_sm; cps >= 1; --cps) {
            // small systems take fewer CTAs (about kPcgEntriesPerCta blocks
            // each), which keeps the barriers short and leaves SMs to other
            // scenes running concurrently; FP64 blocks take a quarter of that
            // (twice the bytes, and B300's narrow FP64 pipe: the blocks then
            // fit in shared memory and their arithmetic spreads over more SMs)
            const int per_cta = sizeof(MT) == 8 ? kPcgEntriesPerCta / 4 : kPcgEntriesPerCta;
            const int grid = std::max(1, std::min(nsm * cps, cdiv(S.nfull, per_cta)));
            if (grid > kPcgMaxGrid) continue;
            const int block = (kPcgThreads / cps) & ~31;
            int mr = 0, me = 0, mw = 0, ml = 0;
            int st = make_partition(S, grid, &mr, &me, &mw, &ml);
            if (st == BF_E_CAPACITY) continue;
            if (st) return st;
            const size_t avail = (size_t)smem_optin - fa.sharedSizeBytes;
            const size_t L0 = layout_bytes(mr, mw, me, ml, 0);
            if (L0 > avail) continue;
            int kc = S.pcg_no_cache ? 0 : (int)std::min<size_t>(kPcgMaxCached, (avail - L0) / pcg_contact_bytes(sizeof(CT)));
            while (kc > 0 && layout_bytes(mr, mw, me, ml, kc) > avail) --kc;
            const size_t Ltotal = layout_bytes(mr, mw, me, ml, kc);
            // the attribute is an upper bound shared by every scene: set it to
            // the most any launch may ask for, so concurrent set-ups agree
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)avail);
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, Ltotal);
            if (occ < cps) continue;
            if (mode == PCG_CG1) {  // published row sums, contact parts, (r, s), H x
                if (S.pcg_cg1buf) dev_free(S, S.pcg_cg1buf);
                const PcgCg1Buf cbl = pcg_cg1_buf(S.nv, sizeof(CT));
                S.pcg_cg1buf = (unsigned char *)dev_alloc(S, cbl.total);
                if (!S.pcg_cg1buf) return BF_E_OOM;
                cudaMemsetAsync(S.pcg_cg1buf + cbl.fl, 0, cbl.total - cbl.fl, S.stream);  // no vertex flagged
            }
            if (mode == PCG_GLOBAL) {  // jagged block copy and per-CTA vectors in global memory
                const size_t stride = (pcg_vec_layout(mixed, sizeof(CT), mr).total + 255) & ~(size_t)255;
                if (S.pcg_gvec) dev_free(S, S.pcg_gvec);
                if (S.pcg_jval) dev_free(S, S.pcg_jval);
                S.pcg_gvec = (unsigned char *)dev_alloc(S, stride * grid);
                S.pcg_jval = dev_alloc(S, 9 * (size_t)S.nfull * sizeof(MT));
                if (!S.pcg_gvec || !S.pcg_jval) return BF_E_OOM;
                S.pcg_gvec_stride = stride;
            }
            S.pcg_grid = grid;
            S.pcg_block = block;
            S.pcg_smem = (int)Ltotal;
            S.pcg_resident = mode;
            S.pcg_max_rows = mr;
            S.pcg_max_ent = me;
            S.pcg_max_win = mw;
            S.pcg_max_len = ml;
            S.pcg_kc = kc;
            return BF_OK;
        }
    }
    return BF_E_CAPACITY;
}

// global variant: the blocks of every CTA in jagged order, 9 planes
template <class MT>
__global__ void k_jagged_gather(int nfull, const int *__restrict__ fblk, const int *__restrict__ edst,
                                const MT *__restrict__ val, MT *__restrict__ jval)
{
    const int fe = blockIdx.x * blockDim.x + threadIdx.x;
    if (fe >= nfull) return;
    const int fb = fblk[fe];
    const MT *src = val + 9 * (size_t)(fb & 0x7fffffff);
    const size_t d = (size_t)edst[fe];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) jval[(size_t)(3 * i + j) * nfull + d] = fb < 0 ? src[3 * j + i] : src[3 * i + j];
}

// Persistent kernels launched from different streams (scenes of a batch)
// may run at the same time only if all their CTAs fit on the device
// together: each CTA spins at grid barriers for the others, so two grids
// that each hold part of the SMs while waiting for the rest would wait for
// each other.  A process-wide budget of SM slots per device enforces that;
// ordinary kernels always finish, so they only delay a grid.
constexpr int kSlotsPerSm = 12;  // a CTA of a grid at c CTAs per SM takes 12 / c slots

struct CoopSlots {
    std::mutex mu;
    std::condition_variable cv;
    int used = 0;
};

static CoopSlots &coop_slots(int dev)
{
    static CoopSlots slots[64];
    return slots[dev & 63];
}

// takes `units` SM slots of device `dev` (waiting until they are free);
// returns the units taken
static int coop_acquire(int dev, int units, int capacity)
{
    CoopSlots &c = coop_slots(dev);
    units = std::min(units, capacity);
    std::unique_lock<std::mutex> lk(c.mu);
    c.cv.wait(lk, [&] { return c.used + units <= capacity; });
    c.used += units;
    return units;
}

static void coop_release(int dev, int units)
{
    CoopSlots &c = coop_slots(dev);
    {
        std::lock_guard<std::mutex> lk(c.mu);
        c.used -= units;
    }
    c.cv.notify_all();
}

// the slots of a launched solve go back once it has completed
static void release_pcg_slots(Scene &S)
{
    if (S.pcg_slots_held) coop_release(S.pcg_slots_dev, S.pcg_slots_held);
    S.pcg_slots_held = 0;
}

template <class MT, class VT>
static int persistent_impl(Scene &S, const MT *val, const MT *pinv, VT *p0, VT *p1, VT *z, const double *b,
                           double *x, double tol, int maxit, int *iters, bool defer)
{
    if (S.pcg_grid == 0) {
        const int st = setup_persistent<MT, VT>(S);
        if (st) return st;
    }
    const int grid = S.pcg_grid;
    PcgArgs A;
    A.nv = S.nv;
    A.nc = n_terms(S);  // augmented-Lagrangian pairs and friction terms
    A.part = S.part;
    A.win = S.win;
    A.frowptr = S.frowptr;
    A.eslot = S.pcg_eslot;
    A.rinfo = S.pcg_rinfo;
    A.lvl = S.pcg_lvl;
    A.lvlptr = S.pcg_lvlptr;
    A.fnbr = S.fnbr;
    A.fblk = S.fblk;
    A.val = val;
    A.cv = S.cv;
    A.cg = S.cg;
    A.cw = S.cw;
    A.cmask = S.cmask;
    A.pinv = pinv;
    A.b = b;
    A.x = x;
    A.z = z;
    A.p0 = p0;
    A.p1 = p1;
    A.qd = S.cg_qc;  // FP64 contact part of H p, and of H x in the reliable updates
    A.res = S.dscal + S_RES;
    A.bar = S.bar;
    A.bar_poll = S.pcg_bar_fail ? S.bar + 1 : S.bar;  // failure-detection test: a word no CTA increments
    A.tol2 = tol * tol;
    A.maxit = maxit;
    A.max_replace = 64;
    A.max_rows = S.pcg_max_rows;
    A.max_ent = S.pcg_max_ent;
    A.max_win = S.pcg_max_win;
    A.max_len = S.pcg_max_len;
    A.jval = S.pcg_jval;
    A.jnbr = S.pcg_jnbr;
    A.gvec = S.pcg_gvec;
    A.gvec_stride = S.pcg_gvec_stride;
    A.nfull = S.nfull;
    if (S.pcg_resident == PCG_GLOBAL) {
        k_jagged_gather<MT><<<cdiv(S.nfull, kThreads), kThreads, 0, S.stream>>>(S.nfull, S.fblk, S.pcg_edst, val,
                                                                              (MT *)S.pcg_jval);
        ++S.n_launch;
    }
    A.uval = S.pcg_uval;
    A.yq = S.pcg_yq;
    {
        const PcgCg1Buf cbl = pcg_cg1_buf(S.nv, sizeof(VT) == 4 ? 4 : 8);
        unsigned char *cb = S.pcg_cg1buf;
        A.cwq = cb ? cb + cbl.wq : nullptr;
        A.cqc = cb ? (double *)(cb + cbl.qc) : nullptr;
        A.crs = cb ? cb + cbl.rs : nullptr;
        A.chx = cb ? (double *)(cb + cbl.hx) : nullptr;
        A.cpp = S.pcg_resident == PCG_SYM ? (void *)S.pcg_pp : cb ? (void *)(cb + cbl.pp) : nullptr;
        A.cfl = cb ? cb + cbl.fl : nullptr;
        A.z4 = S.pcg_z4;
    }
    if (S.pcg_resident == PCG_SYM) {
        if constexpr (std::is_same<MT, float>::value) {
            k_jagged_gather_upper<<<cdiv(S.nnzb, kThreads), kThreads, 0, S.stream>>>(
                S.nnzb, (const int2 *)S.pcg_uedst, S.pcg_unbr, val, (unsigned char *)S.pcg_uval);
            ++S.n_launch;
        } else {
            return BF_E_ARG;
        }
    }
    A.kc = S.pcg_kc;
    A.dscal = S.dscal;
    A.dflag = S.dflag;
    cudaMemsetAsync(S.bar, 0, 4 * sizeof(unsigned), S.stream);
    cudaMemsetAsync(S.dscal + S_RES, 0, 24 * sizeof(double), S.stream);  // the three accumulator slots
    cudaMemsetAsync(S.dflag + F_ERR, 0, sizeof(int), S.stream);
    void *args[] = {&A};
    cudaError_t e;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int cps = std::max(1, kPcgThreads / S.pcg_block);
    release_pcg_slots(S);
    S.pcg_slots_dev = dev;  // held until the solve has completed
    S.pcg_slots_held = coop_acquire(dev, grid * (kSlotsPerSm / std::min(cps, kSlotsPerSm)), nsm * kSlotsPerSm);
    {
        ScopedTimer tm(S, T_PCG_PERSISTENT);
        const void *kern = S.pcg_resident == PCG_RESIDENT ? (const void *)k_pcg_persistent<MT, VT, PCG_RESIDENT>
                           : S.pcg_resident == PCG_STREAM ? (const void *)k_pcg_persistent<MT, VT, PCG_STREAM>
                           : S.pcg_resident == PCG_SYM    ? (const void *)k_pcg_sym
                           : S.pcg_resident == PCG_CG1    ? (const void *)k_pcg_cg1<MT, VT>
                                                          : (const void *)k_pcg_persistent<MT, VT, PCG_GLOBAL>;
        e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(S.pcg_block), args, (size_t)S.pcg_smem, S.stream);
        ++S.n_launch;
    }
    if (e != cudaSuccess) {
        release_pcg_slots(S);
        return BF_E_CUDA;
    }
    if (defer) return BF_OK;
    const int st = sync_flags(S);
    if (st) {
        release_pcg_slots(S);
        return st;
    }
    return pcg_finish(S, iters);
}

// status of the last persistent solve, after a sync_flags
int pcg_finish(Scene &S, int *iters)
{
    release_pcg_slots(S);
    if (iters) *iters = S.h_flag[F_ITERS];
    if (S.timers_on) {  // per-phase device time seen by CTA 0 (globaltimer)
        const int ids[7] = {T_PCG_PH_SPMV, T_PCG_PH_RED1, T_PCG_PH_UPD, T_PCG_PH_RED2, T_PCG_PH_STAGE,
                            T_PCG_PH_ROWS, T_PCG_PH_CONTACT};
        const int slots[7] = {S_T_SPMV, S_T_RED1, S_T_UPD, S_T_RED2, S_T_STAGE, S_T_ROWS, S_T_CONTACT};
        for (int i = 0; i < 7; ++i) {
            S.t_launch[ids[i]] += S.h_flag[F_ITERS];
            S.t_ms[ids[i]] += S.h_scal[slots[i]];
        }
    }
    if (S.h_flag[F_ERR] & ERR_BARRIER) return BF_E_CUDA;
    if (S.h_flag[F_ERR] & ERR_NONFINITE) return BF_E_NONFINITE;
    return S.h_flag[F_MAXIT] ? BF_E_CG_MAXIT : BF_OK;
}

// Falls back to the per-phase launches when no persistent configuration
// fits (a vertex window beyond 16-bit offsets, or too little shared memory).
static int persistent_entry(Scene &S, const double *b, double *x, double tol, int maxit, int *iters, bool defer,
                            int *pending)
{
    int st;
    if (S.prm.precision == BF_PREC_MIXED)
        st = persistent_impl<float, float>(S, S.valf, S.pinvf, S.cg_pf, S.cg_pf2, S.cg_zf, b, x, tol, maxit,
                                           iters, defer);
    else
        st = persistent_impl<double, double>(S, S.val, S.pinv, S.cg_p, S.cg_p2, S.cg_z, b, x, tol, maxit,
                                             iters, defer);
    if (st == BF_E_CAPACITY && S.pcg_grid == 0) {
        S.pcg_mode = 0;
        return run_pcg(S, b, x, tol, maxit, iters);
    }
    if (pending) *pending = defer && st == BF_OK;
    return st;
}

void pcg_release(Scene &S) { release_pcg_slots(S); }

int run_pcg_persistent(Scene &S, const double *b, double *x, double tol, int maxit, int *iters)
{
    return persistent_entry(S, b, x, tol, maxit, iters, false, nullptr);
}

int run_pcg_async(Scene &S, const double *b, double *x, double tol, int maxit, int *iters, int *pending)
{
    *pending = 0;
    if (S.pcg_mode != 1) return run_pcg(S, b, x, tol, maxit, iters);
    return persistent_entry(S, b, x, tol, maxit, iters, true, pending);
}

}  // namespace bf
