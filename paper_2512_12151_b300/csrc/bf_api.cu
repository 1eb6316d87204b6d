// C ABI (include/bf.h) and the host-side drivers of Alg. 1 (time step) and
// Alg. 2 (SolveSubproblem).  Every arithmetic step runs in the kernels of
// bf_elastic.cu, bf_contact.cu, bf_linalg.cu and bf_ccd.cu; this file owns
// the scene set-up (lumped mass, Dm^-1, surface, block pattern), memory,
// control flow and the scalar decisions (line-search acceptance, alpha,
// beta), which it reads back from the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <chrono>
#include <cmath>
#include <cstring>
#include <tuple>
#include <vector>

#include "bf.h"
#include "bf_device.cuh"
#include "bf_internal.cuh"

struct bf_scene {
    bf::Scene s;
    std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> pending;
};

namespace bf {

void launch_linearize_out(Scene &S, const double *xlin, double *dout, double *gout);

static bf_scene *owner_of(Scene &S) { return reinterpret_cast<bf_scene *>(&S); }

// ---------------------------------------------------------------------------
// memory
// ---------------------------------------------------------------------------
// Without a caller allocator, scene memory comes from the device's
// stream-ordered pool (cudaMallocAsync on the scene's stream), which keeps
// freed blocks for reuse instead of returning them at every synchronisation,
// so that creating and destroying scenes while others run (a serving loop)
// neither synchronises the device nor pays for fresh allocations.
static void pool_keep_memory()
{
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    });
}

void *dev_alloc(Scene &S, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (S.has_alloc) {
        p = S.alloc.alloc(bytes, S.alloc.ctx);
    } else {
        pool_keep_memory();
        if (cudaMallocAsync(&p, bytes, S.stream) != cudaSuccess) p = nullptr;
    }
    if (p) {
        S.owned.push_back(p);
        S.owned_bytes.push_back(bytes);
        S.bytes += bytes;
    }
    return p;
}

void dev_free(Scene &S, void *p)
{
    if (!p) return;
    auto it = std::find(S.owned.begin(), S.owned.end(), p);
    if (it != S.owned.end()) {
        const size_t k = it - S.owned.begin();
        S.bytes -= S.owned_bytes[k];
        S.owned_bytes.erase(S.owned_bytes.begin() + k);
        S.owned.erase(it);
    }
    if (S.has_alloc) S.alloc.free(p, S.alloc.ctx);
    else cudaFreeAsync(p, S.stream);
}

int check_cuda(cudaError_t e) { return e == cudaSuccess ? BF_OK : BF_E_CUDA; }

int sync_flags(Scene &S)
{
    cudaMemcpyAsync(S.h_scal, S.dscal, S_NSCAL * sizeof(double), cudaMemcpyDeviceToHost, S.stream);
    cudaMemcpyAsync(S.h_flag, S.dflag, F_NFLAG * sizeof(int), cudaMemcpyDeviceToHost, S.stream);
    cudaError_t e;
    if (S.sync_blocking && S.sync_ev) {
        e = cudaEventRecord(S.sync_ev, S.stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(S.sync_ev);
    } else {
        e = cudaStreamSynchronize(S.stream);
    }
    if (e != cudaSuccess) return BF_E_CUDA;
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// timers
// ---------------------------------------------------------------------------
static const char *kTimerNames[T_N] = {"elastic_grad_hess", "spmv_bsr_contact", "pcg_update", "pcg_direction",
                                       "contact_assemble", "energy", "ccd_narrow_accd", "lbvh_build",
                                       "pcg_persistent", "pcg_phase_spmv", "pcg_phase_reduce1",
                                       "pcg_phase_update", "pcg_phase_reduce2", "pcg_phase_stage_cum",
                                       "pcg_phase_rows_cum", "pcg_phase_contact_cum", "ccd_broad_query"};

ScopedTimer::ScopedTimer(Scene &s, int tid) : S(&s), id(tid)
{
    if (!S->timers_on) return;
    auto take = [&]() {
        cudaEvent_t e;
        if (!S->ev_pool.empty()) {
            e = S->ev_pool.back();
            S->ev_pool.pop_back();
        } else {
            cudaEventCreate(&e);
        }
        return e;
    };
    a = take();
    b = take();
    cudaEventRecord(a, S->stream);
}

ScopedTimer::~ScopedTimer()
{
    if (!a) return;
    cudaEventRecord(b, S->stream);
    owner_of(*S)->pending.emplace_back(id, a, b);
}

void flush_timers(Scene &S)
{
    auto &P = owner_of(S)->pending;
    for (auto &t : P) {
        float ms = 0.f;
        cudaEventSynchronize(std::get<2>(t));
        cudaEventElapsedTime(&ms, std::get<1>(t), std::get<2>(t));
        S.t_launch[std::get<0>(t)] += 1;
        S.t_ms[std::get<0>(t)] += ms;
        S.ev_pool.push_back(std::get<1>(t));
        S.ev_pool.push_back(std::get<2>(t));
    }
    P.clear();
}

// ---------------------------------------------------------------------------
// small kernels used by the host-side step functions
// ---------------------------------------------------------------------------
__global__ void k_scale(int n, double *__restrict__ out, const double *__restrict__ in, double s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = s * in[i];
}

// *out = |v| (grid sum)
__global__ void k_norm(int n, const double *__restrict__ v, double *partials, unsigned *counter, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s[1] = {i < n ? v[i] * v[i] : 0.0}, tot[1];
    if (grid_sum<1>(s, partials, counter, tot)) *out = sqrt(tot[0]);
}

// out = -in / |in| (zero for a zero vector)
__global__ void k_neg_unit(int n, double *__restrict__ out, const double *__restrict__ in,
                           const double *__restrict__ nrm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double g = *nrm;
    if (i < n) out[i] = g > 0.0 ? -in[i] / g : 0.0;
}

__global__ void k_apply_targets(int nd, const int *__restrict__ ids, const double *__restrict__ tg,
                                double *__restrict__ x)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nd) return;
    const int v = ids[i];
    x[3 * v] = tg[3 * i];
    x[3 * v + 1] = tg[3 * i + 1];
    x[3 * v + 2] = tg[3 * i + 2];
}

__global__ void k_set_double(double *p, double v) { *p = v; }
__global__ void k_fill(int n, double *__restrict__ out, double v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}

// ---------------------------------------------------------------------------
// active set storage
// ---------------------------------------------------------------------------
static int partials_reserve(Scene &S)
{
    const long long work = (long long)S.nnzb + S.nt + S.nv + S.ccap + 1024;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // per-phase grids need 2 values per CTA; the persistent PCG 3 per
    // co-resident CTA (at most 8 per SM)
    const int need = std::max(2 * cdiv(work, kThreads), 3 * 8 * std::max(nsm, 1)) + 64;
    if (need <= S.npartials) return BF_OK;
    if (S.partials) dev_free(S, S.partials);
    S.partials = (double *)dev_alloc(S, need * sizeof(double));
    if (!S.partials) return BF_E_OOM;
    S.npartials = need;
    return BF_OK;
}

int active_reserve(Scene &S, int n)
{
    if (n <= S.ccap) return BF_OK;
    const int cap = std::max(n + n / 2, std::max(2 * S.ccap, 1024));
    auto grow = [&](auto *&p, size_t elem, size_t per, bool keep) -> bool {
        void *q = dev_alloc(S, (size_t)cap * per * elem);
        if (!q) return false;
        if (keep && p && S.nc)
            cudaMemcpyAsync(q, p, (size_t)S.nc * per * elem, cudaMemcpyDeviceToDevice, S.stream);
        if (p) {
            cudaStreamSynchronize(S.stream);
            dev_free(S, p);
        }
        p = reinterpret_cast<std::remove_reference_t<decltype(p)>>(q);
        return true;
    };
    bool ok = grow(S.ctype, sizeof(int), 1, true) && grow(S.ca, sizeof(int), 1, true) &&
              grow(S.cb, sizeof(int), 1, true) && grow(S.cv, sizeof(int4), 1, true) &&
              grow(S.clam, sizeof(double), 1, true) && grow(S.cgam, sizeof(double), 1, true) &&
              grow(S.cd, sizeof(double), 1, true) && grow(S.cg, sizeof(double), 12, true) &&
              grow(S.cs, sizeof(double), 1, true) && grow(S.cw, sizeof(double), 1, true) &&
              grow(S.cmask, 1, 1, true) && grow(S.ckey, sizeof(unsigned long long), 1, false) &&
              grow(S.ckey_sorted, sizeof(unsigned long long), 1, false);
    if (!ok) return BF_E_OOM;
    S.ccap = cap;
    return partials_reserve(S);
}

// ---------------------------------------------------------------------------
// Newton step pieces
// ---------------------------------------------------------------------------
static int assemble(Scene &S, const double *xtilde, const double *xlin, const double *xhat)
{
    cudaMemsetAsync(S.dflag + F_ERR, 0, sizeof(int), S.stream);
    if (!S.elastic_ready) {
        launch_vertex_init(S, xtilde, xhat);
        launch_elastic(S, xhat);
    }
    S.elastic_ready = false;
    launch_contact_assemble(S, xlin, xhat);
    const int st = launch_friction_assemble(S, xhat);
    if (st) return st;
    launch_pinv(S);
    return BF_OK;
}

static double mu_init(Scene &S, const double *xtilde, const double *xhat)
{
    launch_vertex_init(S, xtilde, xhat);
    launch_elastic(S, xhat);
    const double mx = run_mu_max_diag(S);
    S.mu = S.prm.c_mu * mx;
    return S.mu;
}

// |v|_inf of a vector -> *out (zeroed before; non-negative doubles compare
// like their bit patterns)
__global__ void k_absmax(int n, const double *__restrict__ v, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double m = i < n ? fabs(v[i]) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomic_max_pos(out, m);
}

// Gradient-norm residual of IPC (section 6): (1/h) |H^-1 grad L|_inf at x,
// L linearised at x with the current active set, multipliers, mu and delta
// and taken at xhat = x.  H p = -G is solved for the unit right-hand side
// (as in the Newton loop) and |p|_inf scaled back by |G|.
static int newton_residual(Scene &S, const double *xtilde, const double *x, double *res)
{
    const int n = 3 * S.nv;
    S.elastic_ready = false;
    launch_linearize(S, x);
    int st = assemble(S, xtilde, x, x);
    if (st) return st;
    k_norm<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, S.grad, S.partials, S.counter, S.dscal + S_GNORM);
    k_neg_unit<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, S.cg_b, S.grad, S.dscal + S_GNORM);
    S.n_launch += 2;
    int it = 0;
    st = run_pcg(S, S.cg_b, S.pdir, S.prm.cg_tol, S.prm.max_cg, &it);
    if (st && st != BF_E_CG_MAXIT) return st;
    cudaMemsetAsync(S.dscal + S_RESID, 0, sizeof(double), S.stream);
    k_absmax<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, S.pdir, S.dscal + S_RESID);
    ++S.n_launch;
    st = sync_flags(S);
    if (st) return st;
    *res = S.h_scal[S_GNORM] * S.h_scal[S_RESID] / S.prm.dt;
    return std::isfinite(*res) ? BF_OK : BF_E_NONFINITE;
}

struct SolveStats {
    int newton = 0, cg = 0, ls_fail = 0, cg_maxit = 0, newton_cap = 0;
};

// Alg. 2 SolveSubproblem (xhat in/out).  Line search: r = 1, 1/2, ...,
// 2^-max_ls with L(xhat + r p) <= L(xhat) + 1e-12 max(|L(xhat)|, L_s) and
// the slacks of the current Newton iteration held fixed; L_s (S.L_scale) is
// |L| at the first Newton iterate of the time step (of the call when called
// alone), so that round-off cannot reject full steps once L has converged to
// about zero, as in free fall, where a later subproblem starts at its
// optimum.
static int solve_subproblem(Scene &S, const double *xtilde, const double *xlin, double *xhat, SolveStats &ss)
{
    const int n = 3 * S.nv;
    launch_linearize(S, xlin);
    while (true) {
        if (ss.newton >= S.prm.max_newton) {
            ss.newton_cap++;
            break;
        }
        int st = assemble(S, xtilde, xlin, xhat);
        if (st) return st;
        // H p = -G solved for the unit right-hand side, p scaled back by |G|
        // on the device: the FP32 products of the mixed-precision solve would
        // underflow for a gradient at its rounding floor (a subproblem that
        // starts at its optimum)
        k_norm<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, S.grad, S.partials, S.counter, S.dscal + S_GNORM);
        k_neg_unit<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, S.cg_b, S.grad, S.dscal + S_GNORM);
        S.n_launch += 2;
        int it = 0, pending = 0;
        st = run_pcg_async(S, S.cg_b, S.pdir, S.prm.cg_tol, S.prm.max_cg, &it, &pending);
        if (st && st != BF_E_CG_MAXIT) return st;
        // L at xhat and at the full step queued behind the solve: one
        // synchronisation for the three
        launch_axpy_scaled(S, S.xtmp, xhat, 1.0, S.pdir, S.dscal + S_GNORM, n);
        launch_energy(S, xtilde, xlin, xhat, S.dscal + S_E0);
        launch_energy(S, xtilde, xlin, S.xtmp, S.dscal + S_E1);
        const int sst = sync_flags(S);
        if (sst) {
            pcg_release(S);
            return sst;
        }
        if (pending) st = pcg_finish(S, &it);
        ss.cg += it;
        if (st == BF_E_CG_MAXIT) ss.cg_maxit++;
        else if (st) return st;
        const double L0 = S.h_scal[S_E0];
        if (!std::isfinite(L0)) return BF_E_NONFINITE;
        if (S.L_scale < 0.0) S.L_scale = std::fabs(L0);
        const double ls_tol = 1e-12 * std::max(std::fabs(L0), S.L_scale);
        double r = 1.0, L1 = S.h_scal[S_E1];
        bool ok = false;
        for (int j = 0; j <= S.prm.max_ls; ++j) {
            if (j > 0) {
                launch_axpy_scaled(S, S.xtmp, xhat, r, S.pdir, S.dscal + S_GNORM, n);
                L1 = run_energy(S, xtilde, xlin, S.xtmp);
            }
            if (std::isfinite(L1) && L1 <= L0 + ls_tol) {
                ok = true;
                break;
            }
            r *= 0.5;
        }
        ss.newton++;
        if (!ok) {
            ss.ls_fail++;
            break;
        }
        cudaMemcpyAsync(xhat, S.xtmp, n * sizeof(double), cudaMemcpyDeviceToDevice, S.stream);
        if (r == 1.0) break;
    }
    launch_multiplier_update(S, xlin, xhat);
    return check_cuda(cudaGetLastError());
}

// Alg. 1: one time step.
static int step_once(Scene &S, bf_step_stats *out)
{
    S.elastic_ready = false;
    auto t0 = std::chrono::steady_clock::now();
    const int n = 3 * S.nv;
    const size_t nb = n * sizeof(double);
    bf_step_stats st{};
    st.min_alpha = 1.0;
    cudaMemcpyAsync(S.xt, S.x, nb, cudaMemcpyDeviceToDevice, S.stream);
    launch_xtilde(S, S.xtilde);
    cudaMemcpyAsync(S.xk, S.x, nb, cudaMemcpyDeviceToDevice, S.stream);
    cudaMemcpyAsync(S.xh, S.x, nb, cudaMemcpyDeviceToDevice, S.stream);
    if (S.has_targets && S.ndir)
        {
            k_apply_targets<<<cdiv(S.ndir, kThreads), kThreads, 0, S.stream>>>(S.ndir, S.dir_ids, S.targets, S.xh); ++S.n_launch;
        }
    {
        const int fst = friction_setup(S);  // from the AL state the previous step left (appendix A)
        if (fst) return fst;
    }
    S.delta = S.prm.delta;
    S.L_scale = -1.0;  // set by the step's first Newton iterate
    S.bvh_tri.topo_valid = S.bvh_edge.topo_valid = 0;  // one tree topology per time step
    S.bvh_reuse = true;
    struct ReuseOff {
        Scene &s;
        ~ReuseOff() { s.bvh_reuse = false; }
    } reuse_off{S};
    mu_init(S, S.xtilde, S.xh);
    if (!(S.mu > 0.0) || !std::isfinite(S.mu)) return BF_E_NONFINITE;
    // the first Newton iterate of the first subproblem is x_hat^[0]: its
    // inertia and elastic terms are the ones mu_init just assembled
    S.elastic_ready = true;
    double beta = 1.0, asum = 0.0;
    int k = 0, stall = 0, status = BF_OK;
    SolveStats ss;
    const bool resmode = S.prm.res_tol > 0.0;  // IPC-style termination (section 6) instead of Eq. termination
    S.res_log.clear();
    for (;;) {
        if (resmode) {
            double r = 0.0;
            const int rc = newton_residual(S, S.xtilde, S.xk, &r);
            if (rc) return rc;
            S.res_log.push_back(r);
            if (r < S.prm.res_tol) break;
        } else if (!(beta > S.prm.eps)) {
            break;
        }
        if (k >= S.prm.max_outer) {
            status = BF_E_OUTER_MAXIT;
            break;
        }
        cudaMemcpyAsync(S.xh_prev, S.xh, nb, cudaMemcpyDeviceToDevice, S.stream);
        int rc = solve_subproblem(S, S.xtilde, S.xk, S.xh, ss);
        if (rc) return rc;
        // UpdateActiveSet along x^k -> xhat^k and MaxStepSize along
        // x^k -> xhat^{k+1}: one broad phase serves both
        int nh = 0;
        double alpha = 1.0;
        rc = S.prm.ccd_reuse ? run_ccd_reuse(S, S.xk, S.xh, &nh, &alpha)  // one CCD for both
                             : run_ccd_two(S, S.xk, S.xh_prev, S.xh, &nh, &alpha);
        if (rc) return rc;
        rc = apply_active_set_hits(S, nh);
        if (rc) return rc;
        launch_blend(S, S.xk, S.xh, alpha, n);
        if (k + 1 >= S.prm.k_min) beta = (1.0 - alpha) * beta;
        ++k;
        asum += alpha;
        st.min_alpha = std::min(st.min_alpha, alpha);
        if (alpha < 1e-4) {
            if (++stall >= 50) {  // section 5.2 stall rule
                S.mu *= 2.0;
                S.delta *= 0.5;
                stall = 0;
                st.stalls++;
            }
        } else {
            stall = 0;
        }
    }
    launch_velocity(S);
    int rc = sync_flags(S);
    if (rc) return rc;
    if (S.timers_on) flush_timers(S);
    st.outer_iters = k;
    st.newton_iters = ss.newton;
    st.cg_iters = ss.cg;
    st.n_contacts = S.nc;
    st.ls_fail = ss.ls_fail;
    st.cg_maxit = ss.cg_maxit;
    st.mean_alpha = k ? asum / k : 0.0;
    st.mu = S.mu;
    st.beta = beta;
    st.delta = S.delta;
    st.status = status;
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (out) *out = st;
    return status;
}

// ---------------------------------------------------------------------------
// scene creation
// ---------------------------------------------------------------------------
// LSD radix sort of non-negative 64-bit keys (16-bit digits; a digit on
// which every key agrees is skipped), carrying a payload when one is given.
// Scene creation sorts a few million keys, where this is several times
// faster than a comparison sort.
template <class K, class V>
static void radix_sort(std::vector<K> &key, std::vector<V> *val)
{
    const size_t n = key.size();
    std::vector<K> k2(n);
    std::vector<V> v2(val ? n : 0);
    std::vector<size_t> cnt(1 << 16);
    for (int shift = 0; shift < 64; shift += 16) {
        std::fill(cnt.begin(), cnt.end(), 0);
        for (size_t i = 0; i < n; ++i) cnt[((unsigned long long)key[i] >> shift) & 0xffff]++;
        if (n == 0 || cnt[((unsigned long long)key[0] >> shift) & 0xffff] == n) continue;
        size_t sum = 0;
        for (auto &c : cnt) {
            const size_t t = c;
            c = sum;
            sum += t;
        }
        for (size_t i = 0; i < n; ++i) {
            const size_t d = cnt[((unsigned long long)key[i] >> shift) & 0xffff]++;
            k2[d] = key[i];
            if (val) v2[d] = (*val)[i];
        }
        key.swap(k2);
        if (val) val->swap(v2);
    }
}

static long long tri_key_sorted(int a, int b, int c)
{
    int t[3] = {a, b, c};
    std::sort(t, t + 3);
    return ((long long)t[0] << 42) | ((long long)t[1] << 21) | (long long)t[2];
}

static int create(Scene &S, const bf_mesh_desc *m, const bf_params *prm)
{
    const int nv = m->n_verts, nt = m->n_tets, nm = m->n_mats, nx = m->n_obst_tris;
    if (nv <= 0 || nt < 0 || nx < 0 || (nt > 0 && nm <= 0) || !m->rest_pos || !m->init_pos) return BF_E_ARG;
    if ((nt > 0 && (!m->tets || !m->tet_mat || !m->mats)) || (nx > 0 && !m->obst_tris)) return BF_E_ARG;
    if (nv >= (1 << 21) || nt >= (1 << 29)) return BF_E_ARG;  // triangle keys pack 3 vertex ids of 21 bits
    if (prm->dt <= 0 || prm->delta < 0 || prm->eps <= 0 || prm->cg_tol <= 0 || prm->k_min < 1 ||
        prm->max_cg < 1 || prm->max_newton < 1 || prm->max_outer < 1 || prm->max_ls < 0 || prm->s_ccd <= 0 ||
        prm->s_ccd >= 1 || !(prm->mu_f >= 0) || (prm->mu_f > 0 && !(prm->eps_v > 0)) || !(prm->res_tol >= 0) ||
        (prm->model != BF_MODEL_SNH && prm->model != BF_MODEL_COR && prm->model != BF_MODEL_NH))
        return BF_E_ARG;
    S.nv = nv;
    S.nt = nt;
    S.nm = nm;
    S.nx = nx;
    S.prm = *prm;
    S.delta = prm->delta;
    S.h_dir.assign(nv, 0);
    if (m->dirichlet)
        for (int v = 0; v < nv; ++v) S.h_dir[v] = m->dirichlet[v] ? 1 : 0;
    for (int v = 0; v < nv; ++v)
        if (S.h_dir[v]) S.h_dir_ids.push_back(v);
    S.ndir = (int)S.h_dir_ids.size();
    // per-tet rest data and lumped mass
    std::vector<double> B(9 * (size_t)nt), vol(nt), emu(nt), elam(nt), mass(nv, 0.0);
    for (int e = 0; e < nt; ++e) {
        const int *t = m->tets + 4 * e;
        for (int k = 0; k < 4; ++k)
            if (t[k] < 0 || t[k] >= nv) return BF_E_ARG;
        const int mi = m->tet_mat[e];
        if (mi < 0 || mi >= nm) return BF_E_ARG;
        double D[9];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) D[3 * r + k] = m->rest_pos[3 * t[k + 1] + r] - m->rest_pos[3 * t[0] + r];
        const double det = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                           D[2] * (D[3] * D[7] - D[4] * D[6]);
        if (!(det > 0.0)) return BF_E_ARG;
        double *o = B.data() + 9 * (size_t)e;
        o[0] = (D[4] * D[8] - D[5] * D[7]) / det;
        o[1] = (D[2] * D[7] - D[1] * D[8]) / det;
        o[2] = (D[1] * D[5] - D[2] * D[4]) / det;
        o[3] = (D[5] * D[6] - D[3] * D[8]) / det;
        o[4] = (D[0] * D[8] - D[2] * D[6]) / det;
        o[5] = (D[2] * D[3] - D[0] * D[5]) / det;
        o[6] = (D[3] * D[7] - D[4] * D[6]) / det;
        o[7] = (D[1] * D[6] - D[0] * D[7]) / det;
        o[8] = (D[0] * D[4] - D[1] * D[3]) / det;
        vol[e] = det / 6.0;
        const double E = m->mats[3 * mi], nu = m->mats[3 * mi + 1], rho = m->mats[3 * mi + 2];
        if (!(E > 0) || !(nu > -1 && nu < 0.5) || !(rho > 0)) return BF_E_ARG;
        emu[e] = E / (2.0 * (1.0 + nu));
        elam[e] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));  // COR, NH: the Lame constant
        if (prm->model == BF_MODEL_SNH) elam[e] += emu[e];      // SNH: shifted (linear small-strain limit)
        for (int k = 0; k < 4; ++k) mass[t[k]] += rho * vol[e] / 4.0;
    }
    for (int v = 0; v < nv; ++v) {
        if (S.h_dir[v]) mass[v] = 1.0;
        else if (!(mass[v] > 0.0)) return BF_E_ARG;  // a free vertex must belong to a tet
    }
    // surface: tet faces used exactly once (outward order (1,2,3), (0,3,2),
    // (0,1,3), (0,2,1) of a positively oriented tet), then obstacle triangles
    static const int fl[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
    std::vector<long long> fkey(4 * (size_t)nt);
    std::vector<int> fidx(4 * (size_t)nt);
    for (int e = 0; e < nt; ++e)
        for (int f = 0; f < 4; ++f) {
            const int *t = m->tets + 4 * e;
            fkey[4 * e + f] = tri_key_sorted(t[fl[f][0]], t[fl[f][1]], t[fl[f][2]]);
            fidx[4 * e + f] = 4 * e + f;
        }
    radix_sort(fkey, &fidx);  // stable: equal keys keep their face order
    for (size_t i = 0; i < fkey.size();) {
        size_t j = i;
        while (j < fkey.size() && fkey[j] == fkey[i]) ++j;
        if (j - i == 1) {
            const int e = fidx[i] / 4, f = fidx[i] % 4;
            for (int k = 0; k < 3; ++k) S.h_st.push_back(m->tets[4 * e + fl[f][k]]);
        }
        i = j;
    }
    for (int i = 0; i < nx; ++i)
        for (int k = 0; k < 3; ++k) {
            const int v = m->obst_tris[3 * i + k];
            if (v < 0 || v >= nv) return BF_E_ARG;
            S.h_st.push_back(v);
        }
    S.nst = (int)(S.h_st.size() / 3);
    std::vector<long long> ek;
    for (int i = 0; i < S.nst; ++i)
        for (int k = 0; k < 3; ++k) {
            const int a = S.h_st[3 * i + k], b = S.h_st[3 * i + (k + 1) % 3];
            ek.push_back(((long long)std::min(a, b) << 32) | (long long)std::max(a, b));
        }
    radix_sort(ek, (std::vector<int> *)nullptr);
    ek.erase(std::unique(ek.begin(), ek.end()), ek.end());
    for (long long k : ek) {
        S.h_se.push_back((int)(k >> 32));
        S.h_se.push_back((int)(k & 0xffffffff));
    }
    S.nse = (int)ek.size();
    {
        std::vector<char> on(nv, 0);
        for (int v : S.h_st) on[v] = 1;
        for (int v = 0; v < nv; ++v)
            if (on[v]) S.h_sv.push_back(v);
        S.nsv = (int)S.h_sv.size();
    }
    {
        std::vector<long long> tk(S.nst);
        std::vector<int> ti(S.nst);
        for (int i = 0; i < S.nst; ++i) {
            tk[i] = tri_key_sorted(S.h_st[3 * i], S.h_st[3 * i + 1], S.h_st[3 * i + 2]);
            ti[i] = i;
        }
        radix_sort(tk, &ti);
        S.h_tri_key_sorted = tk;
        S.h_tri_key_idx = ti;
    }
    // upper block pattern: diagonal of every vertex + (a, b), a < b, sharing a tet
    std::vector<long long> pk;
    pk.reserve((size_t)nv + 10 * (size_t)nt);
    for (int v = 0; v < nv; ++v) pk.push_back(((long long)v << 32) | v);
    for (int e = 0; e < nt; ++e) {
        const int *t = m->tets + 4 * e;
        for (int i = 0; i < 4; ++i)
            for (int j = i + 1; j < 4; ++j) {
                const int a = std::min(t[i], t[j]), b = std::max(t[i], t[j]);
                pk.push_back(((long long)a << 32) | b);
            }
    }
    radix_sort(pk, (std::vector<int> *)nullptr);
    pk.erase(std::unique(pk.begin(), pk.end()), pk.end());
    S.nnzb = (int)pk.size();
    S.h_rowptr.assign(nv + 1, 0);
    S.h_col.resize(S.nnzb);
    std::vector<int> rowid(S.nnzb), diagblk(nv);
    for (int k = 0; k < S.nnzb; ++k) {
        const int r = (int)(pk[k] >> 32), c = (int)(pk[k] & 0xffffffff);
        S.h_col[k] = c;
        rowid[k] = r;
        S.h_rowptr[r + 1]++;
        if (r == c) diagblk[r] = k;
    }
    for (int v = 0; v < nv; ++v) S.h_rowptr[v + 1] += S.h_rowptr[v];
    auto find_blk = [&](int r, int c) {
        auto b = S.h_col.begin() + S.h_rowptr[r], e = S.h_col.begin() + S.h_rowptr[r + 1];
        return (int)(std::lower_bound(b, e, c) - S.h_col.begin());
    };
    // full-row view: for row r, its diagonal and upper blocks (r, c) and the
    // lower blocks (c, r) stored in row c, transposed
    {
        std::vector<int> cnt(nv, 0);
        for (int k = 0; k < S.nnzb; ++k) {
            cnt[rowid[k]]++;
            if (S.h_col[k] != rowid[k]) cnt[S.h_col[k]]++;
        }
        S.h_frowptr.assign(nv + 1, 0);
        for (int v = 0; v < nv; ++v) S.h_frowptr[v + 1] = S.h_frowptr[v] + cnt[v];
        S.nfull = S.h_frowptr[nv];
    }
    std::vector<int> fnbr(S.nfull), fblk(S.nfull);
    {
        std::vector<int> fill(S.h_frowptr.begin(), S.h_frowptr.end() - 1);
        for (int k = 0; k < S.nnzb; ++k) {  // rows in order, so each row's entries end up sorted by neighbour
            const int r = rowid[k], c = S.h_col[k];
            fnbr[fill[r]] = c;
            fblk[fill[r]++] = k;
        }
        // lower blocks, appended after each row's upper ones would break
        // neighbour order; insert them and sort each row by neighbour
        for (int k = 0; k < S.nnzb; ++k) {
            const int r = rowid[k], c = S.h_col[k];
            if (r == c) continue;
            fnbr[fill[c]] = r;
            fblk[fill[c]++] = k | (int)0x80000000u;
        }
        std::vector<std::pair<int, int>> tmp;
        for (int v = 0; v < nv; ++v) {
            const int b = S.h_frowptr[v], e = S.h_frowptr[v + 1];
            tmp.clear();
            for (int i = b; i < e; ++i) tmp.push_back({fnbr[i], fblk[i]});
            std::sort(tmp.begin(), tmp.end());
            for (int i = b; i < e; ++i) {
                fnbr[i] = tmp[i - b].first;
                fblk[i] = tmp[i - b].second;
            }
        }
    }
    std::vector<int> tblk(10 * (size_t)nt);
    for (int e = 0; e < nt; ++e) {
        const int *t = m->tets + 4 * e;
        int p = 0;
        for (int i = 0; i < 4; ++i)
            for (int j = i; j < 4; ++j, ++p) {
                const int a = t[i], b = t[j];
                tblk[10 * (size_t)e + p] = a <= b ? find_blk(a, b) : (find_blk(b, a) | (int)0x80000000u);
            }
    }
    // ---- device buffers ----
    const size_t n3 = 3 * (size_t)nv;
    auto D = [&](size_t bytes) { return dev_alloc(S, bytes); };
#define BF_ALLOC(ptr, type, count)                         \
    do {                                                   \
        ptr = (type *)D((size_t)(count) * sizeof(type));   \
        if (!ptr) return BF_E_OOM;                         \
    } while (0)
    BF_ALLOC(S.x, double, n3);
    BF_ALLOC(S.v, double, n3);
    BF_ALLOC(S.xt, double, n3);
    BF_ALLOC(S.xtilde, double, n3);
    BF_ALLOC(S.xk, double, n3);
    BF_ALLOC(S.xh, double, n3);
    BF_ALLOC(S.xh_prev, double, n3);
    BF_ALLOC(S.xtmp, double, n3);
    BF_ALLOC(S.targets, double, 3 * (size_t)std::max(S.ndir, 1));
    BF_ALLOC(S.dir, uint8_t, nv);
    BF_ALLOC(S.mass, double, nv);
    BF_ALLOC(S.tets, int4, std::max(nt, 1));
    BF_ALLOC(S.B, double, 9 * (size_t)std::max(nt, 1));
    BF_ALLOC(S.vol, double, std::max(nt, 1));
    BF_ALLOC(S.emu, double, std::max(nt, 1));
    BF_ALLOC(S.elam, double, std::max(nt, 1));
    BF_ALLOC(S.tblk, int, 10 * (size_t)std::max(nt, 1));
    BF_ALLOC(S.rowptr, int, nv + 1);
    BF_ALLOC(S.col, int, S.nnzb);
    BF_ALLOC(S.rowid, int, S.nnzb);
    BF_ALLOC(S.diagblk, int, nv);
    BF_ALLOC(S.frowptr, int, nv + 1);
    BF_ALLOC(S.fnbr, int, S.nfull);
    BF_ALLOC(S.fblk, int, S.nfull);
    if (S.prm.precision == BF_PREC_MIXED) {
        BF_ALLOC(S.valf, float, 9 * (size_t)S.nnzb);
        BF_ALLOC(S.pinvf, float, 9 * (size_t)nv);
        BF_ALLOC(S.cg_pf, float, n3);
        BF_ALLOC(S.cg_qf, float, n3);
        BF_ALLOC(S.cg_zf, float, n3);
        BF_ALLOC(S.cg_pf2, float, n3);
    } else {
        BF_ALLOC(S.pinv, double, 9 * (size_t)nv);
    }
    BF_ALLOC(S.val, double, 9 * (size_t)S.nnzb);  // FP64 block sums (the FP32 copy in mixed precision)
    BF_ALLOC(S.cdiag, double, 9 * (size_t)nv);
    BF_ALLOC(S.grad, double, n3);
    BF_ALLOC(S.cg_x, double, n3);
    BF_ALLOC(S.cg_r, double, n3);
    BF_ALLOC(S.cg_b, double, n3);
    BF_ALLOC(S.cg_p, double, n3);
    BF_ALLOC(S.cg_q, double, n3);
    BF_ALLOC(S.cg_z, double, n3);
    BF_ALLOC(S.pdir, double, n3);
    BF_ALLOC(S.cg_p2, double, n3);
    BF_ALLOC(S.cg_qc, double, n3);
    BF_ALLOC(S.bar, unsigned, 4);
    BF_ALLOC(S.counter, unsigned, 4);
    BF_ALLOC(S.dscal, double, S_NSCAL);
    BF_ALLOC(S.dflag, int, F_NFLAG);
    BF_ALLOC(S.sv, int, std::max(S.nsv, 1));
    BF_ALLOC(S.st, int, 3 * (size_t)std::max(S.nst, 1));
    BF_ALLOC(S.se, int, 2 * (size_t)std::max(S.nse, 1));
    BF_ALLOC(S.tv, unsigned long long, nv);
    BF_ALLOC(S.bounds, double, 8);
    BF_ALLOC(S.dir_ids, int, std::max(S.ndir, 1));
#undef BF_ALLOC
    if (cudaMallocHost(&S.h_scal, S_NSCAL * sizeof(double)) != cudaSuccess) return BF_E_OOM;
    if (cudaMallocHost(&S.h_flag, F_NFLAG * sizeof(int)) != cudaSuccess) return BF_E_OOM;
    cudaStream_t s = S.stream;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    up(S.x, m->init_pos, n3 * 8);
    if (m->init_vel) up(S.v, m->init_vel, n3 * 8);
    else cudaMemsetAsync(S.v, 0, n3 * 8, s);
    up(S.dir, S.h_dir.data(), nv);
    up(S.mass, mass.data(), nv * 8);
    up(S.tets, m->tets, (size_t)nt * 16);
    up(S.B, B.data(), B.size() * 8);
    up(S.vol, vol.data(), nt * 8);
    up(S.emu, emu.data(), nt * 8);
    up(S.elam, elam.data(), nt * 8);
    up(S.tblk, tblk.data(), tblk.size() * 4);
    up(S.rowptr, S.h_rowptr.data(), (nv + 1) * 4);
    up(S.col, S.h_col.data(), S.nnzb * 4);
    up(S.rowid, rowid.data(), S.nnzb * 4);
    up(S.diagblk, diagblk.data(), nv * 4);
    up(S.frowptr, S.h_frowptr.data(), (nv + 1) * 4);
    up(S.fnbr, fnbr.data(), (size_t)S.nfull * 4);
    S.h_fnbr = fnbr;
    up(S.fblk, fblk.data(), (size_t)S.nfull * 4);
    up(S.sv, S.h_sv.data(), S.nsv * 4);
    up(S.st, S.h_st.data(), S.h_st.size() * 4);
    up(S.se, S.h_se.data(), S.h_se.size() * 4);
    up(S.dir_ids, S.h_dir_ids.data(), S.ndir * 4);
    cudaMemsetAsync(S.counter, 0, 16, s);
    cudaMemsetAsync(S.dscal, 0, S_NSCAL * 8, s);
    cudaMemsetAsync(S.dflag, 0, F_NFLAG * 4, s);
    int st = active_reserve(S, 1024);
    if (st) return st;
    st = ccd_reserve(S, 1 << 16, 1 << 16, 1 << 14);
    if (st) return st;
    st = partials_reserve(S);
    if (st) return st;
    // keep host copies of everything the hot path needs for the duration of
    // the async uploads
    st = check_cuda(cudaStreamSynchronize(s));
    return st;
}

static void destroy(Scene &S)
{
    if (S.stream) cudaStreamSynchronize(S.stream);
    pcg_release(S);
    if (S.sync_ev) cudaEventDestroy(S.sync_ev);
    S.sync_ev = nullptr;
    std::vector<void *> o = S.owned;
    for (void *p : o) dev_free(S, p);
    if (S.h_scal) cudaFreeHost(S.h_scal);
    if (S.h_flag) cudaFreeHost(S.h_flag);
    for (cudaEvent_t e : S.ev_pool) cudaEventDestroy(e);
}

// canonical key (bf.h) of an internal pair
static void canon(const Scene &S, int type, int a, int b, int32_t *k)
{
    k[0] = type;
    if (type == PT) {
        int t[3] = {S.h_st[3 * b], S.h_st[3 * b + 1], S.h_st[3 * b + 2]};
        std::sort(t, t + 3);
        k[1] = a;
        k[2] = t[0];
        k[3] = t[1];
        k[4] = t[2];
    } else {
        k[1] = S.h_se[2 * a];
        k[2] = S.h_se[2 * a + 1];
        k[3] = S.h_se[2 * b];
        k[4] = S.h_se[2 * b + 1];
    }
}

static int find_edge(const Scene &S, int a, int b)
{
    int lo = 0, hi = S.nse - 1;
    while (lo <= hi) {
        const int m = (lo + hi) / 2;
        const int ma = S.h_se[2 * m], mb = S.h_se[2 * m + 1];
        if (ma == a && mb == b) return m;
        if (ma < a || (ma == a && mb < b)) lo = m + 1;
        else hi = m - 1;
    }
    return -1;
}

static int4 host_pair_verts(const Scene &S, int type, int a, int b)
{
    if (type == PT) return make_int4(a, S.h_st[3 * b], S.h_st[3 * b + 1], S.h_st[3 * b + 2]);
    return make_int4(S.h_se[2 * a], S.h_se[2 * a + 1], S.h_se[2 * b], S.h_se[2 * b + 1]);
}

}  // namespace bf

using namespace bf;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
#define SCENE_OR_ARG(p)             \
    if (!(p)) return BF_E_ARG;      \
    Scene &S = (p)->s

extern "C" {

int bf_scene_create(const bf_mesh_desc *mesh, const bf_params *params, const bf_allocator *alloc, void *stream,
                    bf_scene **out)
{
    if (!mesh || !params || !out) return BF_E_ARG;
    *out = nullptr;
    bf_scene *h = new bf_scene();
    Scene &S = h->s;
    S.stream = (cudaStream_t)stream;
    if (alloc && alloc->alloc && alloc->free) {
        S.alloc = *alloc;
        S.has_alloc = true;
    }
    const int st = create(S, mesh, params);
    if (st) {
        destroy(S);
        delete h;
        return st;
    }
    *out = h;
    return BF_OK;
}

int bf_scene_destroy(bf_scene *scene)
{
    if (!scene) return BF_E_ARG;
    destroy(scene->s);
    delete scene;
    return BF_OK;
}

int bf_set_sync_mode(bf_scene *scene, int32_t blocking)
{
    SCENE_OR_ARG(scene);
    if (blocking && !S.sync_ev &&
        cudaEventCreateWithFlags(&S.sync_ev, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
        S.sync_ev = nullptr;
        return BF_E_CUDA;
    }
    S.sync_blocking = blocking != 0;
    return BF_OK;
}

int bf_set_stream(bf_scene *scene, void *stream)
{
    SCENE_OR_ARG(scene);
    cudaStreamSynchronize(S.stream);
    S.stream = (cudaStream_t)stream;
    return BF_OK;
}

int bf_scene_bytes(bf_scene *scene, int64_t *bytes)
{
    SCENE_OR_ARG(scene);
    if (!bytes) return BF_E_ARG;
    *bytes = (int64_t)S.bytes;
    return BF_OK;
}

int bf_step(bf_scene *scene, int32_t n_steps, bf_step_stats *stats)
{
    SCENE_OR_ARG(scene);
    if (n_steps < 0) return BF_E_ARG;
    for (int i = 0; i < n_steps; ++i) {
        bf_step_stats st{};
        const int rc = step_once(S, &st);
        if (stats) stats[i] = st;
        if (rc) return rc;
    }
    return BF_OK;
}

int bf_step_host(bf_scene *scene, const double *x_in, const double *v_in, double *x_out, double *v_out,
                 bf_step_stats *stats)
{
    SCENE_OR_ARG(scene);
    const size_t nb = 3 * (size_t)S.nv * sizeof(double);
    if (x_in) cudaMemcpyAsync(S.x, x_in, nb, cudaMemcpyHostToDevice, S.stream);
    if (v_in) cudaMemcpyAsync(S.v, v_in, nb, cudaMemcpyHostToDevice, S.stream);
    int rc = step_once(S, stats);
    if (rc) return rc;
    if (x_out) cudaMemcpyAsync(x_out, S.x, nb, cudaMemcpyDeviceToHost, S.stream);
    if (v_out) cudaMemcpyAsync(v_out, S.v, nb, cudaMemcpyDeviceToHost, S.stream);
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_get_state(bf_scene *scene, double *x, double *v)
{
    SCENE_OR_ARG(scene);
    const size_t nb = 3 * (size_t)S.nv * sizeof(double);
    if (x) cudaMemcpyAsync(x, S.x, nb, cudaMemcpyDeviceToHost, S.stream);
    if (v) cudaMemcpyAsync(v, S.v, nb, cudaMemcpyDeviceToHost, S.stream);
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_set_state(bf_scene *scene, const double *x, const double *v)
{
    SCENE_OR_ARG(scene);
    const size_t nb = 3 * (size_t)S.nv * sizeof(double);
    if (x) cudaMemcpyAsync(S.x, x, nb, cudaMemcpyHostToDevice, S.stream);
    if (v) cudaMemcpyAsync(S.v, v, nb, cudaMemcpyHostToDevice, S.stream);
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_set_obstacle_targets(bf_scene *scene, const double *targets)
{
    SCENE_OR_ARG(scene);
    if (!targets) {
        S.has_targets = 0;
        return BF_OK;
    }
    if (S.ndir == 0) return BF_E_ARG;
    cudaMemcpyAsync(S.targets, targets, 3 * (size_t)S.ndir * sizeof(double), cudaMemcpyHostToDevice, S.stream);
    S.has_targets = 1;
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_get_active_set(bf_scene *scene, int32_t cap, int32_t *n, int32_t *keys, double *lam, double *gam)
{
    SCENE_OR_ARG(scene);
    if (n) *n = S.nc;
    const int m = std::min(cap, S.nc);
    if (m <= 0) return BF_OK;
    std::vector<int> t(m), a(m), b(m);
    std::vector<double> l(m), g(m);
    cudaMemcpyAsync(t.data(), S.ctype, m * 4, cudaMemcpyDeviceToHost, S.stream);
    cudaMemcpyAsync(a.data(), S.ca, m * 4, cudaMemcpyDeviceToHost, S.stream);
    cudaMemcpyAsync(b.data(), S.cb, m * 4, cudaMemcpyDeviceToHost, S.stream);
    cudaMemcpyAsync(l.data(), S.clam, m * 8, cudaMemcpyDeviceToHost, S.stream);
    cudaMemcpyAsync(g.data(), S.cgam, m * 8, cudaMemcpyDeviceToHost, S.stream);
    const int st = check_cuda(cudaStreamSynchronize(S.stream));
    if (st) return st;
    for (int i = 0; i < m; ++i) {
        if (keys) canon(S, t[i], a[i], b[i], keys + 5 * i);
        if (lam) lam[i] = l[i];
        if (gam) gam[i] = g[i];
    }
    return BF_OK;
}

int bf_set_active_set(bf_scene *scene, int32_t n, const int32_t *keys, const double *lam, const double *gam)
{
    SCENE_OR_ARG(scene);
    if (n < 0 || (n > 0 && (!keys || !lam || !gam))) return BF_E_ARG;
    std::vector<int> t(n), a(n), b(n);
    std::vector<int4> v(n);
    for (int i = 0; i < n; ++i) {
        const int32_t *k = keys + 5 * i;
        if (k[0] == PT) {
            const long long key = tri_key_sorted(k[2], k[3], k[4]);
            auto it = std::lower_bound(S.h_tri_key_sorted.begin(), S.h_tri_key_sorted.end(), key);
            if (it == S.h_tri_key_sorted.end() || *it != key) return BF_E_NOT_FOUND;
            t[i] = PT;
            a[i] = k[1];
            b[i] = S.h_tri_key_idx[it - S.h_tri_key_sorted.begin()];
            if (a[i] < 0 || a[i] >= S.nv) return BF_E_NOT_FOUND;
        } else if (k[0] == EE) {
            t[i] = EE;
            a[i] = find_edge(S, k[1], k[2]);
            b[i] = find_edge(S, k[3], k[4]);
            if (a[i] < 0 || b[i] < 0) return BF_E_NOT_FOUND;
            if (a[i] > b[i]) std::swap(a[i], b[i]);
        } else {
            return BF_E_ARG;
        }
        v[i] = host_pair_verts(S, t[i], a[i], b[i]);
    }
    S.nc = 0;
    int st = active_reserve(S, std::max(n, 1));
    if (st) return st;
    if (n) {
        cudaMemcpyAsync(S.ctype, t.data(), n * 4, cudaMemcpyHostToDevice, S.stream);
        cudaMemcpyAsync(S.ca, a.data(), n * 4, cudaMemcpyHostToDevice, S.stream);
        cudaMemcpyAsync(S.cb, b.data(), n * 4, cudaMemcpyHostToDevice, S.stream);
        cudaMemcpyAsync(S.cv, v.data(), n * 16, cudaMemcpyHostToDevice, S.stream);
        cudaMemcpyAsync(S.clam, lam, n * 8, cudaMemcpyHostToDevice, S.stream);
        cudaMemcpyAsync(S.cgam, gam, n * 8, cudaMemcpyHostToDevice, S.stream);
    }
    S.nc = n;
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_get_mu(bf_scene *scene, double *mu, double *delta)
{
    SCENE_OR_ARG(scene);
    if (mu) *mu = S.mu;
    if (delta) *delta = S.delta;
    return BF_OK;
}

// checkpoint layout: header (8 int64: magic, version, n_verts, n_pairs,
// whether obstacle targets are set, n_prescribed, 2 reserved), mu, delta,
// x (3 n_verts), v (3 n_verts), the pairs' lambdas, their gammas, the
// obstacle targets (3 n_prescribed) when set, then the pairs' 5-int keys
// (every double stays 8-byte aligned)
static const int64_t kCheckpointMagic = 0x4b43435f4642LL;  // "BF_CCK"

static size_t checkpoint_bytes(int nv, int nc, int ntarget)
{
    return 8 * sizeof(int64_t) + 2 * sizeof(double) + 6 * (size_t)nv * sizeof(double) +
           (size_t)nc * (5 * sizeof(int32_t) + 2 * sizeof(double)) + 3 * (size_t)ntarget * sizeof(double);
}

int bf_save(bf_scene *scene, void *buf, size_t cap, size_t *used)
{
    SCENE_OR_ARG(scene);
    if (!used) return BF_E_ARG;
    const int ntarget = S.has_targets ? S.ndir : 0;
    const size_t need = checkpoint_bytes(S.nv, S.nc, ntarget);
    *used = need;
    if (!buf) return BF_OK;  // size query
    if (cap < need) return BF_E_CAPACITY;
    unsigned char *p = (unsigned char *)buf;
    const int64_t hdr[8] = {kCheckpointMagic, 1, S.nv, S.nc, S.has_targets ? 1 : 0, S.ndir, 0, 0};
    std::memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    double md[2] = {S.mu, S.delta};
    std::memcpy(p, md, sizeof(md));
    p += sizeof(md);
    double *x = (double *)p, *v = x + 3 * (size_t)S.nv;
    int st = bf_get_state(scene, x, v);
    if (st) return st;
    p += 6 * (size_t)S.nv * sizeof(double);
    double *lam = (double *)p, *gam = lam + S.nc, *tgt = gam + S.nc;
    int32_t *keys = (int32_t *)(tgt + 3 * (size_t)ntarget);
    int32_t n = 0;
    st = bf_get_active_set(scene, S.nc, &n, keys, lam, gam);
    if (st || !ntarget) return st;
    cudaMemcpyAsync(tgt, S.targets, 3 * (size_t)ntarget * sizeof(double), cudaMemcpyDeviceToHost, S.stream);
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_load(bf_scene *scene, const void *buf, size_t size)
{
    SCENE_OR_ARG(scene);
    if (!buf || size < 8 * sizeof(int64_t)) return BF_E_ARG;
    const unsigned char *p = (const unsigned char *)buf;
    int64_t hdr[8];
    std::memcpy(hdr, p, sizeof(hdr));
    if (hdr[0] != kCheckpointMagic || hdr[1] != 1 || hdr[2] != S.nv || hdr[3] < 0 || hdr[3] > (1 << 30) ||
        (hdr[4] != 0 && hdr[4] != 1) || hdr[5] != S.ndir)
        return BF_E_ARG;
    const int nc = (int)hdr[3], ntarget = hdr[4] ? S.ndir : 0;
    if (size < checkpoint_bytes(S.nv, nc, ntarget)) return BF_E_ARG;
    p += sizeof(hdr);
    double md[2];
    std::memcpy(md, p, sizeof(md));
    p += sizeof(md);
    const double *x = (const double *)p, *v = x + 3 * (size_t)S.nv;
    int st = bf_set_state(scene, x, v);
    if (st) return st;
    p += 6 * (size_t)S.nv * sizeof(double);
    const double *lam = (const double *)p, *gam = lam + nc, *tgt = gam + nc;
    const int32_t *keys = (const int32_t *)(tgt + 3 * (size_t)ntarget);
    st = bf_set_active_set(scene, nc, keys, lam, gam);
    if (st) return st;
    st = bf_set_obstacle_targets(scene, ntarget ? tgt : nullptr);
    if (st || !(md[0] > 0.0)) return st;  // mu is 0 until a scene's first step
    return bf_set_mu(scene, md[0], md[1]);
}

int bf_set_mu(bf_scene *scene, double mu, double delta)
{
    SCENE_OR_ARG(scene);
    if (!(mu > 0.0) || delta < 0.0) return BF_E_ARG;
    S.mu = mu;
    S.delta = delta;
    return BF_OK;
}

int bf_scene_info(bf_scene *scene, int32_t *info)
{
    SCENE_OR_ARG(scene);
    if (!info) return BF_E_ARG;
    info[0] = S.nsv;
    info[1] = S.nst;
    info[2] = S.nse;
    info[3] = S.nnzb;
    info[4] = S.ndir;
    return BF_OK;
}

const char *bf_status_str(int status)
{
    switch (status) {
    case BF_OK: return "ok";
    case BF_E_ARG: return "invalid argument";
    case BF_E_OOM: return "device allocation failed";
    case BF_E_CUDA: return "CUDA error";
    case BF_E_CG_MAXIT: return "PCG reached max_cg";
    case BF_E_NEWTON_MAXIT: return "Newton loop reached max_newton";
    case BF_E_LS_FAIL: return "line search failed";
    case BF_E_OUTER_MAXIT: return "time step reached max_outer";
    case BF_E_NONFINITE: return "non-finite value";
    case BF_E_CAPACITY: return "work buffer capacity exceeded";
    case BF_E_NOT_FOUND: return "pair key or ticket not found";
    case BF_E_BUDGET: return "HBM budget exceeded";
    default: return "unknown status";
    }
}

int bf_xtilde(bf_scene *scene, double *xtilde)
{
    SCENE_OR_ARG(scene);
    if (!xtilde) return BF_E_ARG;
    launch_xtilde(S, xtilde);
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_mu_init(bf_scene *scene, const double *xtilde, const double *xhat, double *mu)
{
    SCENE_OR_ARG(scene);
    if (!xtilde || !xhat) return BF_E_ARG;
    const double m = mu_init(S, xtilde, xhat);
    if (mu) *mu = m;
    return std::isfinite(m) && m > 0 ? BF_OK : BF_E_NONFINITE;
}

int bf_linearize(bf_scene *scene, const double *xlin, double *dist, double *grad)
{
    SCENE_OR_ARG(scene);
    if (!xlin) return BF_E_ARG;
    launch_linearize_out(S, xlin, dist, grad);
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_assemble(bf_scene *scene, const double *xtilde, const double *xlin, const double *xhat, double *grad,
                double *energy)
{
    SCENE_OR_ARG(scene);
    if (!xtilde || !xlin || !xhat) return BF_E_ARG;
    S.elastic_ready = false;
    if (!(S.mu > 0.0)) return BF_E_ARG;
    int st = assemble(S, xtilde, xlin, xhat);
    if (st) return st;
    if (grad) cudaMemcpyAsync(grad, S.grad, 3 * (size_t)S.nv * 8, cudaMemcpyDeviceToDevice, S.stream);
    if (energy) {
        *energy = run_energy(S, xtilde, xlin, xhat);
    }
    st = sync_flags(S);
    if (st) return st;
    return (S.h_flag[F_ERR] & ERR_NONFINITE) ? BF_E_NONFINITE : BF_OK;
}

int bf_friction_setup(bf_scene *scene, int32_t *n_pairs)
{
    SCENE_OR_ARG(scene);
    const int st = friction_setup(S);
    if (n_pairs) *n_pairs = S.nf;
    return st;
}

int bf_friction_get(bf_scene *scene, int32_t cap, int32_t *n, int32_t *v4, double *w4, double *n3, double *k)
{
    SCENE_OR_ARG(scene);
    if (n) *n = S.nf;
    const int m = std::min(cap, S.nf);
    if (m <= 0) return BF_OK;
    if (v4) cudaMemcpyAsync(v4, S.fv, (size_t)m * sizeof(int4), cudaMemcpyDeviceToHost, S.stream);
    if (w4) cudaMemcpyAsync(w4, S.fw, 4 * (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, S.stream);
    if (n3) cudaMemcpyAsync(n3, S.fn, 3 * (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, S.stream);
    if (k) cudaMemcpyAsync(k, S.fk, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, S.stream);
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_hess_apply(bf_scene *scene, const double *x, double *y)
{
    SCENE_OR_ARG(scene);
    if (!x || !y) return BF_E_ARG;
    launch_spmv(S, x, y, false, nullptr);
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_get_bsr(bf_scene *scene, int32_t *row_ptr, int32_t *col, double *val)
{
    SCENE_OR_ARG(scene);
    if (row_ptr) std::memcpy(row_ptr, S.h_rowptr.data(), (S.nv + 1) * 4);
    if (col) std::memcpy(col, S.h_col.data(), (size_t)S.nnzb * 4);
    if (val) {
        std::vector<double> planes(9 * (size_t)S.nnzb);
        if (S.prm.precision == BF_PREC_MIXED) {
            std::vector<float> pf(9 * (size_t)S.nnzb);
            cudaMemcpyAsync(pf.data(), S.valf, pf.size() * 4, cudaMemcpyDeviceToHost, S.stream);
            cudaStreamSynchronize(S.stream);
            for (size_t i = 0; i < pf.size(); ++i) planes[i] = pf[i];
        } else {
            cudaMemcpyAsync(planes.data(), S.val, planes.size() * 8, cudaMemcpyDeviceToHost, S.stream);
        }
        const int st = check_cuda(cudaStreamSynchronize(S.stream));
        if (st) return st;
        for (int k = 0; k < S.nnzb; ++k)
            for (int e = 0; e < 9; ++e) val[9 * (size_t)k + e] = planes[9 * (size_t)k + e];
    }
    return BF_OK;
}

int bf_pcg(bf_scene *scene, const double *b, double *x, double tol, int32_t maxit, int32_t *iters)
{
    SCENE_OR_ARG(scene);
    if (!b || !x || !(tol > 0) || maxit < 1) return BF_E_ARG;
    int it = 0;
    const int st = run_pcg(S, b, x, tol, maxit, &it);
    if (iters) *iters = it;
    return st;
}

int bf_energy(bf_scene *scene, const double *xtilde, const double *xlin, const double *xhat, double *L)
{
    SCENE_OR_ARG(scene);
    if (!xtilde || !xlin || !xhat || !L) return BF_E_ARG;
    *L = run_energy(S, xtilde, xlin, xhat);
    return std::isfinite(*L) ? BF_OK : BF_E_NONFINITE;
}

int bf_solve_subproblem(bf_scene *scene, const double *xtilde, const double *xlin, double *xhat, int32_t *newton,
                        int32_t *cg)
{
    SCENE_OR_ARG(scene);
    if (!xtilde || !xlin || !xhat || !(S.mu > 0)) return BF_E_ARG;
    S.elastic_ready = false;
    SolveStats ss;
    S.L_scale = -1.0;  // called alone: the scale comes from this call's first iterate
    const int st = solve_subproblem(S, xtilde, xlin, xhat, ss);
    if (newton) *newton = ss.newton;
    if (cg) *cg = ss.cg;
    if (st) return st;
    return check_cuda(cudaStreamSynchronize(S.stream));
}

int bf_ccd_hits(bf_scene *scene, const double *x0, const double *x1, int32_t cap, int32_t *n, int32_t *keys,
                double *toi)
{
    SCENE_OR_ARG(scene);
    if (!x0 || !x1) return BF_E_ARG;
    int nh = 0;
    int st = run_ccd(S, x0, x1, true, nullptr, &nh);
    if (st) return st;
    if (n) *n = nh;
    const int m = std::min(cap, nh);
    if (m <= 0) return BF_OK;
    std::vector<int> t(m), a(m), b(m);
    std::vector<double> tt(m);
    cudaMemcpyAsync(t.data(), S.hit_type, m * 4, cudaMemcpyDeviceToHost, S.stream);
    cudaMemcpyAsync(a.data(), S.hit_a, m * 4, cudaMemcpyDeviceToHost, S.stream);
    cudaMemcpyAsync(b.data(), S.hit_b, m * 4, cudaMemcpyDeviceToHost, S.stream);
    cudaMemcpyAsync(tt.data(), S.hit_toi, m * 8, cudaMemcpyDeviceToHost, S.stream);
    st = check_cuda(cudaStreamSynchronize(S.stream));
    if (st) return st;
    for (int i = 0; i < m; ++i) {
        if (keys) canon(S, t[i], a[i], b[i], keys + 5 * i);
        if (toi) toi[i] = tt[i];
    }
    return BF_OK;
}

int bf_update_active_set(bf_scene *scene, const double *x, const double *xhat, int32_t *n_active)
{
    SCENE_OR_ARG(scene);
    if (!x || !xhat) return BF_E_ARG;
    const int st = run_update_active_set(S, x, xhat);
    if (n_active) *n_active = S.nc;
    return st;
}

int bf_max_step_size(bf_scene *scene, const double *x0, const double *x1, double *alpha)
{
    SCENE_OR_ARG(scene);
    if (!x0 || !x1 || !alpha) return BF_E_ARG;
    return run_ccd(S, x0, x1, false, alpha, nullptr);
}

int bf_newton_residual(bf_scene *scene, const double *xtilde, const double *x, double *res)
{
    SCENE_OR_ARG(scene);
    if (!xtilde || !x || !res || !(S.mu > 0) || S.nv < 1) return BF_E_ARG;
    return newton_residual(S, xtilde, x, res);
}

int bf_get_residual_log(bf_scene *scene, int32_t cap, int32_t *n, double *out)
{
    SCENE_OR_ARG(scene);
    if (cap < 0 || (cap > 0 && !out)) return BF_E_ARG;
    const int m = (int)S.res_log.size();
    for (int i = 0; i < m && i < cap; ++i) out[i] = S.res_log[i];
    if (n) *n = m;
    return BF_OK;
}

int bf_inversion_step(bf_scene *scene, const double *x0, const double *x1, double *alpha)
{
    SCENE_OR_ARG(scene);
    if (!x0 || !x1 || !alpha) return BF_E_ARG;
    const double one = 1.0;
    int st = check_cuda(cudaMemcpyAsync(S.dscal + S_TOI, &one, sizeof(double), cudaMemcpyHostToDevice, S.stream));
    if (st) return st;
    launch_inversion_bound(S, x0, x1, S.dscal + S_TOI);
    st = sync_flags(S);
    if (st) return st;
    *alpha = std::min(1.0, S.h_scal[S_TOI]);
    return BF_OK;
}

int bf_accd(int32_t type, int32_t n, const double *x0, const double *x1, double s, double *toi, void *stream)
{
    if ((type != PT && type != EE) || n < 0 || (n > 0 && (!x0 || !x1 || !toi)) || !(s > 0 && s < 1))
        return BF_E_ARG;
    const int st = accd_pairs(type, n, x0, x1, s, toi, (cudaStream_t)stream);
    if (st) return st;
    return check_cuda(cudaStreamSynchronize((cudaStream_t)stream));
}

int bf_enable_timers(bf_scene *scene, int32_t on)
{
    SCENE_OR_ARG(scene);
    S.timers_on = on != 0;
    for (int i = 0; i < T_N; ++i) {
        S.t_launch[i] = 0;
        S.t_ms[i] = 0.0;
    }
    return BF_OK;
}

int bf_test_pcg_barrier_fail(bf_scene *scene, int32_t on)
{
    SCENE_OR_ARG(scene);
    S.pcg_bar_fail = on ? 1 : 0;
    return BF_OK;
}

int bf_set_pcg_mode(bf_scene *scene, int32_t mode)
{
    SCENE_OR_ARG(scene);
    if (mode < 0 || mode > 511) return BF_E_ARG;
    S.pcg_mode = mode == 0 ? 0 : 1;
    if (mode > 0) {
        S.pcg_ctas_per_sm = mode & 15;
        S.pcg_allow_resident = (mode & 16) ? 0 : 1;
        S.pcg_force_global = (mode & 32) ? 1 : 0;
        S.pcg_no_sym = (mode & 64) ? 1 : 0;
        S.pcg_cg1 = (mode & 128) ? 0 : 1;
        S.pcg_no_cache = (mode & 256) ? 1 : 0;
        S.pcg_grid = 0;  // recomputed at the next solve
    }
    return BF_OK;
}

// PCG autotuner: on the system assembled last, times `iters` iterations of
// each candidate execution configuration with CUDA events on the scene's
// stream (after one untimed solve that sets the configuration up and warms
// it) and keeps the fastest per iteration; the right-hand side is all ones
// (a converged gradient would end the solves at once).  A persistent
// candidate that falls back to the per-phase launches (no fitting
// partition) is skipped.  Candidates come in order of preference (the
// default first); a later one replaces the choice only when it is more
// than 2 % faster, so timing noise does not flip the configuration.
int bf_autotune_pcg(bf_scene *scene, int32_t iters, int32_t cap, int32_t *modes, double *us_per_iter,
                    int32_t *n_out, int32_t *best)
{
    SCENE_OR_ARG(scene);
    if (iters < 8 || cap < 0 || (cap > 0 && (!modes || !us_per_iter)) || !best || S.nv < 1) return BF_E_ARG;
    static const int kCand[] = {1, 2, 129, 130, 17, 18, 33, 34, 97, 98, 0};
    const int n = 3 * S.nv;
    const int keep_mode = S.pcg_mode == 0 ? 0
                          : (S.pcg_ctas_per_sm | (S.pcg_allow_resident ? 0 : 16) | (S.pcg_force_global ? 32 : 0) |
                             (S.pcg_no_sym ? 64 : 0) | (S.pcg_cg1 ? 0 : 128) | (S.pcg_no_cache ? 256 : 0));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return BF_E_CUDA;
    }
    int nt = 0, best_mode = -1;
    double best_us = 0.0;
    int st = BF_OK;
    k_fill<<<cdiv(n, kThreads), kThreads, 0, S.stream>>>(n, S.cg_b, 1.0);
    ++S.n_launch;
    for (int mode : kCand) {
        bf_set_pcg_mode(scene, mode);
        int it = 0;
        st = run_pcg(S, S.cg_b, S.pdir, 1e-30, std::max(1, iters / 4), &it);  // set-up and warm-up
        if (st && st != BF_E_CG_MAXIT) break;
        st = BF_OK;
        if (mode != 0 && S.pcg_mode == 0) continue;  // did not fit: fell back to the per-phase launches
        if ((mode & 128) && S.pcg_resident != 1) continue;  // not resident: the same as mode & 127
        cudaEventRecord(e0, S.stream);
        int st2 = run_pcg(S, S.cg_b, S.pdir, 1e-30, iters, &it);
        cudaEventRecord(e1, S.stream);
        if (st2 && st2 != BF_E_CG_MAXIT) {
            st = st2;
            break;
        }
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = BF_E_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (it < iters / 2) continue;  // stopped early (breakdown): no usable timing
        const double us = 1e3 * ms / it;
        if (nt < cap) {
            modes[nt] = mode;
            us_per_iter[nt] = us;
        }
        ++nt;
        if (best_mode < 0 || us < 0.98 * best_us) {
            best_mode = mode;
            best_us = us;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bf_set_pcg_mode(scene, best_mode >= 0 ? best_mode : keep_mode);
    if (n_out) *n_out = nt;
    *best = best_mode;
    if (st) return st;
    return best_mode >= 0 ? BF_OK : BF_E_ARG;
}

int bf_get_pcg_config(bf_scene *scene, int32_t *cfg)
{
    SCENE_OR_ARG(scene);
    if (!cfg) return BF_E_ARG;
    cfg[0] = S.pcg_mode;
    cfg[1] = S.pcg_grid;
    cfg[2] = S.pcg_block;
    cfg[3] = S.pcg_smem;
    cfg[4] = S.pcg_resident;
    cfg[5] = S.pcg_max_rows;
    cfg[6] = S.pcg_max_ent;
    cfg[7] = S.pcg_max_win;
    return BF_OK;
}

int bf_get_launch_count(bf_scene *scene, int64_t *n)
{
    SCENE_OR_ARG(scene);
    if (!n) return BF_E_ARG;
    *n = S.n_launch;
    return BF_OK;
}

int bf_get_timers(bf_scene *scene, int32_t cap, int64_t *launches, double *ms, const char **names)
{
    SCENE_OR_ARG(scene);
    cudaStreamSynchronize(S.stream);
    flush_timers(S);
    for (int i = 0; i < T_N && i < cap; ++i) {
        if (launches) launches[i] = S.t_launch[i];
        if (ms) ms[i] = S.t_ms[i];
        if (names) names[i] = kTimerNames[i];
    }
    return T_N;
}

}  // extern "C"
