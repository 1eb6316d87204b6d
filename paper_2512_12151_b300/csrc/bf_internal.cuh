// Internal declarations of the CUDA library behind include/bf.h.
//
// Data layout in HBM (one scene):
//  - positions / velocities / gradients: (nv, 3) FP64 AoS;
//  - tets: int4; Dm^-1 as 9 FP64 per tet; per-tet Lame parameters and rest
//    volume; tblk: for each tet its 10 upper 3x3 blocks (i' <= j') as BSR
//    block indices, bit 31 set when the block is stored transposed;
//  - Hessian: upper block-sparse rows (diagonal + upper blocks of the
//    elastic / mass pattern), 3x3 blocks stored contiguously (9 values,
//    FP64, or FP32 in mixed precision); a full-row view (frowptr, fnbr,
//    fblk: every block of a vertex row, upper ones and transposed lower
//    ones) serves the row-gather SpMV of the PCG; contact terms stay rank-1
//    per pair (mu gamma_i g_i g_i^T) and are applied matrix-free;
//  - active set: SoA arrays (type, prim a, prim b, 4 vertex ids, lambda,
//    gamma, d, 12 gradient entries, slack, free-vertex mask).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "bf.h"

namespace bf {

enum { PT = 0, EE = 1 };

// device scalar slots (dscal)
enum {
    S_RZ = 0, S_BB, S_ALPHA, S_BETA, S_RR, S_PQ, S_E0, S_E1, S_MU, S_TOI, S_DOT, S_MAXDIAG,
    S_T_SPMV, S_T_RED1, S_T_UPD, S_T_RED2, S_RES = 16,  // S_RES..S_RES+23: reduction accumulators
    S_T_STAGE = 40, S_T_ROWS, S_T_CONTACT, S_GNORM, S_RESID,
    S_NSCAL = 48
};
// device flag slots (dflag)
enum {
    F_DONE = 0, F_ITERS, F_ERR, F_MAXIT, F_NCAND_PT, F_NCAND_EE, F_NHIT, F_NKEEP, F_NSCRATCH, F_NFRIC,
    F_NFLAG = 32
};
// error bits in dflag[F_ERR]
enum { ERR_NONFINITE = 1, ERR_CAND_OVERFLOW = 2, ERR_HIT_OVERFLOW = 4, ERR_PQ = 8, ERR_BARRIER = 16 };

enum TimerId { T_ELASTIC = 0, T_SPMV, T_PCG_UPDATE, T_PCG_DIR, T_CONTACT, T_ENERGY, T_CCD_NARROW,
               T_BVH, T_PCG_PERSISTENT, T_PCG_PH_SPMV, T_PCG_PH_RED1, T_PCG_PH_UPD, T_PCG_PH_RED2,
               T_PCG_PH_STAGE, T_PCG_PH_ROWS, T_PCG_PH_CONTACT, T_CCD_QUERY, T_N };

struct LBVH {
    int n = 0, cap = 0, npad = 0;  // leaves, capacity, leaves padded to a power of two
    unsigned *morton = nullptr, *morton_alt = nullptr;
    int *prim = nullptr, *prim_alt = nullptr;  // primitive of each leaf (Morton order)
    double *lo = nullptr, *hi = nullptr;    // exact leaf boxes in leaf order, 3 each
    double *plo = nullptr, *phi = nullptr;  // exact primitive boxes, 3 per primitive
    float4 *node = nullptr;  // implicit tree: node h at node[2h] (lo), node[2h + 1] (hi), FP32 outward-rounded
    int topo_valid = 0;      // the leaf order may be kept and only the boxes recomputed
};

struct Scene {
    int nv = 0, nt = 0, nm = 0, nx = 0, ndir = 0;
    int nsv = 0, nst = 0, nse = 0, nnzb = 0;
    bf_params prm{};
    double mu = 0.0, delta = 0.0;
    double L_scale = -1.0;  // |L| at the time step's first Newton iterate (< 0: unset)
    std::vector<double> res_log;  // gradient-norm residuals of the last step (residual mode)
    // the step's mu_init left the inertia and elastic parts of G and H at
    // the first Newton iterate: the next assembly adds only the rest
    bool elastic_ready = false;
    // host waits sleep on a blocking-sync event instead of spinning
    // (scenes of a batch: many worker threads share the host cores)
    bool sync_blocking = false;
    cudaEvent_t sync_ev = nullptr;
    int has_targets = 0;
    cudaStream_t stream = nullptr;
    bf_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> owned;
    std::vector<size_t> owned_bytes;  // size of each owned allocation
    size_t bytes = 0;                 // device bytes the scene holds

    // host topology
    std::vector<int> h_sv, h_st, h_se, h_rowptr, h_col;
    std::vector<uint8_t> h_dir;
    std::vector<int> h_dir_ids;
    std::vector<long long> h_tri_key_sorted;  // sorted-vertex triangle keys, ascending
    std::vector<int> h_tri_key_idx;

    // device state
    double *x = nullptr, *v = nullptr, *xt = nullptr, *xtilde = nullptr, *xk = nullptr,
           *xh = nullptr, *xh_prev = nullptr, *xtmp = nullptr, *targets = nullptr;
    uint8_t *dir = nullptr;
    double *mass = nullptr;
    int4 *tets = nullptr;
    double *B = nullptr, *vol = nullptr, *emu = nullptr, *elam = nullptr;
    int *tblk = nullptr;
    int *rowptr = nullptr, *col = nullptr, *rowid = nullptr, *diagblk = nullptr;
    int nfull = 0;
    int *frowptr = nullptr, *fnbr = nullptr, *fblk = nullptr;  // full-row view
    std::vector<int> h_frowptr;
    int *part = nullptr;      // persistent PCG: CTA row ranges (grid + 1)
    int pcg_smem = 0;         // dynamic shared memory of the persistent PCG (bytes)
    int pcg_resident = 0;     // persistent PCG variant: 0 streamed via the BSR, 1 resident, 2 global vectors, 3 symmetric,
                              // 4 resident with one reduction per iteration
    double *val = nullptr;  // 9 planes FP64
    float *valf = nullptr;  // 9 planes FP32 (mixed)
    double *grad = nullptr;
    double *cdiag = nullptr;  // contact diagonal blocks (nv x 9) for the preconditioner
    double *pinv = nullptr;
    float *pinvf = nullptr;
    // PCG work vectors (n = 3 nv)
    double *cg_x = nullptr, *cg_r = nullptr, *cg_b = nullptr, *cg_p = nullptr, *cg_q = nullptr,
           *cg_z = nullptr, *pdir = nullptr;
    float *cg_pf = nullptr, *cg_qf = nullptr, *cg_zf = nullptr, *cg_pf2 = nullptr;
    double *cg_qc = nullptr;  // contact part of H p (accumulated with atomics)
    double *cg_p2 = nullptr;  // second direction buffer of the persistent PCG
    unsigned *bar = nullptr;  // grid barrier: count, generation
    int pcg_grid = 0;         // co-resident CTAs of the persistent PCG (0 = not set up)
    int pcg_mode = 1;         // 1 = persistent cooperative kernel, 0 = one launch per phase
    int pcg_ctas_per_sm = 1;  // persistent PCG: CTAs per SM (capped by occupancy)
    int pcg_allow_resident = 1;  // persistent PCG may keep the matrix in shared memory
    int pcg_force_global = 0;    // persistent PCG: use the global-vectors variant only
    int pcg_max_rows = 0, pcg_max_ent = 0, pcg_max_win = 0, pcg_block = 256;
    int pcg_slots_held = 0, pcg_slots_dev = 0;  // SM slots held by a launched persistent solve
    unsigned short *pcg_eslot = nullptr;  // persistent PCG: shared-memory slot of every full-row entry
    int *pcg_rinfo = nullptr, *pcg_lvl = nullptr, *pcg_lvlptr = nullptr;  // rows by length, level offsets
    int pcg_max_len = 0;
    int *pcg_edst = nullptr;              // persistent PCG, global variant: jagged position of each entry
    unsigned short *pcg_jnbr = nullptr;   // ... window offset of each jagged slot
    void *pcg_jval = nullptr;             // ... jagged copy of the blocks (9 planes)
    unsigned char *pcg_gvec = nullptr;    // ... per-CTA vectors
    size_t pcg_gvec_stride = 0;
    int pcg_kc = 0;               // persistent PCG: contacts per CTA cached in shared memory
    int pcg_no_sym = 0;           // persistent PCG: skip the symmetric (upper-only) variant
    int pcg_cg1 = 1;              // persistent PCG: single-reduction recurrence when the blocks are resident
    int pcg_no_cache = 0;         // persistent PCG: no contact pairs cached in shared memory
    int pcg_bar_fail = 0;         // persistent PCG: barriers poll an idle word (failure-detection test hook)
    unsigned char *pcg_cg1buf = nullptr;  // ... its published row sums, contact parts, (r, s) and H x
    int *pcg_uedst = nullptr;             // symmetric variant: jagged position of each upper block
    unsigned short *pcg_unbr = nullptr;   // ... window offset of each jagged slot
    float *pcg_uval = nullptr;            // ... jagged copy of the upper blocks (9 planes, FP32)
    float4 *pcg_yq = nullptr;             // ... transposed products and contact terms (one float4 per vertex)
    float *pcg_pp = nullptr;              // ... upper triangle of the block-Jacobi inverse, six planes
    float4 *pcg_z4 = nullptr;             // ... z = P r, one float4 per vertex
    int *win = nullptr;       // persistent PCG: staged vertex window per CTA
    std::vector<int> h_fnbr;
    // reductions
    double *partials = nullptr;
    int npartials = 0;
    unsigned *counter = nullptr;
    double *dscal = nullptr;
    int *dflag = nullptr;
    double *h_scal = nullptr;  // pinned mirrors
    int *h_flag = nullptr;

    // surface primitives
    int *sv = nullptr, *st = nullptr, *se = nullptr;

    // active set (capacity ccap)
    int nc = 0, ccap = 0;
    int *ctype = nullptr, *ca = nullptr, *cb = nullptr;
    int4 *cv = nullptr;
    double *clam = nullptr, *cgam = nullptr, *cd = nullptr, *cg = nullptr, *cs = nullptr,
           *cw = nullptr;
    unsigned char *cmask = nullptr;
    unsigned long long *ckey = nullptr, *ckey_sorted = nullptr;
    // CCD work
    LBVH bvh_tri, bvh_edge;
    bool bvh_reuse = false;  // within a time step: refit the trees instead of rebuilding them
    int cand_cap = 0;
    int2 *cand_pt = nullptr, *cand_ee = nullptr;
    // friction pairs of the time step (appendix A): vertices, closest-point
    // weights and unit normal at x^t (fx0), coefficient mu_f mu F, free mask
    int nf = 0, fcap = 0;
    int4 *fv = nullptr;
    double *fw = nullptr, *fn = nullptr, *fk = nullptr, *fx0 = nullptr;
    unsigned char *fmask = nullptr;
    int hit_cap = 0;
    int *hit_type = nullptr, *hit_a = nullptr, *hit_b = nullptr;
    double *hit_toi = nullptr;
    unsigned long long *hit_key = nullptr, *hit_key_alt = nullptr;
    int *hit_idx = nullptr, *hit_idx_alt = nullptr;
    unsigned long long *tv = nullptr;  // per-vertex min TOI bits
    int *keep = nullptr;
    void *cub_tmp = nullptr;
    size_t cub_tmp_bytes = 0;
    double *bounds = nullptr;  // Morton-code box (6 ordered ints)
    int *dir_ids = nullptr;    // prescribed vertex ids (ndir)

    // kernel launches issued by this scene (own kernels, not library sorts)
    long long n_launch = 0;
    // timers
    bool timers_on = false;
    int64_t t_launch[T_N] = {0};
    double t_ms[T_N] = {0};
    std::vector<cudaEvent_t> ev_pool;
};

// ---- memory ----
void *dev_alloc(Scene &S, size_t bytes);
void dev_free(Scene &S, void *p);

// ---- timers (per-kernel CUDA events on the scene's stream) ----
struct ScopedTimer {
    Scene *S;
    int id;
    cudaEvent_t a = nullptr, b = nullptr;
    ScopedTimer(Scene &s, int tid);
    ~ScopedTimer();
};
void flush_timers(Scene &S);

// ---- launchers: linear algebra (bf_linalg.cu) ----
void launch_zero(Scene &S, double *p, size_t n);
void launch_spmv(Scene &S, const double *x, double *y, bool with_dot, const int *done);
void launch_pinv(Scene &S);
int run_pcg(Scene &S, const double *b, double *x, double tol, int maxit, int *iters);
// rank-one terms of the Hessian applied by the PCG and the SpMV: the
// augmented-Lagrangian pairs, then two per friction pair
inline int n_terms(const Scene &S) { return S.nc + 2 * S.nf; }
int friction_setup(Scene &S);                              // at a time step's start
int launch_friction_assemble(Scene &S, const double *xhat);  // per Newton iteration
// Launches a solve whose completion the caller reads after its next
// sync_flags with pcg_finish (*pending = 1: the persistent kernel); when
// the solve had to complete here (*pending = 0) its status is returned.
int run_pcg_async(Scene &S, const double *b, double *x, double tol, int maxit, int *iters, int *pending);
int pcg_finish(Scene &S, int *iters);
void pcg_release(Scene &S);  // gives back the SM slots of a launched solve (error paths, destruction)
int run_pcg_persistent(Scene &S, const double *b, double *x, double tol, int maxit, int *iters);
void launch_axpy_to(Scene &S, double *out, const double *a, double r, const double *p, int n);
// out = a + r * (*scale) * p, scale on the device
void launch_axpy_scaled(Scene &S, double *out, const double *a, double r, const double *p, const double *scale,
                        int n);
void launch_blend(Scene &S, double *xk, const double *xh, double alpha, int n);
void launch_velocity(Scene &S);

// ---- launchers: elasticity (bf_elastic.cu) ----
void launch_vertex_init(Scene &S, const double *xtilde, const double *xhat);
void launch_elastic(Scene &S, const double *xhat);
double run_energy(Scene &S, const double *xtilde, const double *xlin, const double *xhat);
// L(xhat) into *out (device), no synchronisation
void launch_energy(Scene &S, const double *xtilde, const double *xlin, const double *xhat, double *out);
// one CCD along x0 -> x1 for both the active-set hits and the step bound
int run_ccd_reuse(Scene &S, const double *x0, const double *x1, int *nhits, double *alpha);
// inversion bound of MaxStepSize along x0 -> x1, min-reduced into *tmin
void launch_inversion_bound(Scene &S, const double *x0, const double *x1, double *tmin);
double run_mu_max_diag(Scene &S);
void launch_xtilde(Scene &S, double *xtilde);

// ---- launchers: contacts (bf_contact.cu) ----
void launch_contact_assemble(Scene &S, const double *xlin, const double *xhat);
void launch_multiplier_update(Scene &S, const double *xlin, const double *xhat);
void launch_contact_energy(Scene &S, const double *xlin, const double *xhat, double *partials,
                           int nblocks_offset);

// ---- launchers: CCD and active set (bf_ccd.cu) ----
void launch_linearize(Scene &S, const double *xlin);
int run_ccd(Scene &S, const double *x0, const double *x1, bool collect_hits, double *alpha_out,
            int *nhits_out);
int run_update_active_set(Scene &S, const double *x, const double *xhat);
// both CCD passes of an outer iteration from one broad phase: hits along
// x0 -> xa (collected, count to *nhits_a) and the TOI along x0 -> xb
int run_ccd_two(Scene &S, const double *x0, const double *xa, const double *xb, int *nhits_a, double *alpha_b);
// Alg. 3 on the hits collected by the last CCD pass
int apply_active_set_hits(Scene &S, int nh);
int accd_pairs(int type, int n, const double *x0, const double *x1, double s, double *toi,
               cudaStream_t st);
int ccd_reserve(Scene &S, int npt, int nee, int nhit);
int active_reserve(Scene &S, int n);

// ---- sync helpers ----
int sync_flags(Scene &S);  // copies dscal/dflag to host mirrors, returns CUDA status
int check_cuda(cudaError_t e);

inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }
constexpr int kThreads = 256;
constexpr int kAccdMaxIter = 100000;

}  // namespace bf
