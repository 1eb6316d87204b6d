/*
 * bf.h -- C ABI of the B300 (sm_103a) implementation of the inner Newton
 * step, active-set update and CCD of the barrier-free augmented-Lagrangian
 * (AL) contact method of "Robust and Efficient Penetration-Free
 * Elastodynamics without Barriers" (arXiv 2512.12151).
 *
 * Problem statement (section 3): linear tetrahedra with stacked positions
 * x and velocities v in R^{3N}, lumped mass M, implicit Euler through the
 * incremental potential E(x, x~) = 1/2 (x - x~)^T M (x - x~) + h^2 U(x),
 * x~ = x^t + h v^t + h^2 M^-1 f_ext, subject to a penetration-free path.
 * A time step (Alg. 1) alternates SolveSubproblem (Alg. 2, Newton on the AL
 * energy of Eq. total-energy), UpdateActiveSet (Alg. 3) and MaxStepSize
 * (CCD), blending x^[k+1] = (1 - alpha) x^[k] + alpha xhat^[k+1]
 * (Eq. CCD-clamp) until the first K_min blend weights sum below eps
 * (Eq. termination).
 *
 * Conventions for every entry point:
 *  - Status: every function returns an int; 0 is BF_OK, negative values are
 *    the BF_E_* codes below.  bf_status_str() names them.  Errors are per
 *    call; a device-side error word is latched per scene and reported by
 *    the next call that synchronises.
 *  - Layout: positions and velocities are (n, 3) row-major FP64 (x0 y0 z0
 *    x1 ...).  Pair keys are 5 int32: PT = {0, p, t0, t1, t2} with the
 *    triangle's vertex ids sorted ascending; EE = {1, a0, a1, b0, b1} with
 *    each edge's ids ascending and edge (a0, a1) < edge (b0, b1)
 *    lexicographically.
 *  - Memory: "host" arguments are caller-owned host buffers, copied during
 *    the call; "device" arguments are caller-owned device buffers on the
 *    scene's device, read or written on the scene's stream, and must stay
 *    valid until that stream reaches the call's work.  The library owns all
 *    scene state; it allocates it at creation through the optional
 *    allocator (else cudaMalloc) and frees it in bf_scene_destroy.
 *  - Threads: calls on one scene must not overlap; distinct scenes may be
 *    driven from different host threads.
 */
#ifndef BF_H
#define BF_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BF_OK 0
#define BF_E_ARG (-1)          /* invalid argument or size */
#define BF_E_OOM (-2)          /* device allocation failed */
#define BF_E_CUDA (-3)         /* CUDA runtime error */
#define BF_E_CG_MAXIT (-4)     /* PCG hit max_cg (result is the last iterate) */
#define BF_E_NEWTON_MAXIT (-5) /* Newton loop hit max_newton */
#define BF_E_LS_FAIL (-6)      /* line search found no decrease */
#define BF_E_OUTER_MAXIT (-7)  /* Alg. 1 loop hit max_outer */
#define BF_E_NONFINITE (-8)    /* NaN / Inf detected in a solve */
#define BF_E_CAPACITY (-9)     /* a work buffer overflowed and could not grow */
#define BF_E_NOT_FOUND (-10)   /* a pair key (or batch ticket) names nothing known */
#define BF_E_BUDGET (-11)      /* batch admission refused: the HBM budget would be exceeded */

#define BF_PREC_FP64 0  /* everything FP64 */
#define BF_PREC_MIXED 1 /* FP32 Hessian blocks (summed in FP64, stored in FP32) / SpMV /
                           preconditioner; FP64 gradient, dots, residuals, energies, CCD,
                           TOI and multipliers */

typedef struct bf_scene bf_scene;

/* Mesh (section 3).  Vertices with dirichlet[v] = 1 are prescribed
 * (section 5.3): obstacles are triangle meshes on such vertices.  tets are
 * positively oriented at rest; mats holds (E [Pa], nu, rho [kg/m^3]) per
 * material; tet_mat picks a material per tet. */
typedef struct {
    int32_t n_verts, n_tets, n_mats, n_obst_tris;
    const double *rest_pos;  /* host, n_verts*3 */
    const double *init_pos;  /* host, n_verts*3 */
    const double *init_vel;  /* host, n_verts*3 (may be NULL: zero) */
    const int32_t *tets;     /* host, n_tets*4 */
    const int32_t *tet_mat;  /* host, n_tets */
    const double *mats;      /* host, n_mats*3 */
    const int32_t *obst_tris;/* host, n_obst_tris*3 (vertex ids of prescribed vertices) */
    const uint8_t *dirichlet;/* host, n_verts (may be NULL: none) */
} bf_mesh_desc;

/* Solver parameters.  Paper defaults (section 6, Alg. 1-3): eps = 1e-3,
 * k_min = 2, gamma_decay (Gamma) = 0.9, c_mu (C of section 5.2) = 0.1.
 * s_ccd is the ACCD conservative rescaling (target gap s_ccd * d(x0)).
 * mu_f and eps_v [m/s] are the friction coefficient and the velocity
 * threshold of the smoothed semi-implicit friction of appendix A (mu_f = 0:
 * no friction; the paper uses k_min = 6 with friction).  res_tol > 0
 * replaces Eq. termination by the IPC-style criterion of section 6: a step's
 * outer loop ends once the gradient-norm residual (bf_newton_residual) at
 * x^[k] is below res_tol, checked before every outer iteration (0: off).
 * ccd_reuse = 1 updates the active set from the MaxStepSize segment
 * x^[k] -> xhat^[k+1] instead of Alg. 1's x^[k] -> xhat^[k], so one CCD
 * (one broad phase, one narrow pass) serves both per outer iteration and
 * the pairs that cut a step join C one iteration earlier (a CCD fitted to
 * the constraint-set expansion, the direction the paper's conclusion names;
 * 0: Alg. 1 as printed).  model selects the
 * material of every tet: BF_MODEL_SNH (stable Neo-Hookean, section 3),
 * BF_MODEL_COR (corotated linear) or BF_MODEL_NH (Neo-Hookean,
 * Psi = mu/2 (|F|^2 - 3) - mu ln J + lam/2 (ln J)^2, +inf for J <= 0),
 * the other models of Tab. 2.  NH is not defined for inverted elements, so
 * its MaxStepSize also bounds the step by element inversion (section 4.1;
 * bf_inversion_step), and a state with an inverted element makes its
 * energy infinite. */
enum { BF_MODEL_SNH = 0, BF_MODEL_COR = 1, BF_MODEL_NH = 2 };
typedef struct {
    double dt, delta, gravity[3], eps, cg_tol, gamma_decay, c_mu, s_ccd, mu_f, eps_v, res_tol;
    int32_t k_min, max_outer, max_newton, max_ls, max_cg, precision, model;
    int32_t ccd_reuse;
} bf_params;

/* Per-time-step statistics (the columns of Tab. 1 / Tab. 2). */
typedef struct {
    int32_t outer_iters, newton_iters, cg_iters, n_contacts, status, ls_fail, cg_maxit, stalls;
    double mean_alpha, min_alpha, mu, beta, delta, seconds;
} bf_step_stats;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns NULL on failure.  Both run on the calling host thread. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} bf_allocator;

/* ---- scene lifetime --------------------------------------------------- */

/* Creates a scene on the current CUDA device: copies the mesh, derives the
 * lumped mass m_v = sum_e rho V_e / 4 (prescribed vertices get mass 1 and
 * no elastic energy), Dm^-1, the surface (tet faces used once, plus the
 * obstacle triangles), the block-sparse pattern, and sizes work buffers.
 * stream: a cudaStream_t (NULL = default stream) used by all later calls.
 * Limits: n_verts < 2^21, n_tets < 2^29.
 * Errors: BF_E_ARG (bad sizes, ids out of range, degenerate tets), BF_E_OOM. */
int bf_scene_create(const bf_mesh_desc *mesh, const bf_params *params, const bf_allocator *alloc,
                    void *stream, bf_scene **out);
int bf_scene_destroy(bf_scene *scene);
int bf_set_stream(bf_scene *scene, void *stream);

/* Host waits of the scene's steps: 0 (default) synchronises the stream
 * (the waiting thread spins: lowest latency); 1 waits on a blocking-sync
 * event (the thread sleeps: for many worker threads sharing host cores). */
int bf_set_sync_mode(bf_scene *scene, int32_t blocking);

/* Checkpoint of the evolving state (no counterpart in the paper; lets a
 * server evict a scene and re-admit it later): positions, velocities, the
 * active set with multipliers and decay factors, mu and delta, and the
 * obstacle targets when set, in a self-describing host buffer (8-byte
 * aligned).  bf_save with buf NULL only sets *used to the bytes needed;
 * with cap too small it returns BF_E_CAPACITY.  bf_load
 * restores a checkpoint into a scene created from the same mesh (same
 * vertex and prescribed-vertex counts, else BF_E_ARG, as for a buffer that
 * is not a checkpoint or is cut short; pair keys that name no primitive of
 * the mesh give the error bf_set_active_set gives). */
int bf_save(bf_scene *scene, void *buf, size_t cap, size_t *used);
int bf_load(bf_scene *scene, const void *buf, size_t size);

/* Device bytes the scene holds (all its allocations); *bytes host. */
int bf_scene_bytes(bf_scene *scene, int64_t *bytes);

/* ---- time stepping (Alg. 1) ------------------------------------------- */

/* Advances n_steps time steps with the cumulative-TOI termination of
 * Eq. termination.  stats (host, n_steps entries, may be NULL) receives
 * per-step statistics.  Returns the first non-zero step status. */
int bf_step(bf_scene *scene, int32_t n_steps, bf_step_stats *stats);

/* Same as bf_step for one step, with the state exchanged through host
 * buffers: x_in/v_in (host, n_verts*3, may be NULL to keep the resident
 * state) are uploaded first and x_out/v_out (host, may be NULL) are
 * downloaded after the step. */
int bf_step_host(bf_scene *scene, const double *x_in, const double *v_in, double *x_out,
                 double *v_out, bf_step_stats *stats);

/* State access (host buffers, n_verts*3 each, either may be NULL). */
int bf_get_state(bf_scene *scene, double *x, double *v);
int bf_set_state(bf_scene *scene, const double *x, const double *v);

/* Moving boundary (section 5.3): target positions of the prescribed
 * vertices at the end of the next step, in vertex order (host,
 * n_prescribed*3).  They are applied to xhat^[0] of every later step until
 * replaced. */
int bf_set_obstacle_targets(bf_scene *scene, const double *targets);

/* Active set C = {(i, lambda_i, gamma_i)} (Alg. 1-3).  get: writes up to
 * cap pairs (keys host cap*5, lam/gam host cap) and the count to *n.
 * set: replaces C (BF_E_NOT_FOUND if a key names no surface pair). */
int bf_get_active_set(bf_scene *scene, int32_t cap, int32_t *n, int32_t *keys, double *lam,
                      double *gam);
int bf_set_active_set(bf_scene *scene, int32_t n, const int32_t *keys, const double *lam,
                      const double *gam);

/* Penalty stiffness mu and contact offset delta of the AL energy (section
 * 4.2, section 5.2).  bf_step recomputes mu at the start of each step. */
int bf_get_mu(bf_scene *scene, double *mu, double *delta);
int bf_set_mu(bf_scene *scene, double mu, double delta);

/* Sizes: n_surface_verts, n_surface_tris, n_surface_edges, nnz 3x3 blocks
 * of the upper block-sparse pattern, n_prescribed (host int32[5]). */
int bf_scene_info(bf_scene *scene, int32_t *info);

const char *bf_status_str(int status);

/* ---- teacher-forced entry points (same state as a step uses) ----------- */
/* All positions below are device buffers of n_verts*3 FP64. */

/* x~ = x^t + h v^t + h^2 g from the resident state (Alg. 1, inertia target). */
int bf_xtilde(bf_scene *scene, double *xtilde);

/* Section 5.2: mu = c_mu * max_i (grad^2 E)_ii over free DoFs at xhat,
 * from the PSD-projected elastic Hessian plus mass; stores and returns it. */
int bf_mu_init(bf_scene *scene, const double *xtilde, const double *xhat, double *mu);

/* Alg. 2, linearisation: d_i(x) and grad d_i(x) for every pair of C at xlin.
 * dist (device, |C|) and grad (device, |C|*12, vertex order of the pair:
 * PT point, t0, t1, t2 / EE a0, a1, b0, b1 of the internal primitive) may
 * be NULL. */
int bf_linearize(bf_scene *scene, const double *xlin, double *dist, double *grad);

/* Alg. 2, Newton system at xhat (after bf_linearize): gradient G (device,
 * n_verts*3) of the AL energy with Dirichlet rows zeroed, and the
 * assembled H kept in the scene (elastic PSD blocks + mass in upper BSR,
 * contacts as mu gamma_i grad d_i grad d_i^T).  *energy (host, may be
 * NULL) receives E(xhat). */
int bf_assemble(bf_scene *scene, const double *xtilde, const double *xlin, const double *xhat,
                double *grad, double *energy);

/* Semi-implicit friction (appendix A).  bf_friction_setup builds the
 * friction pairs from the current state and active set, with the current
 * mu and delta, as every time step does at its start: the active pairs
 * with k = mu_f mu max(0, lambda/mu - c(x)) > 0, their closest-point
 * weights and unit normal at x; later assemblies, energies, Hessian
 * products and solves include their terms until the next step replaces
 * them.  *n_pairs (host, may be NULL) receives their count.  bf_friction_get
 * copies up to cap pairs (host, any may be NULL; order unspecified): 4
 * vertex ids, 4 weights, the normal and k per pair; *n their count.
 * mu_f = 0 gives no pairs. */
int bf_friction_setup(bf_scene *scene, int32_t *n_pairs);
int bf_friction_get(bf_scene *scene, int32_t cap, int32_t *n, int32_t *v4, double *w4, double *n3, double *k);

/* y = H x with the H of the last bf_assemble (device n_verts*3 each);
 * prescribed rows/columns are eliminated (identity on the diagonal). */
int bf_hess_apply(bf_scene *scene, const double *x, double *y);

/* Copies the upper block-sparse H (host): row_ptr (n_verts+1), col (nnzb),
 * val (nnzb*9, row-major 3x3 blocks).  Any pointer may be NULL. */
int bf_get_bsr(bf_scene *scene, int32_t *row_ptr, int32_t *col, double *val);

/* Block-Jacobi PCG on the last assembled H (section 5.1): x (device) = the
 * solution of H x = b (device) to ||r|| <= tol ||b||, at most maxit
 * iterations; *iters (host) receives the count.  BF_E_CG_MAXIT if capped. */
int bf_pcg(bf_scene *scene, const double *b, double *x, double tol, int32_t maxit, int32_t *iters);

/* AL energy L (Eq. total-energy) at xhat with the slacks of the last
 * bf_assemble held fixed (*L host). */
int bf_energy(bf_scene *scene, const double *xtilde, const double *xlin, const double *xhat,
              double *L);

/* Alg. 2 SolveSubproblem: xhat (device, in/out) from xhat, updating the
 * multipliers and decay factors of C.  Newton ends when the line search
 * accepts the full step (r = 1 among r = 1, 1/2, ..., 2^-max_ls, accepted
 * when L(xhat + r p) <= L(xhat) + 1e-12 max(|L(xhat)|, |L| at the first
 * Newton iterate of the time step, or of this call)) or after max_newton
 * iterations.  newton/cg (host, may be NULL). */
int bf_solve_subproblem(bf_scene *scene, const double *xtilde, const double *xlin, double *xhat,
                        int32_t *newton, int32_t *cg);

/* CCD hits (broad phase + ACCD, section 5.1) along x0 -> x1 over all
 * admissible PT/EE pairs: up to cap keys (host cap*5) and TOIs (host cap);
 * *n receives the total count. */
int bf_ccd_hits(bf_scene *scene, const double *x0, const double *x1, int32_t cap, int32_t *n,
                int32_t *keys, double *toi);

/* Alg. 3 UpdateActiveSet(x, xhat, C); *n_active (host, may be NULL). */
int bf_update_active_set(bf_scene *scene, const double *x, const double *xhat, int32_t *n_active);

/* MaxStepSize: alpha = min(1, min_i TOI_i) along x0 -> x1 (*alpha host);
 * with BF_MODEL_NH also at most bf_inversion_step's bound. */
int bf_max_step_size(bf_scene *scene, const double *x0, const double *x1, double *alpha);

/* Gradient-norm residual of IPC (section 6): *res (host) =
 * (1/h) ||H^-1 grad L||_inf at x (device, n_verts*3), L the AL energy
 * (Eq. total-energy) linearised at x with the scene's active set,
 * multipliers, decay factors, mu and delta, taken at xhat = x with the
 * optimal slacks; H its PSD-projected Hessian, solved by the block-Jacobi
 * PCG to cg_tol.  Overwrites the assembled system.  Synchronises the
 * scene's stream. */
int bf_newton_residual(bf_scene *scene, const double *xtilde, const double *x, double *res);

/* Residuals of the last time step's outer iterations when res_tol > 0
 * (the first at x^t, the last below res_tol unless the step failed):
 * copies min(cap, count) into out (host), *n (host) = count. */
int bf_get_residual_log(bf_scene *scene, int32_t cap, int32_t *n, double *out);

/* Inversion bound of MaxStepSize (section 4.1, for non-invertible
 * materials): along x0 + t (x1 - x0) (device, n_verts*3 each) every element
 * with a free vertex keeps J(t) = det F(t) above s_ccd * J(0); *alpha (host)
 * = the smallest t in (0, 1] with J(t) = s_ccd J(0) over those elements,
 * else 1; an element with J(0) <= 0 gives 0.  Evaluated for any model;
 * the time step applies it with BF_MODEL_NH only.  Synchronises the
 * scene's stream. */
int bf_inversion_step(bf_scene *scene, const double *x0, const double *x1, double *alpha);

/* Narrow phase only: additive CCD on n explicit pairs of one type (0 = PT,
 * 1 = EE); x0, x1 (device, n*12: the 4 vertices of each pair), toi
 * (device, n; +inf = no hit within [0, 1]).  s: conservative rescaling.
 * stream: cudaStream_t or NULL. */
int bf_accd(int32_t type, int32_t n, const double *x0, const double *x1, double s, double *toi,
            void *stream);

/* Allocation-free MaxStepSize over explicit pairs: *alpha = min(1, min_i
 * TOI_i) over n pairs of one type (0 = PT, 1 = EE), with TOI_i the additive
 * CCD result that bf_accd returns for the same pair and s (so, for finite
 * inputs, alpha equals min(1, min of bf_accd's output) exactly; a pair with
 * a non-finite coordinate gives alpha = 0, no step).  x0, x1 (device, n*12),
 * alpha (device, 1 double).  stream: cudaStream_t or NULL; the call
 * synchronizes that stream before it returns.
 *
 * The paper has no counterpart of this entry point: it exists for callers
 * that may not allocate device memory once they are running (a host that
 * hands the library a fixed memory budget, or a real-time loop where an
 * allocation could block or fail).  It calls no cudaMalloc/cudaFree and no
 * allocating library routine: its scratch is a static device array of
 * 8,224 x 8 bytes inside the library, which bounds n to 1,048,576 pairs;
 * larger n returns BF_E_ARG without launching anything.
 * - The first call on each device looks up the array's device address and
 *   caches it, so make that first call (n may be 0) before any stream
 *   capture.  The cached address belongs to the device's primary context
 *   (the one the CUDA runtime uses); after cudaDeviceReset, or from another
 *   context, it is stale: do not call the entry point there.
 * - The array is shared by all calls on a device and keeps the previous
 *   call's contents; each call resets the part that must start at zero.
 *   Calls that overlap on the GPU (other streams, threads or processes
 *   sharing the context) race on it and may return a wrong alpha: serialize
 *   them.
 * Errors: BF_E_ARG (bad type, s outside (0,1), n < 0 or too large, NULL
 * pointers), BF_E_CUDA. */
int bf_max_step_size_pairs_noalloc(int32_t type, int32_t n, const double *x0, const double *x1, double s,
                                   double *alpha, void *stream);

/* Per-kernel CUDA-event timing of the hot kernels during bf_step (off by
 * default).  bf_get_timers fills, per kernel id 0..n-1, launches and total
 * milliseconds (host int64 launches[n], double ms[n]); names[n] points to
 * static strings.  Returns the number of timed kernels. */
int bf_enable_timers(bf_scene *scene, int32_t on);
/* PCG execution.  0 = three launches per iteration with the scalar
 * recurrences kept on the device.  1..4 = one persistent cooperative launch
 * per solve with up to `mode` CTAs per SM (default 1), keeping the matrix
 * in shared memory when it fits, else streaming it, with the per-row
 * vectors in global memory when they do not fit in shared memory either.
 * With the matrix in shared memory the iteration is the single-reduction
 * recurrence of Chronopoulos and Gear (one grid-wide reduction per
 * iteration); adding 128 selects the two-reduction form there.  The
 * streamed variants use two reductions per iteration.  Adding 16 forbids
 * the shared-memory copy of the matrix; adding 32 forces a global-memory
 * variant: in mixed precision the symmetric one (upper blocks streamed
 * once, transposed products by vector reductions into global memory),
 * else, or with 64 added, the one that streams both triangles.  Adding 256
 * keeps no contact pair in shared memory (every pair is read from global
 * memory in every iteration; by default up to 256 pairs per CTA are cached
 * in the shared memory left over).  The same Krylov method in every mode
 * (the same iterates in exact arithmetic); the order of floating-point sums
 * differs. */
int bf_set_pcg_mode(bf_scene *scene, int32_t mode);

/* Configuration of the persistent PCG chosen at the scene's first solve
 * (host int32[8]): mode, CTAs, threads per CTA, shared memory bytes per
 * CTA, variant (0: blocks streamed through the BSR map, vectors in shared
 * memory; 1: blocks resident in shared memory, two reductions per
 * iteration; 2: blocks streamed from a jagged global copy, per-row vectors
 * in global memory; 3: upper blocks streamed from a jagged global copy,
 * transposed products reduced in global memory; 4: blocks resident in
 * shared memory, one reduction per iteration), max rows, max blocks and max
 * window vertices per CTA (zeros before the first solve). */
int bf_get_pcg_config(bf_scene *scene, int32_t *cfg);

/* PCG autotuner: on the system assembled last (bf_step or bf_assemble must
 * have run), times `iters` (>= 8) PCG iterations of each execution
 * configuration (bf_set_pcg_mode 1, 2, 129, 130, 17, 18, 33, 34, 97, 98 and
 * 0; a persistent configuration that does not fit is skipped, and so are 129
 * and 130 where the matrix is not resident, as they then equal 1 and 2) with
 * CUDA events on the
 * scene's stream, then sets the fastest per iteration (a configuration later
 * in that list replaces the choice so far only when it is more than 2 %
 * faster, so timing noise does not flip it).  modes / us_per_iter
 * (host, cap entries each) receive the measured configurations in order,
 * *n_out (host, may be NULL) their count, *best (host) the chosen mode.
 * The solution buffers it uses are scratch; results of later steps do not
 * depend on the choice beyond the order of floating-point sums.  Returns
 * BF_E_ARG when no configuration could be timed (no assembled system). */
int bf_autotune_pcg(bf_scene *scene, int32_t iters, int32_t cap, int32_t *modes, double *us_per_iter,
                    int32_t *n_out, int32_t *best);

/* Failure-detection test of the persistent PCG's bounded waits (not needed
 * in normal use).  With `on` nonzero, the scene's next persistent solves
 * arrive at their grid barriers as usual but wait on a device word that no
 * CTA increments, so the first grid-wide reduction of a solve never
 * completes: every CTA gives up after its time limit (2 s), the kernel
 * ends, the solve returns BF_E_CUDA, and the scene and the CUDA context stay
 * usable (call again with 0 to solve normally).  Returns BF_E_ARG for a NULL
 * scene. */
int bf_test_pcg_barrier_fail(bf_scene *scene, int32_t on);

/* Number of this library's own kernel launches issued for the scene since
 * creation (sorts and scans done by CUB are not counted); *n host. */
int bf_get_launch_count(bf_scene *scene, int64_t *n);
int bf_get_timers(bf_scene *scene, int32_t cap, int64_t *launches, double *ms, const char **names);

/* ---- Batches: many independent scenes advanced concurrently ------------
 * The paper advances one scene; this runner serves many.  A batch owns
 * n_workers host threads, each with its own CUDA stream.  bf_batch_admit
 * binds a created scene to the stream of the least-loaded worker and
 * queues n_steps time steps (Alg. 1 each, exactly as bf_step); workers
 * advance their scenes one step per turn, round robin, so scenes admitted
 * while others run join at the next turn and the kernels of different
 * scenes overlap on the device.  Admission returns BF_E_BUDGET, and queues
 * nothing, when the device bytes (bf_scene_bytes) of the batch's unfinished
 * scenes plus this one would exceed hbm_budget_bytes; the caller may retry
 * after a ticket finishes.  Times are seconds since bf_batch_create.
 * Ownership: the caller keeps every scene and must not call it, nor destroy
 * it, while its ticket is unfinished; bf_batch_release (finished tickets
 * only) and bf_batch_destroy put the scene back on the default stream.
 * Scenes admitted to a batch should use the default allocator or one that
 * is not bound to a stream.  A failing step (status < 0) finishes its
 * ticket with that status. */
typedef struct bf_batch bf_batch;
int bf_batch_create(int32_t n_workers, int64_t hbm_budget_bytes, bf_batch **out);
/* Stops the workers after their current step and frees the batch; unfinished
 * tickets are abandoned (their scenes stay valid). */
int bf_batch_destroy(bf_batch *batch);
/* *ticket (host) identifies the job. */
int bf_batch_admit(bf_batch *batch, bf_scene *scene, int32_t n_steps, int64_t *ticket);
/* Waits until the ticket finished or timeout_ms passed (< 0: no limit);
 * *done (host) = 1 when finished. */
int bf_batch_wait(bf_batch *batch, int64_t ticket, int32_t timeout_ms, int32_t *done);
/* Progress of a ticket (all host, any may be NULL): steps done, status of
 * the last step, admission time, completion time of each step and its
 * statistics (up to cap entries). */
int bf_batch_result(bf_batch *batch, int64_t ticket, int32_t cap, int32_t *steps_done, int32_t *status,
                    double *t_admit, double *t_steps, bf_step_stats *stats);
/* Forgets a finished ticket. */
int bf_batch_release(bf_batch *batch, int64_t ticket);
/* info[6] (host int64): resident bytes of unfinished scenes, budget,
 * workers, queued scenes, finished tickets, tickets issued. */
int bf_batch_info(bf_batch *batch, int64_t *info);
/* Seconds since bf_batch_create (the clock of t_admit and t_steps). */
double bf_batch_now(bf_batch *batch);

/* Per-bucket PCG autotuning in the batch (off by default): scenes are
 * bucketed by floor(log2(matrix blocks + 1)); the first scene of a bucket
 * is tuned with bf_autotune_pcg after its first step, and every scene of
 * that bucket takes the chosen configuration at its next turn. */
int bf_batch_set_autotune(bf_batch *batch, int32_t on);
/* Admitted scenes wait with blocking-sync events (bf_set_sync_mode 1) until
 * released (off by default). */
int bf_batch_set_blocking_sync(bf_batch *batch, int32_t on);
/* The tuned buckets so far, ascending: up to cap (bucket, mode) pairs into
 * buckets / modes (host); *n (host, may be NULL) = their count. */
int bf_batch_tuned(bf_batch *batch, int32_t cap, int32_t *buckets, int32_t *modes, int32_t *n);

#ifdef __cplusplus
}
#endif
#endif
