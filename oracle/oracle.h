/*
 * Plain, slow, single-threaded FP64 CPU oracle of the barrier-free
 * augmented-Lagrangian contact method ("Robust and Efficient
 * Penetration-Free Elastodynamics without Barriers", arXiv 2512.12151).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code with
 * the CUDA library and never runs on its behalf.
 *
 * Everything is FP64, compiled with -ffp-contract=off.  Each routine cites
 * the paper passage it follows (section, equation or algorithm).
 *
 * Pins (tests that check this code against facts fixed outside it): energy,
 * stress and Hessian by finite differences and the small-strain limit; the
 * eigensolver and PSD projection against a dense library eigensolver and an
 * independent analytic eigensystem; distances by brute-force minimisation;
 * ACCD by closed-form cases and root bracketing; lumped mass and mu_init in
 * closed form; PCG against a dense solve; the AL subproblem against an
 * independent constrained solve (KKT point); the active-set filter and decay
 * on hand-built cases; the time step by free fall, momentum, the beta product,
 * the moving-boundary bound and penetration-free states; friction by the
 * smoothing function's boundary values, finite differences of its energy and
 * gradient, and the sliding and sticking block on an incline (closed-form
 * acceleration g (sin theta - mu_f cos theta)).  Whole trajectories
 * of contact scenes have no value fixed outside this code: parity unpinned
 * beyond the invariants above.
 */
#ifndef BF_ORACLE_H
#define BF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double dt, delta, gravity[3], eps, cg_tol, gamma_decay, c_mu, s_ccd, mu_f, eps_v;
    double res_tol; /* > 0: end the outer loop once the gradient-norm residual is below it (not beta) */
    int32_t k_min, max_outer, max_newton, max_ls, max_cg, precision, model; /* model: 0 SNH, 1 COR, 2 NH */
    int32_t ccd_reuse; /* 1: UpdateActiveSet takes the MaxStepSize segment x^[k] -> xhat^[k+1] */
} or_params;

typedef struct {
    int32_t outer_iters, newton_iters, cg_iters, n_contacts, status, ls_fail, cg_maxit, stalls;
    double mean_alpha, min_alpha, mu, beta, delta;
} or_stats;

typedef struct or_scene or_scene;

/* ---- element level (section 3, section 5.1) ---- */
double or_snh_psi(const double F[9], double mu, double lam);
void or_snh_pk1(const double F[9], double mu, double lam, double P[9]);
void or_snh_hess9(const double F[9], double mu, double lam, double H[81]);
int or_sym_eig(int n, const double *A, double *w, double *Q);
void or_psd_project(int n, const double *A, double *Ap);
void or_elem_F(const double x[12], const double B[9], double F[9]);
void or_elem_grad_hess(const double x[12], const double B[9], double vol, double mu, double lam,
                       int project, double *psi, double g[12], double H[144]);
void or_lame(double E, double nu, double *mu, double *lam);
/* corotated linear elasticity (COR, Tab. 2) */
double or_cor_psi(const double F[9], double mu, double lam);
void or_cor_pk1(const double F[9], double mu, double lam, double P[9]);
void or_cor_hess9(const double F[9], double mu, double lam, double H[81]);
double or_nh_psi(const double F[9], double mu, double lam);
void or_nh_pk1(const double F[9], double mu, double lam, double P[9]);
void or_nh_hess9(const double F[9], double mu, double lam, double H[81]);
double or_model_psi(int model, const double F[9], double mu, double lam);
double or_cubic_first_root(const double c[4]);
void or_det_cubic(const double A[9], const double B[9], double s, double c[4]);
/* element energy, gradient and (projected) Hessian of material model
 * model (0 SNH, 1 COR, 2 NH); or_elem_grad_hess is model 0 */
void or_elem_grad_hess_model(int model, const double x[12], const double B[9], double vol, double mu, double lam,
                             int project, double *psi, double g[12], double H[144]);

/* ---- distances and CCD (section 4.2, section 5.1) ---- */
double or_pt_dist2(const double p[3], const double a[3], const double b[3], const double c[3]);
double or_ee_dist2(const double a0[3], const double a1[3], const double b0[3], const double b1[3]);
double or_pair_dist_grad(int type, const double x[12], double g[12]);
int or_accd(int type, const double x0[12], const double x1[12], double s, double tmax,
            int32_t max_iter, double *toi);

/* ---- scene ---- */
or_scene *or_create(int32_t nv, const double *rest, const double *x0, const double *v0,
                    int32_t nt, const int32_t *tets, const int32_t *tet_mat, int32_t nm,
                    const double *mats, int32_t nx, const int32_t *xtris, const uint8_t *dir,
                    const or_params *prm);
void or_destroy(or_scene *S);
void or_get_state(const or_scene *S, double *x, double *v);
void or_set_state(or_scene *S, const double *x, const double *v);
void or_set_dirichlet_targets(or_scene *S, const double *targets);
void or_surface_sizes(const or_scene *S, int32_t *nsv, int32_t *nst, int32_t *nse);
void or_surface(const or_scene *S, int32_t *sv, int32_t *st, int32_t *se);
void or_mass(const or_scene *S, double *m);
double or_get_mu(const or_scene *S);
void or_set_mu_delta(or_scene *S, double mu, double delta);

/* active set, exchanged as canonical vertex keys (5 ints per pair) */
int32_t or_active_count(const or_scene *S);
void or_active_get(const or_scene *S, int32_t *keys, double *lam, double *gam);
void or_active_verts(const or_scene *S, int32_t *v4);
int32_t or_active_set(or_scene *S, int32_t n, const int32_t *keys, const double *lam,
                      const double *gam);

/* teacher-forced pieces of Alg. 1-3 */
void or_xtilde(const or_scene *S, double *xt);
double or_mu_init(or_scene *S, const double *xhat, const double *xtilde);
void or_linearize(or_scene *S, const double *xlin, double *d, double *g);
double or_assemble(or_scene *S, const double *xtilde, const double *xlin, const double *xhat,
                   double *grad);
void or_slacks(const or_scene *S, double *s);
void or_hess_apply(const or_scene *S, const double *in, double *out);
void or_hess_dense(const or_scene *S, double *out);
int32_t or_pcg(const or_scene *S, const double *b, double *x, double tol, int32_t maxit);
double or_energy_L(or_scene *S, const double *xtilde, const double *xlin, const double *xhat,
                   const double *sfix);
int32_t or_solve_subproblem(or_scene *S, const double *xtilde, const double *xlin, double *xhat,
                            int32_t *cg_iters, int32_t *ls_fail);
int32_t or_ccd_hits(or_scene *S, const double *x0, const double *x1, int32_t brute,
                    int32_t cap, int32_t *keys, double *toi);
int32_t or_update_active_set(or_scene *S, const double *x, const double *xhat);
double or_max_step_size(or_scene *S, const double *x0, const double *x1);
double or_inversion_step(or_scene *S, const double *x0, const double *x1);
/* IPC-style gradient-norm residual (1/h) |H^-1 grad L|_inf at x, L
 * linearised at x with the current active set, multipliers, mu and delta */
double or_newton_residual(or_scene *S, const double *xtilde, const double *x);
/* residuals of the last time step's outer iterations (residual mode):
 * copies up to cap into out, returns their count */
int32_t or_get_residual_log(const or_scene *S, int32_t cap, double *out);
int32_t or_step(or_scene *S, int32_t nsteps, or_stats *stats, double *alpha_log,
                int32_t alpha_cap);
/* test hook: log xhat^[k] of the following steps' outer iterations into
 * buf (cap states of 3 nv doubles; NULL stops); the count logged so far */
int32_t or_set_xhat_log(or_scene *S, double *buf, int32_t cap);
int32_t or_xhat_log_count(const or_scene *S);
int32_t or_min_distance(or_scene *S, const double *x, double *dmin);

/* ---- semi-implicit friction (appendix A) ---- */
/* f0(y; eh) with eh = h eps_v, and its first two derivatives */
double or_friction_f0(double y, double eh, double *f1, double *f2);
/* friction pairs from the current state and active set (done at every
 * time step's start by or_step); returns their count */
int32_t or_friction_setup(or_scene *S);
int32_t or_friction_count(const or_scene *S);
/* per pair: 4 vertex ids, 4 closest-point weights, unit normal, coefficient
 * k = mu_f mu max(0, lambda/mu - c(x^t)) */
void or_friction_get(const or_scene *S, int32_t *v4, double *w4, double *n3, double *k);
/* friction energy at xhat; gradient (3 nv, may be NULL) and per-pair 3x3
 * tangent Hessians (9 per pair, may be NULL) */
double or_friction_eval(or_scene *S, const double *xhat, double *grad, double *A9);

#ifdef __cplusplus
}
#endif
#endif
