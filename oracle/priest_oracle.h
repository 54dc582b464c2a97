/*
 * priest_oracle.h -- plain FP64 CPU oracle for PRIEST
 * (Rastgar et al., "PRIEST: Projection Guided Sampling-Based Optimization
 * for Autonomous Navigation", arXiv 2309.08235).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and its library are loaded by the
 * test-suite, by the package smoke check and by the benchmark's CPU-baseline
 * leg; nothing on the product path includes, links or calls them.  The
 * oracle shares no code, header, table or helper with the CUDA library.
 *
 * Layout conventions (all row-major, FP64):
 *   n_v = degree + 1 coefficients per axis.
 *   xi / xi_bar / lambda of one sample: [c_x(0..n_v-1), c_y(...), (c_z(...))],
 *   D = dims * n_v values.  Batches are N x D.
 *   Basis matrices P, Pd, Pdd: n_p x n_v, row k is time t_k = horizon*k/(n_p-1).
 *   Obstacles: center n_obs x dims at t = 0, vel n_obs x dims (constant
 *   velocity), semi n_obs x 2 = (a, b): semi-axes (a, a, b); 2-D uses a only.
 *
 * Return codes: 0 on success, negative on invalid input / numerical failure.
 *
 * Parity status of each function is stated beside it ("pinned by ..." or
 * "parity unpinned").
 */
#ifndef PRIEST_ORACLE_H
#define PRIEST_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dims;            /* 2 or 3 */
    int degree;          /* polynomial degree n, n_v = n + 1 */
    int n_p;             /* number of time stamps */
    double horizon;      /* T_h, seconds */
    double rho;          /* augmented-Lagrangian weight */
    double vmax, amax;   /* velocity / acceleration bounds */
    int use_bounds;      /* workspace bounds G xi <= tau on/off */
    double smin[3], smax[3];
    int bc_final_mask;   /* bit q set: q-th derivative fixed at t_f (start: all of q = 0,1,2) */
    double b0[3][3];     /* [axis][q] start position / velocity / acceleration */
    double bf[3][3];     /* [axis][q] final values */
    int n_obs;
    const double *center, *vel, *semi;
    /* c_1: 0 = sum of squared accelerations (point-to-point benchmark);
     * 1 = BARN-style (Sec. Baselines and Benchmarks): per time stamp
     * w_acc |a|^2 + w_curv kappa^2 + w_path d^2 with the curvature
     * kappa = |v x a| / (|v|^2 + curv_eps^2)^(3/2) and d the distance from the
     * point to the start-goal segment */
    int cost_kind;
    double w_acc, w_curv, w_path, curv_eps;
} orc_problem;

typedef struct {
    int proj_iters;      /* K */
    int cem_iters;       /* L (the paper's N) */
    int n_samples;       /* N_b */
    int n_proj;          /* N_proj */
    int n_elite;         /* N_elite */
    double sigma_lr;     /* sigma, learning rate of the refit */
    double gamma;        /* temperature of the refit weights */
    double chol_eps;     /* relative jitter: Sigma + chol_eps*tr(Sigma)/D * I */
    double init_std;     /* default Sigma_0 = init_std^2 I */
} orc_cem;

/* Bernstein basis and its time derivatives (Sec. II-A.2, eq. parametrized). */
int orc_basis(int degree, int n_p, double horizon, double *P, double *Pd, double *Pdd);

/* Equality block A (n_eq x n_v, identical for every axis) and b (dims x n_eq)
 * (Sec. II-A.2, A xi = b_eq).  Returns n_eq (>0) or <0. */
int orc_equality(const orc_problem *pr, double *A, double *b);

/* Dense per-axis KKT matrix [[I + rho F^T F, A^T], [A, 0]] of eq. matrix_vec,
 * size (n_v + n_eq)^2; F^T F summed block by block over the stacked F of
 * eq. f_e (+ G of eq. bound_con).  Returns n_v + n_eq or <0. */
int orc_kkt_matrix(const orc_problem *pr, double *K);

/* Closed-form alternating-minimisation updates of one obstacle row block
 * (Appendix, eqs. comp_alpha, comp_beta, comp_d for eq.
 * collision_avoidance_proposed).  pos, o: dims.  Writes alpha, beta
 * (pi/2 in 2-D), d (>= 1) and the target point e (dims). */
void orc_obstacle_polar(int dims, const double *pos, const double *o, double a, double b,
                        double *alpha, double *beta, double *d, double *e);

/* Same for the velocity / acceleration bound blocks (eqs. fv, fa):
 * 0 <= d <= 1, target e = d * vmax * direction. */
void orc_bound_polar(int dims, const double *v, double vmax,
                     double *alpha, double *beta, double *d, double *e);

/* Projection of N samples (Sec. III-A, Appendix eqs. comp_alpha..comp_zeta):
 * xi_bar^0 = Pi_A(xi) (if xi_bar0 == NULL) else xi_bar0; lambda^0 =
 * lambda_io (NULL -> zeros); K alternating-minimisation iterations.
 * Outputs xi_bar (N x D); lambda_io updated in place if non-NULL.
 * Pinned per iteration (dense restatement, Lagrangian minimiser, zero
 * obstacles = Pi_A, feasible fixed point) and, converged, on a two-variable
 * case by brute force and the fixed-point identity xi_bar = Pi_A(xi + lambda);
 * the converged multi-obstacle result in general: parity unpinned. */
int orc_project(const orc_problem *pr, int K, int N, const double *xi, const double *xi_bar0,
                double *lambda_io, double *xi_bar_out);

/* Euclidean projection onto {A c = b} for every axis (K = 0 of the above). */
int orc_project_eq(const orc_problem *pr, int N, const double *xi, double *out);

/* Residual r(xi_bar) (Alg. 1, "compute the residuals") as the 2-norm of the
 * stacked constraint residual with a fresh e(xi_bar), each block evaluated in
 * closed form (exact zero for inactive rows), and the acceleration cost
 * c_1 = sum_t sum_axis acc^2 (Sec. IV, point-to-point cost). */
int orc_residual_cost(const orc_problem *pr, int N, const double *xi_bar, double *r, double *c1);

/* The same residual computed literally as || F xi_bar - e(alpha,beta,d) ||_2
 * through the trigonometric targets of eq. f_e (used only to pin the
 * closed form above). */
int orc_residual_stacked(const orc_problem *pr, int N, const double *xi_bar, double *r);

/* ConstraintEliteSet / EliteSet selection (Alg. 1): the n_proj samples of
 * least r, then among them the n_elite of least c_aug = c_1 + r; ties go to
 * the lower sample index.  proj_idx may be NULL. */
int orc_select(int N, const double *r, const double *c_aug, int n_proj, int n_elite,
               int *proj_idx, int *elite_idx);

/* MPPI-like refit (eqs. update_mean, update_covariance) in place. */
int orc_refit(int D, int n_elite, const double *elites, const double *c_aug,
              double sigma_lr, double gamma, double *mu, double *cov);

/* Textbook Cholesky S = L L^T (lower).  Returns -6 on a non-positive pivot. */
int orc_cholesky(int D, const double *S, double *L);

/* Host Gaussian stream: SplitMix64 -> 53-bit uniforms -> Box-Muller. */
void orc_rng_normal(uint64_t seed, int64_t count, double *out);

/* Defaults: mu_0 = straight-line Bernstein coefficients, Sigma_0 = s0^2 I. */
int orc_default_mean(const orc_problem *pr, double *mu);

/* Full PRIEST (Alg. 1).  z: L x N x D standard normals, or NULL to draw them
 * from orc_rng_normal(seed).  mu0/cov0 may be NULL (defaults).
 * Outputs: best xi_bar (D), its r and c_aug, final mu (D) and cov (D x D),
 * the last iteration's elite indices (n_elite, sorted by c_aug). */
int orc_plan(const orc_problem *pr, const orc_cem *cem, const double *mu0, const double *cov0,
             const double *z, uint64_t seed, double *best, double *best_r, double *best_caug,
             double *mu_out, double *cov_out, int *elite_out);

/* Alg. 1 with a multiplier warm start (the serving loop's replans): lam0
 * (N x D, or NULL for 0) is lambda^0 of the first CEM iteration's
 * projection; later iterations start from 0.  lam_out (N x D, or NULL)
 * receives the multipliers after the last CEM iteration's projection.
 * orc_plan is this with both NULL. */
int orc_plan_warm(const orc_problem *pr, const orc_cem *cem, const double *mu0, const double *cov0,
                  const double *lam0, const double *z, uint64_t seed, double *best, double *best_r,
                  double *best_caug, double *mu_out, double *cov_out, int *elite_out, double *lam_out);

/* D-PRIEST (Sec. D-PRIEST): M distributions, N_b / M samples each, stacked
 * row-wise for one projection, selections (N_proj / M, N_elite / M) and
 * refits per distribution, best of M by c_aug.  orc_multi_default_means
 * gives the default means (the straight line bowed sideways by
 * (j - (M-1)/2) spread). */
int orc_multi_default_means(const orc_problem *pr, int M, double spread, double *mu);
int orc_plan_multi(const orc_problem *pr, const orc_cem *cem, int M, const double *mu0, const double *cov0,
                   const double *z, uint64_t seed, double *best, double *best_caug, int *best_dist,
                   double *dist_best, double *dist_r, double *dist_caug, double *mu_out);

#ifdef __cplusplus
}
#endif
#endif
