/*
 * priest.h -- C ABI of the GB300 (sm_103a) PRIEST library.
 *
 * PRIEST (Rastgar et al., "PRIEST: Projection Guided Sampling-Based
 * Optimization for Autonomous Navigation", arXiv 2309.08235) draws Gaussian
 * samples of Bernstein trajectory coefficients, pushes every sample towards
 * the feasible set with a batched projection (alternating minimisation over
 * polar-form obstacle / velocity / acceleration residuals and one shared KKT
 * inverse, Sec. III-A and Appendix), scores the projected samples, keeps
 * elites and refits the sampling distribution (Alg. 1, eqs. update_mean /
 * update_covariance).  Every step of that path runs in CUDA kernels for
 * sm_103a; there is no CPU fallback: a missing or unusable GPU is reported
 * as PRIEST_ERR_CUDA.
 *
 * Conventions shared by all entry points
 *   - Coefficients of one sample are stored axis-major:
 *     [c_x(0..n_v-1), c_y(0..n_v-1), (c_z(0..n_v-1))], D = dims * n_v,
 *     n_v = degree + 1; batches are row-major N x D, FP64 at the boundary.
 *   - Host pointers are read (or written) during the call only and remain
 *     owned by the caller.  Device memory used internally is owned by the
 *     context.  Entry points named *_device take device pointers owned by the
 *     caller and run asynchronously on the context's stream.
 *   - Errors are returned as priest_status; nothing is thrown across the ABI.
 *     priest_last_error() gives a message for the last failure of a context.
 *   - A context is used by one host thread at a time, except priest_submit /
 *     priest_poll, which lock internally.
 */
#ifndef PRIEST_H
#define PRIEST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PRIEST_MAX_DIMS 3
#define PRIEST_MAX_NV 16        /* degree <= 15 */
#define PRIEST_MAX_D 48         /* PRIEST_MAX_DIMS * PRIEST_MAX_NV */
#define PRIEST_MAX_NP 512       /* time stamps per trajectory */
#define PRIEST_MAX_OBS 2048     /* obstacles per problem */
#define PRIEST_MAX_SAMPLES 8192 /* N_b per problem */
#define PRIEST_MAX_ELITE 1024

typedef enum {
    PRIEST_OK = 0,
    PRIEST_PENDING = 1,        /* priest_poll: request not finished yet */
    PRIEST_ERR_INVALID = -1,   /* rejected argument (sizes, NaN, radius <= 0, ...) */
    PRIEST_ERR_NOMEM = -2,     /* device allocation failed */
    PRIEST_ERR_BUDGET = -3,    /* request does not fit the context's HBM budget */
    PRIEST_ERR_CUDA = -4,      /* CUDA runtime error or no usable GPU */
    PRIEST_ERR_TIMEOUT = -5,   /* a bounded wait gave up */
    PRIEST_ERR_NUMERIC = -6    /* non-positive pivot in a Cholesky / KKT factor, NaN */
} priest_status;

typedef enum {
    PRIEST_FP64_CHECK = 0,     /* every step in FP64 (parity mode) */
    PRIEST_FP32 = 1,           /* projection in FP32, sampling / refit / Cholesky / KKT in FP64 */
    PRIEST_MIXED_BF16 = 2      /* FP32 projection whose (point, obstacle) tests are one BF16 tensor-core
                                  product per CTA (split high/low operands, FP32 accumulation) that
                                  selects the pairs for the exact FP32 test; same results as FP32 up
                                  to summation order.  With cfg.autotune set, the first call of a
                                  projection shape times this kernel against the FP32 kernel and
                                  keeps the faster one (the FP32 kernel, whose neighbour lists skip
                                  most pair tests, on every shape measured so far); with autotune 0
                                  the tensor-core kernel runs.  Shapes it cannot hold (more than ~500
                                  obstacle columns) and the batched / serving paths run the FP32
                                  kernel. */
} priest_precision;

typedef struct priest_ctx priest_ctx;
typedef struct priest_loaded priest_loaded;

/* Context-wide settings and defaults (Alg. 1 and Sec. V-A constants; the
 * constants the paper leaves open are fields). */
typedef struct {
    int dims;              /* 2 or 3 (default for problems that give 0) */
    int degree;            /* Bernstein degree n, 5..15; n_v = n + 1 */
    int n_p;               /* time stamps (default) */
    double horizon;        /* T_h in seconds (default) */
    double rho;            /* augmented-Lagrangian weight of eq. lagrange */
    int proj_iters;        /* K projection iterations per CEM iteration */
    int cem_iters;         /* L CEM iterations (the paper's N) */
    int n_samples;         /* N_b (default) */
    int n_proj;            /* N_proj (default; 0 -> floor(80 N_b / 110)) */
    int n_elite;           /* N_elite (default; 0 -> N_b / 10) */
    double sigma_lr;       /* sigma of eqs. update_mean / update_covariance */
    double gamma;          /* temperature of the refit weights */
    double chol_eps;       /* Cholesky jitter, relative: Sigma + chol_eps tr(Sigma)/D I */
    double init_std;       /* default Sigma_0 = init_std^2 I */
    double vmax, amax;     /* velocity / acceleration bounds (default) */
    int use_bounds;        /* workspace bounds G xi <= tau (eq. bound_con) */
    double smin[3], smax[3];
    int precision;         /* priest_precision */
    size_t hbm_budget;     /* bytes of device memory the serving loop allocates once and admits
                              requests into (0 = 2 GiB); its small per-step staging is extra */
    int autotune;          /* 1: time candidate tilings of the projection kernel on the first
                              call of each problem shape and keep the fastest (the first call
                              then blocks for the trials); 0: cost-model tiling */
    int serve_slots;       /* most requests the serving loop keeps on the device at once
                              (0 = as many as the budget holds) */
} priest_config;

/* One planning problem (Sec. II-A: eqs. acc_cost .. coll_multiagent). */
typedef struct {
    int n_obs;
    const double *center;  /* n_obs x dims, obstacle centres at t = 0 */
    const double *vel;     /* n_obs x dims, constant velocities (NULL = static) */
    const double *semi;    /* n_obs x 2: semi-axes (a, b) of an (a, a, b) ellipsoid; 2-D uses a */
    double b0[3][3];       /* [axis][q]: start position, velocity, acceleration */
    double bf[3][3];       /* [axis][q]: final values */
    int bc_final_mask;     /* bit q: q-th derivative fixed at t_f; 1, 3 or 7 (0 = free end) */
    uint64_t seed;         /* seed of the host Gaussian stream (priest_plan, priest_submit) */
    int64_t robot_id;      /* >= 0: warm-start key for priest_submit; -1: none */
    /* per-problem overrides; 0 keeps the context default */
    int dims, n_p, n_samples, n_proj, n_elite;
    double horizon, vmax, amax;
    /* c_1 of Alg. 1: 0 = sum over time stamps of |acc|^2 (point-to-point
     * benchmark); 1 = BARN-style cost (Sec. Baselines and Benchmarks): per
     * time stamp w_acc |a|^2 + w_curv kappa^2 + w_path d^2, kappa = |v x a| /
     * (|v|^2 + curv_eps^2)^(3/2), d = distance from the point to the
     * straight start-goal segment.  Weights finite and >= 0, curv_eps > 0
     * (used only with cost_kind 1). */
    int cost_kind;
    double w_acc, w_curv, w_path, curv_eps;
} priest_problem;

/* Result of one solve. */
typedef struct {
    int status;            /* priest_status of the solve */
    int D;                 /* coefficients per sample */
    int best_index;        /* sample index of the returned trajectory in the last iteration */
    double xi_best[PRIEST_MAX_D]; /* Alg. 1 output: lowest c_aug member of the last EliteSet */
    double resid;          /* r(xi_best) */
    double cost;           /* c_1(xi_best): summed squared acceleration */
    double c_aug;          /* cost + resid */
    double mu[PRIEST_MAX_D]; /* sampling mean after the last refit */
    double latency_ms;     /* priest_poll: submit-to-completion time */
} priest_result;

/* Creates a context bound to the current CUDA device.  cuda_stream: a
 * cudaStream_t to run on, or NULL for a stream the context creates and owns.
 * Errors: PRIEST_ERR_INVALID (bad config), PRIEST_ERR_CUDA (no usable GPU). */
priest_status priest_create(const priest_config *cfg, void *cuda_stream, priest_ctx **out);

/* Waits for outstanding work, stops the serving worker and frees everything
 * the context owns.  NULL is accepted. */
priest_status priest_destroy(priest_ctx *ctx);

/* Message of the context's last failure ("" if none).  Valid until the next call. */
const char *priest_last_error(const priest_ctx *ctx);

/* Projection only (Sec. III-A; Appendix eqs. comp_alpha .. comp_zeta):
 * xi_bar^0 = Pi_A(xi) (the boundary-condition coefficients set exactly),
 * lambda^0 = lambda_io (or 0 if NULL), then cfg.proj_iters alternating-
 * minimisation iterations, then r and c_1 of the result (Alg. 1 residual and
 * cost).  xi: n x D (host, read); lambda_io: n x D (host, updated) or NULL;
 * xi_bar_out: n x D (host, written); resid_out, cost_out: n (host) or NULL.
 * n may be 0.  Blocks until done. */
priest_status priest_project(priest_ctx *ctx, const priest_problem *prob, int n, const double *xi,
                             double *lambda_io, double *xi_bar_out, double *resid_out,
                             double *cost_out);

/* Full solve (Alg. 1): L CEM iterations of sample -> project -> residual/cost
 * -> ConstraintEliteSet -> EliteSet -> refit, Gaussian draws from the host
 * stream seeded by prob->seed (see priest_rng_normal).  mu0 (D) and cov0
 * (D x D) may be NULL: straight-line Bernstein mean and init_std^2 I.
 * Blocks until done. */
priest_status priest_plan(priest_ctx *ctx, const priest_problem *prob, const double *mu0,
                          const double *cov0, priest_result *out);

/* As priest_plan with the standard-normal draws given explicitly:
 * z is L x N x D (host, read). */
priest_status priest_plan_z(priest_ctx *ctx, const priest_problem *prob, const double *mu0,
                            const double *cov0, const double *z, priest_result *out);

/* D-PRIEST (Sec. D-PRIEST, Fig. fig_decentralized): M Gaussian
 * distributions refined in parallel.  Each draws N_b / M samples (N_b =
 * prob's / the context's sample count, a multiple of M); the samples of all
 * distributions are stacked row-wise (rows j N_b/M .. (j+1) N_b/M - 1 belong
 * to distribution j) and projected in one launch; the selections
 * (N_proj / M, N_elite / M, at least 1) and refits then run per
 * distribution in one segmented launch each.  After L iterations *best is
 * the lowest-c_aug member over the M distributions' best elites (ties: the
 * lower j), *best_dist its distribution, per_dist[j] (M entries, or NULL)
 * each distribution's best elite and final mean; best_index is the sample's
 * index inside its distribution.
 *   mu0: M x D means or NULL: the straight-line coefficients with the
 *        interior coefficients moved by (j - (M-1)/2) * 2 init_std along the
 *        start-goal line's normal (2-D: rotated +90 degrees; 3-D: horizontal);
 *   cov0: M x D x D or NULL (init_std^2 I);
 *   z: L x N_b x D standard normals (host) or NULL for the host stream of
 *      prob->seed.
 * Blocks until done.  Errors: PRIEST_ERR_INVALID (M < 1, N_b not a multiple
 * of M, counts), PRIEST_ERR_NUMERIC, PRIEST_ERR_CUDA. */
priest_status priest_plan_multi(priest_ctx *ctx, const priest_problem *prob, int M, const double *mu0,
                                const double *cov0, const double *z, priest_result *best, int *best_dist,
                                priest_result *per_dist);

/* Serving (continuous batching).  priest_submit copies the problem, queues
 * it and returns a ticket at once.  A worker thread admits queued requests in
 * arrival order while their device buffers fit the budget (cfg.hbm_budget,
 * allocated once at the first submit) and cfg.serve_slots, and advances every
 * admitted request by one CEM iteration per step, all of them in shared
 * launches: one persistent projection launch per (dims, free-coefficient
 * count) group, one selection and one refit launch.  Requests submitted while
 * others are on the device join at the next step; memory of finished
 * requests returns to the budget at once.  The standard-normal draws come
 * from prob->seed through the same stream as priest_rng_normal, computed on
 * the device (see priest_rng_normal_device).  Each request's solve is Alg. 1
 * exactly as priest_plan computes it (the shared launches do not mix data
 * between requests), except for warm starts:
 *   robot_id >= 0 keeps the request's final sampling mean, covariance and
 *   last-projection multipliers resident on the device; the robot's next
 *   request with the same D and sample count starts from that mean and
 *   covariance and uses those multipliers as lambda^0 of its first CEM
 *   iteration.  A robot's requests run one after another.  Resident robot
 *   states are dropped least recently used first when memory is needed.
 * Errors: PRIEST_ERR_INVALID (as priest_plan), PRIEST_ERR_BUDGET (the
 * request alone exceeds the budget), PRIEST_ERR_NOMEM (the budget cannot be
 * allocated). */
priest_status priest_submit(priest_ctx *ctx, const priest_problem *prob, uint64_t *ticket);

/* PRIEST_PENDING until the ticket's solve is done, then PRIEST_OK with its
 * result (result.status holds the solve's own status: PRIEST_OK,
 * PRIEST_ERR_NUMERIC or PRIEST_ERR_CUDA) and the ticket is released.
 * PRIEST_ERR_INVALID for a ticket never issued or already released. */
priest_status priest_poll(priest_ctx *ctx, uint64_t ticket, priest_result *out);

/* As priest_poll, but blocks until the result is there or timeout_ms has
 * passed (negative: no limit); PRIEST_ERR_TIMEOUT leaves the ticket pending. */
priest_status priest_wait(priest_ctx *ctx, uint64_t ticket, double timeout_ms, priest_result *out);

/* Counters of the serving loop. */
typedef struct {
    int64_t submitted;     /* tickets issued */
    int64_t completed;     /* results produced */
    int64_t steps;         /* shared CEM-iteration steps run */
    int64_t slot_steps;    /* requests summed over steps (mean batch = slot_steps / steps) */
    int64_t max_active;    /* most requests in one step */
    int64_t warm_starts;   /* requests started from a robot's resident state */
    int64_t deferred;      /* admission passes that stopped at a request waiting for memory */
    int64_t evictions;     /* resident robot states dropped to make room */
    size_t budget_bytes;   /* device bytes the loop admits into */
    size_t peak_bytes;     /* most of them held at once */
} priest_serve_stats;

priest_status priest_serve_stats_get(priest_ctx *ctx, priest_serve_stats *out);

/* The host Gaussian stream used by priest_plan: SplitMix64 (Steele, Lea,
 * Flood 2014) seeded with `seed`, 53-bit uniforms u = (x >> 11) 2^-53,
 * Box-Muller on (1 - u1, u2) giving cos then sin.  count >= 0 values.
 * Host-only; needs no GPU. */
priest_status priest_rng_normal(uint64_t seed, int64_t count, double *out);

/* The same stream computed on the device: count values into out_dev
 * (device, caller-owned) on cuda_stream (NULL = legacy default stream).  The
 * 53-bit uniforms are bit-identical to the host stream's; the values differ
 * from priest_rng_normal's by the last-place rounding of log, sqrt, cos and
 * sin.  Asynchronous. */
priest_status priest_rng_normal_device(uint64_t seed, int64_t count, double *out_dev, void *cuda_stream);

/* Device-resident problems for callers that keep inputs in HBM.
 * priest_load copies the problem (obstacles, boundary values) to device
 * memory owned by the returned handle and sizes its work buffers. */
priest_status priest_load(priest_ctx *ctx, const priest_problem *prob, priest_loaded **out);
priest_status priest_unload(priest_ctx *ctx, priest_loaded *h);

/* Full solve of a loaded problem, asynchronous on the context stream.
 * z_dev: L x N x D standard normals in device memory (caller-owned).
 * out_dev: device buffer of D + 4 doubles, written with
 * [xi_best (D), resid, cost, c_aug, best_index]. */
priest_status priest_plan_device(priest_ctx *ctx, priest_loaded *h, const double *z_dev,
                                 double *out_dev);

/* Projection of n caller-provided samples of a loaded problem, asynchronous
 * on the context stream; device pointers as in priest_project. */
priest_status priest_project_device(priest_ctx *ctx, priest_loaded *h, int n, const double *xi_dev,
                                    double *lambda_dev, double *xi_bar_dev, double *resid_dev,
                                    double *cost_dev);

/* Batched solve (Alg. 1 for every problem) in shared launches: one setup
 * launch for all problems, then per CEM iteration one persistent projection
 * launch over the samples of every problem (CTAs pull (problem, sample range)
 * items, most expensive first), one selection launch and one refit launch.
 * Problems may differ in sample count, time stamps, horizon, bounds and
 * obstacles; they must share dims, degree and bc_final_mask.
 * probs: n handles from priest_load; z_dev[i]: L x N_i x D draws (device);
 * out_dev[i]: D + 4 doubles (device), laid out as in priest_plan_device.
 * The first call for a given (probs, z_dev, out_dev) list runs the launches
 * directly and records them in a CUDA graph; later calls with the same list
 * replay the graph.  Asynchronous on the context stream.  Errors:
 * PRIEST_ERR_INVALID (mixed dims / degree / mask, n < 1), PRIEST_ERR_CUDA. */
priest_status priest_plan_batch(priest_ctx *ctx, int n, priest_loaded *const *probs,
                                const double *const *z_dev, double *const *out_dev);

/* Batched solve through host buffers (Alg. 1 for every problem, in the shared
 * launches of priest_plan_batch): probs (n host structs, obstacle arrays
 * host memory), z[i] = L x N_i x D standard normals of problem i (host;
 * from page-locked buffers the draws are read in place by a transfer kernel,
 * those of the second and later CEM iterations while the first projection
 * runs; pageable buffers are copied by DMA first), out[i] = problem
 * i's result (host; xi_best, resid, cost, c_aug, best_index and the final
 * mean; latency_ms 0).  Problems must share dims, degree and bc_final_mask;
 * every problem starts from the default distribution (straight-line mean,
 * init_std^2 I).  The context keeps the problems resident between calls:
 * while every problem keeps its layout (dims, degree, mask, n_p, horizon,
 * obstacle count and its static / moving split, sample counts, bounds flag)
 * a call only uploads the obstacles, boundary values and draws, replays the
 * recorded launches and copies the results back; a new layout replaces the
 * resident set (device allocations, autotuning and graph recording on that
 * call).  Blocks until done.  Errors: PRIEST_ERR_INVALID (as priest_plan,
 * mixed dims / degree / mask, n < 1), PRIEST_ERR_NOMEM, PRIEST_ERR_NUMERIC
 * (also written to every result's status), PRIEST_ERR_CUDA. */
priest_status priest_plan_batch_host(priest_ctx *ctx, int n, const priest_problem *probs, const double *const *z,
                                     priest_result *out);

/* Batched projection (Sec. III-A, Appendix eqs. comp_alpha .. comp_zeta):
 * for every loaded problem i, rows[i] caller-given samples (0 <= rows[i] <=
 * its loaded sample count) are projected as priest_project_device does --
 * xi_bar^0 = Pi_A(xi), lambda^0 from lambda_dev[i] (or 0), cfg.proj_iters
 * iterations, then r and c_1 -- all problems in one persistent launch of the
 * kernel and tilings the batched solves use (one setup launch for all
 * problems first).  Device pointers per problem (caller-owned, row-major):
 * xi_dev[i] (rows x D, read), lambda_dev[i] (rows x D, updated in place; the
 * list or an entry may be NULL: lambda^0 = 0, not written), xi_bar_dev[i]
 * (rows x D), resid_dev[i], cost_dev[i] (rows).  Problems must share dims,
 * degree and bc_final_mask.  Asynchronous on the context stream (the first
 * call of a new problem shape class blocks while the autotuner times its
 * candidate tilings).  Errors: PRIEST_ERR_INVALID, PRIEST_ERR_NOMEM,
 * PRIEST_ERR_CUDA. */
priest_status priest_project_batch(priest_ctx *ctx, int n, priest_loaded *const *probs, const int *rows,
                                   const double *const *xi_dev, double *const *lambda_dev,
                                   double *const *xi_bar_dev, double *const *resid_dev, double *const *cost_dev);

/* The selections of the last CEM iteration of a solve (Alg. 1,
 * ConstraintEliteSet / EliteSet): h a loaded problem after priest_plan_device,
 * or NULL for the context's last host-buffer solve (priest_plan,
 * priest_plan_z, priest_plan_plain).  elite_out: the N_elite indices of the
 * EliteSet in ascending (c_aug, index) order; resid_out, cost_out: r and c_1
 * of all N projected samples of that iteration (the ConstraintEliteSet is the
 * N_proj least (r, index)).  Host buffers, each may be NULL.  Waits for the
 * context stream.  Errors: PRIEST_ERR_INVALID (no solve), PRIEST_ERR_CUDA. */
priest_status priest_read_elites(priest_ctx *ctx, const priest_loaded *h, int *elite_out, double *resid_out,
                                 double *cost_out);

/* Instrumentation: the projection kernel of the context's latest projection
 * launch: 0 the chunked kernel, 1 the point-owner FP32 kernel, 2 the
 * tensor-core kernel (PRIEST_MIXED_BF16); -1 before the first launch. */
int priest_last_kernel(const priest_ctx *ctx);

/* Instrumentation: the uniform grid over the static obstacles that the set-up
 * step builds into a problem's FP32 tables (Sec. III-A, eq. comp_d: the point-
 * owner kernel's neighbour-list builds screen a point's cell instead of every
 * static obstacle).  h a loaded problem after a set-up, or NULL for the
 * context's last host-buffer solve.  out[3] (host): cells in x, cells in y,
 * cell entries; all 0 when the problem has no grid (fewer than 16 static
 * obstacles, no list margin, or a cell of more than 64 obstacles).  Waits for
 * the context stream.  Errors: PRIEST_ERR_INVALID (NULL ctx / out, nothing
 * loaded, no FP32 tables), PRIEST_ERR_CUDA. */
priest_status priest_grid_info(priest_ctx *ctx, const priest_loaded *h, int *out);

/* The plain per-problem FP32 path: the same computation as priest_plan /
 * priest_project (same readings, same draws, FP32 projection), implemented
 * as one kernel per step with every intermediate (trajectory tiles, residual
 * tiles, coefficients, multipliers) in device memory and one problem at a
 * time -- a direct GPU port of the method, kept as the comparison point of
 * the fused, batched and serving forms.  Needs cfg.precision == PRIEST_FP32
 * (else PRIEST_ERR_INVALID).  Arguments as priest_plan_z (z NULL: the host
 * stream from prob->seed), priest_plan_device and priest_project. */
priest_status priest_plan_plain(priest_ctx *ctx, const priest_problem *prob, const double *mu0,
                                const double *cov0, const double *z, priest_result *out);
priest_status priest_plan_plain_device(priest_ctx *ctx, priest_loaded *h, const double *z_dev,
                                       double *out_dev);
priest_status priest_project_plain(priest_ctx *ctx, const priest_problem *prob, int n, const double *xi,
                                   double *lambda_io, double *xi_bar_out, double *resid_out,
                                   double *cost_out);

/* Diagnostic of the tensor-core path used by PRIEST_MIXED_BF16: one product
 * D = A B^T on the 5th-generation tensor core (tcgen05.mma, BF16 inputs,
 * FP32 accumulation in tensor memory), A 128 x k and B n x k row-major BF16
 * bit patterns (host), D 128 x n FP32 (host).  n a multiple of 16 in
 * [16, 256], k a multiple of 16 in [16, 64].  swap = 1 exchanges the two
 * byte strides of the shared-memory descriptors (a layout check: the
 * product is right only for swap = 0); swap = 2 issues no product and no
 * completion signal, so the kernel's bounded completion wait (1 s, then 1 s
 * more for work in flight) runs out: a test of the time-out path, which
 * frees the tensor memory, returns PRIEST_ERR_TIMEOUT and leaves the device
 * usable.  Allocates and synchronises; for tests.  PRIEST_ERR_TIMEOUT if
 * the MMA completion was not observed. */
priest_status priest_tc_selftest(int n, int k, int swap, const uint16_t *a_host, const uint16_t *b_host,
                                 float *d_host);

/* Diagnostic of the Cholesky factor used for the sampling factor
 * chol(Sigma + eps I) (Alg. 1, in the setup and after every refit): factors
 * the D x D symmetric matrix a_host (row-major, host; the lower triangle is
 * read) on one CTA of `threads` threads and writes L (row-major, host, strict
 * upper triangle zero) to l_host.  1 <= D <= PRIEST_MAX_D; threads a multiple
 * of 32 in [32, 1024].  PRIEST_ERR_NUMERIC if a pivot was not a positive
 * normal number (that pivot is taken as 1 and l_host is still written).
 * Allocates and synchronises; for tests. */
priest_status priest_chol_selftest(int D, int threads, const double *a_host, double *l_host);

/* Waits for the context stream and reports any kernel-side error status. */
priest_status priest_sync(priest_ctx *ctx);

/* Number of kernels this context has launched so far (instrumentation). */
int64_t priest_kernel_launches(const priest_ctx *ctx);

/* Instrumentation: while enabled, every projection-kernel launch of the
 * context is bracketed by CUDA events recorded on the stream it runs on.
 * priest_profile_read waits for those events and returns how many launches
 * were bracketed and their summed device time in milliseconds, then clears
 * the record.  Off by default; enabling it adds two event records per launch. */
priest_status priest_profile_enable(priest_ctx *ctx, int enable);
priest_status priest_profile_read(priest_ctx *ctx, int64_t *launches, double *ms);

/* Projection that allocates no device memory (the paper has no counterpart;
 * this entry point exists for callers that cannot call cudaMalloc, such as
 * real-time loops with a fixed memory budget or code running inside a
 * pre-provisioned memory pool).  Same computation as priest_project_device:
 * cfg->proj_iters alternating-minimisation iterations from Pi_A(xi), then r
 * and c_1, in cfg->precision (FP32 or FP64 check mode).
 *   cfg, prob: host structs; prob's obstacle arrays are HOST memory and are
 *     copied into the library's scratch during the call.
 *   xi_dev (n x D, read), lambda_dev (n x D, updated in place, or NULL),
 *   xi_bar_dev (n x D), resid_dev (n), cost_dev (n): caller-owned DEVICE memory.
 *   cuda_stream: stream to run on (NULL = legacy default stream).
 * Kernels: those of priest_project with the cost-model tiling (no timing of
 * candidate tilings): in FP32 the point-owner kernel for the degree-10
 * shapes it covers (five free coefficients, or seven in 2-D), the chunked
 * kernel otherwise; obstacles are reordered static-first on the device, as
 * priest_project orders them.
 * Scratch: one fixed 1 MiB device array inside the library, held by every
 * device that loads it until the process exits; every call shares it and it
 * keeps the last call's contents, so calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * A problem whose tables do not fit returns PRIEST_ERR_BUDGET.  The first
 * call on a device looks up the scratch's device address (set-up), so make
 * that first call before any stream capture.  Blocks until the work is done.
 * Errors are reported by the return code only: PRIEST_ERR_INVALID (bad
 * arguments), PRIEST_ERR_BUDGET (too large for the scratch),
 * PRIEST_ERR_NUMERIC (KKT block not positive definite), PRIEST_ERR_CUDA. */
priest_status priest_project_noalloc(const priest_config *cfg, const priest_problem *prob, int n,
                                     const double *xi_dev, double *lambda_dev, double *xi_bar_dev,
                                     double *resid_dev, double *cost_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
