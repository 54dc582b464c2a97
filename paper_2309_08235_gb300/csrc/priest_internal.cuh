// priest_internal.cuh -- shapes, table layouts and launch entry points shared
// by the library's translation units (setup, projection, CEM stages, C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#include <utility>
#include <vector>

#include "priest.h"

namespace priest {

constexpr int kMaxNv = PRIEST_MAX_NV;
constexpr int kFree0 = 3;  // c_0, c_1, c_2 are fixed by the start position / velocity / acceleration

// Doubles of the per-problem FP64 side buffer: fixed coefficients + Gram blocks.
constexpr int kAuxDoubles = 3 * PRIEST_MAX_NV + 3 * PRIEST_MAX_NV * PRIEST_MAX_NV;

// Bits of the device status word.
enum : int {
    kStatusCholesky = 1,   // non-positive pivot in the covariance Cholesky
    kStatusKkt = 2,        // non-positive pivot in the shared KKT block
    kStatusNaN = 4,
    kStatusTensor = 8,     // a tensor-core completion wait ran out of time
};

// Resolved shape and scalar data of one problem.
struct Shape {
    int dims, degree, nv, n_p, n_obs, n_static, nf, bc_mask, use_bounds;
    double horizon, rho, vmax, amax;
    double smin[3], smax[3];
    double b0[3][3], bf[3][3];
    int N, n_proj, n_elite, D;
    int cost_kind;                          // c_1: 0 = sum |a|^2; 1 = BARN-style
    double w_acc, w_curv, w_path, curv_eps;
    double list_delta;                      // neighbour-list margin: 3/4 of the mean of min(a_j, b_j)
                                            // (0 without obstacles)
};

// Neighbour-list margin of a problem: 3/4 of the mean of the obstacles'
// smallest semi-axes (b_j = a_j in 2-D), 0 without obstacles (center:
// n_obs x dims, semi: n_obs x 2).  Any positive margin gives bitwise the
// same results; this one balanced list length against rebuild frequency on
// the measured workloads (a margin of 0.5 to 1 mean semi-axis changed the
// batched rate by under 2 %).  PRIEST_LIST_MARGIN=<multiple> replaces the
// 3/4 (comparisons).  In dense scenes (64 obstacles or more) it is
// capped so that a ball of radius (mean largest semi-axis + margin) holds
// about two obstacle centres on average at the density of the centres'
// bounding box, keeping the lists short of overflow; it stays at least a
// tenth of the mean semi-axis.
inline double list_margin_scale()
{
    const char *v = getenv("PRIEST_LIST_MARGIN");
    if (!v) return 0.75;
    char *end = nullptr;
    const double x = strtod(v, &end);
    return (end != v && x > 0.0 && x < 1e6) ? x : 0.75;
}

inline double list_margin(int dims, int n_obs, const double *center, const double *semi)
{
    if (n_obs <= 0) return 0.0;
    double s = 0.0, big = 0.0, lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int j = 0; j < n_obs; ++j) {
        const double a = semi[2 * j], b = dims == 3 ? semi[2 * j + 1] : a;
        s += a < b ? a : b;
        big += a > b ? a : b;
        for (int ax = 0; ax < dims; ++ax) {
            const double c = center[j * dims + ax];
            lo[ax] = c < lo[ax] ? c : lo[ax];
            hi[ax] = c > hi[ax] ? c : hi[ax];
        }
    }
    s /= n_obs;
    big /= n_obs;
    double delta = list_margin_scale() * s;
    if (n_obs >= 64) {
        double vol = 1.0;
        for (int ax = 0; ax < dims; ++ax) vol *= (hi[ax] - lo[ax]) + 2.0 * big;
        const double rho = n_obs / vol, pi = 3.141592653589793;
        // radius of the ball that holds two centres on average
        const double r2 = dims == 2 ? __builtin_sqrt(2.0 / (pi * rho)) : __builtin_cbrt(1.5 / (pi * rho));
        const double cap = r2 - big;
        if (cap < delta) delta = cap;
        if (delta < 0.1 * s) delta = 0.1 * s;
    }
    return delta;
}

// c_1 of the final pass (Alg. 1 cost): the point-to-point benchmark's
// squared acceleration, or the BARN-style cost w_acc |a|^2 + w_curv kappa^2 +
// w_path d^2 with kappa = |v x a| / (|v|^2 + eps^2)^(3/2) and d the distance
// to the straight start-goal segment (s, unit u, length len; positions in
// the origin-shifted frame of the tables).
template <typename Real>
struct CostParams {
    int kind;
    Real w_acc, w_curv, w_path, eps2;
    Real s[3], u[3], len;
};

template <typename Real>
inline CostParams<Real> make_cost(const Shape &sh)
{
    CostParams<Real> c;
    c.kind = sh.cost_kind;
    c.w_acc = Real(sh.w_acc);
    c.w_curv = Real(sh.w_curv);
    c.w_path = Real(sh.w_path);
    c.eps2 = Real(sh.curv_eps * sh.curv_eps);
    double u[3] = {0.0, 0.0, 0.0}, len = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        const double org = ax < sh.dims ? 0.5 * (sh.b0[ax][0] + sh.bf[ax][0]) : 0.0;
        c.s[ax] = Real(ax < sh.dims ? sh.b0[ax][0] - org : 0.0);
        u[ax] = ax < sh.dims ? sh.bf[ax][0] - sh.b0[ax][0] : 0.0;
        len += u[ax] * u[ax];
    }
    len = len > 0.0 ? __builtin_sqrt(len) : 0.0;
    for (int ax = 0; ax < 3; ++ax) c.u[ax] = Real(len > 0.0 ? u[ax] / len : 0.0);
    c.len = Real(len);
    return c;
}

template <typename Real, int DIMS>
__host__ __device__ __forceinline__ Real point_cost(const CostParams<Real> &c, const Real *p, const Real *v,
                                                    const Real *a, Real a2)
{
    if (c.kind != 1) return a2;
    Real v2 = Real(0), c2, lam = Real(0), d2 = Real(0);
    for (int ax = 0; ax < DIMS; ++ax) v2 += v[ax] * v[ax];
    if (DIMS == 2) {
        const Real cz = v[0] * a[1] - v[1] * a[0];
        c2 = cz * cz;
    } else {
        const Real cx = v[1] * a[DIMS - 1] - v[DIMS - 1] * a[1], cy = v[DIMS - 1] * a[0] - v[0] * a[DIMS - 1],
                   cz = v[0] * a[1] - v[1] * a[0];
        c2 = cx * cx + cy * cy + cz * cz;
    }
    const Real den = v2 + c.eps2;
    if (c.len > Real(0)) {
        for (int ax = 0; ax < DIMS; ++ax) lam += (p[ax] - c.s[ax]) * c.u[ax];
        lam = lam < Real(0) ? Real(0) : (lam > c.len ? c.len : lam);
    }
    for (int ax = 0; ax < DIMS; ++ax) {
        const Real e = p[ax] - c.s[ax] - lam * c.u[ax];
        d2 += e * e;
    }
    return c.w_acc * a2 + c.w_curv * c2 / (den * den * den) + c.w_path * d2;
}

// Number of coefficients fixed at the final time by the Bernstein end-point
// conditions (mask 0, 1, 3, 7 -> 0, 1, 2, 3).
inline int final_fixed(int mask) { return mask == 7 ? 3 : mask == 3 ? 2 : mask == 1 ? 1 : 0; }

// Obstacle record stride in Real units (see the setup kernel for the fields).
__host__ __device__ inline int obs_stride(int dims) { return dims == 2 ? 12 : 16; }

__host__ __device__ inline size_t align8(size_t x) { return (x + 7) & ~size_t(7); }

// Free-coefficient count rounded up to a multiple of 4 (row stride of the
// packed per-time-stamp basis and of the per-sample coefficient rows).
__host__ __device__ inline int nf_padded(int nf) { return (nf + 3) & ~3; }

// Stride of one time stamp in the packed basis: 3 rows of nf_padded(nf),
// plus 4 when needed so the stride is an odd multiple of 4 Real (16-byte
// loads by consecutive lanes then hit distinct bank groups).
__host__ __device__ inline int fb_stride(int nf)
{
    const int s = 3 * nf_padded(nf);
    return ((s / 4) % 2 == 0) ? s + 4 : s;
}

// Uniform grid over the static obstacles in the x-y plane, built by the set-up
// kernel into the FP32 tables: the point-owner kernel's neighbour-list builds
// look up a point's cell instead of screening every static obstacle.  A cell
// lists, in increasing order, the static obstacles whose screening disc (the
// radius the inflated pre-filter can accept, plus slack) meets it; cells are
// at least twice the largest such radius, so an obstacle meets at most 2 x 2
// cells.  Region (4-byte units): header [x0, y0, 1/h, h, nx, ny, entries, 0]
// (nx = 0: no grid), cell starts (uint16, nx * ny + 1), entries (uint16, at
// most 4 per obstacle), then the set-up's per-obstacle cell ranges.
constexpr int kGridMinStatic = 16;  // fewer static obstacles: screened directly
constexpr int kGridCellMax = 64;    // a fuller cell turns the grid off for the problem
__host__ __device__ inline int grid_side(int ns)
{
    int g = 4;
    while (g < 32 && g * g < 2 * ns) ++g;
    return g;
}
struct GridLayout {
    size_t start, ent, rng, smem, total;  // smem: header, starts and entries (what the kernel stages)
};
__host__ __device__ inline GridLayout grid_layout(int ns)
{
    GridLayout g;
    g.start = 8;
    if (ns < kGridMinStatic) {
        g.ent = g.rng = g.smem = g.total = 8;
        return g;
    }
    const int gs = grid_side(ns);
    g.ent = g.start + align8(size_t(gs * gs + 2) / 2);
    g.rng = g.ent + align8(size_t(2) * ns);
    g.smem = g.rng;
    g.total = g.rng + align8(size_t(ns));
    return g;
}

// Per-problem device tables, in units of Real, one contiguous buffer.
struct TableLayout {
    size_t basis;  // [3][n_p][nv]   P, Pd, Pdd
    size_t fb;     // [n_p][fb_stride] free columns of P, Pd, Pdd per time stamp (rows of nfp)
    size_t base;   // [3][dims][n_p] contribution of the fixed coefficients
    size_t W;      // [nf][nf]       (I + rho Q_FF)^-1
    size_t obs;    // [n_obs][stride] pre-scaled obstacle records (static first)
    size_t tval;   // [n_p]          time stamps
    size_t origin; // [3]            shift applied to positions and obstacle centres
    size_t total;
    size_t grid;   // FP32 tables only: the static-obstacle grid (grid_layout of n_static <= n_obs)
    size_t total32; // floats of an FP32 table buffer (total + the grid region)
};

__host__ __device__ inline TableLayout table_layout(int dims, int nv, int nf, int n_p, int n_obs)
{
    TableLayout t;
    size_t o = 0;
    t.basis = o;
    o = align8(o + size_t(3) * n_p * nv);
    t.fb = o;
    o = align8(o + size_t(n_p) * fb_stride(nf));
    t.base = o;
    o = align8(o + size_t(3) * n_p * dims);
    t.W = o;
    o = align8(o + size_t(nf) * nf);
    t.obs = o;
    o = align8(o + size_t(n_obs) * obs_stride(dims));
    t.tval = o;
    o = align8(o + size_t(n_p));
    t.origin = o;
    o = align8(o + 3);
    t.total = o;
    t.grid = o;
    t.total32 = o + grid_layout(n_obs).total;
    return t;
}

// Inputs of the setup kernel (step a0): FP64 basis, fixed coefficients,
// shared KKT block inverse, obstacle records; optionally the default mean /
// covariance and the Cholesky factor of the first sampling covariance.
struct SetupParams {
    Shape sh;
    const double *center, *vel, *semi;  // raw obstacles (device), static first
    double *tab64;                      // FP64 tables (always written)
    void *tab;                          // working tables: == tab64 for FP64, else float copy
    int real_is_double;
    double *cB;                         // [3][kMaxNv] fixed coefficient values (FP64), followed by
                                        // [3][kMaxNv][kMaxNv] Gram blocks of the free coefficients
    int shape_ready;                    // 1: basis, time stamps and Gram blocks are already in place
    double *mu, *cov, *L;               // D, D x D, D x D (plan mode) or null
    int default_mu, default_cov;
    double init_std, chol_eps;
    int *status;
};

// Inputs of the fused projection kernel.
template <typename Real>
struct ProjParams {
    int dims, nv, nf, n_p, n_obs, n_static, use_bounds;
    int N, K, S, C, WS, want_lambda, mode;  // mode 0: xi_in given; 1: xi = mu + L z; WS warps per sample
    int seg_len;                            // mode 1: samples per distribution (mu, Lc hold one per
                                            // segment of seg_len rows; 0 = a single distribution)
    Real list_delta;                        // point-owner kernel: neighbour-list margin (0: screen every
                                            // obstacle in every iteration)
    int list_grid;                          // 1: list builds use the tables' static-obstacle grid
    CostParams<Real> cost;
    Real rho, vmax, amax, smin[3], smax[3];
    const Real *tab;
    TableLayout lay;
    const double *cB;
    const double *xi_in, *mu, *Lc, *z, *lam_in;
    double *xi_bar, *lam_out, *r_out, *c1_out;
};

// Plan of a tensor-core projection launch (project_tc.cu): M-tiles of 128
// trajectory points, obstacle columns (static then moving, each padded to 16),
// column segments per tile (units of work), operand layout.
struct TcPlan {
    int rows, tiles, ns_pad, nm_pad, nseg, regw, kA;  // regw: tensor-memory columns of one segment region
    uint32_t ncols;                            // tensor-memory columns allocated
    size_t smem;                               // dynamic shared memory (0: shape not supported)
    size_t off_marg, off_a, off_bs, off_bm;    // byte offsets of margins, A, B_static, B_moving
};

struct TcParams {
    ProjParams<float> p;                       // p.S samples per CTA, p.C = nseg
    const double *center, *vel, *semi;         // FP64 obstacles, static first
    const double *origin64;                    // frame origin (FP64 tables)
    int *status;
    TcPlan tp;
};

TcPlan tc_plan(const Shape &sh, int S);
TcPlan tc_choose(const Shape &sh, int N, int n_sm, int *S_out);
cudaError_t launch_project_tc(const TcParams &q, cudaStream_t st);

// Tiling chosen for one projection launch.
struct Tiling {
    int S;        // samples per CTA
    int C;        // obstacle chunks per CTA
    int threads;  // CTA size
    int R;        // points per obstacle-loop item / per thread (template value)
    int ws;       // warps per sample
    size_t smem;  // dynamic shared memory bytes
    int kind = 0; // 0: chunked kernel (project_kernel.cuh); 1: point-owner FP32 kernel (project_pts.cuh)
};

// FP32 point-owner kernel (project_pts.cu): degree 10 with 5 free coefficients
// (2-D, 3-D) or 7 (2-D).
bool pts_supported(const Shape &sh);
bool pts_span_ok(const Shape &sh, int R);
bool pts_batch_ok(const Shape &sh);
size_t pts_smem_bytes(const Shape &sh, int S, int R);
int pts_threads(const Shape &sh, int S, int R);
int pts_max_threads(int R);                 // largest CTA of the single-problem variants
int pts_batch_threads(const Shape &sh);     // CTA of the persistent variant for sh

// Raises a kernel's dynamic shared-memory limit to `bytes` (the default limit
// counts static shared memory too, so it is raised whenever more is asked
// than granted so far); `granted` caches the largest value set.
template <typename Kernel>
inline cudaError_t reserve_smem(Kernel kernel, size_t bytes, size_t &granted)
{
    if (bytes <= granted) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) granted = bytes;
    return e;
}

// Programmatic dependent launch along the solve's chain of kernels (setup ->
// projection -> selection -> refit -> projection ...): a kernel launched with
// launch_pdl may be scheduled while the previous kernel of the stream still
// runs; it calls pdl_wait() before touching any memory, which returns once
// that kernel has completed and its writes are visible, so the order of
// memory accesses is that of plain stream order and only the launch latency
// overlaps.  pdl_trigger() lets the next kernel be scheduled.  Both are no-ops
// for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Arguments of the selection and refit stages of one problem (batched launches).
struct CemArgs {
    int N, n_proj, n_elite, D;
    const double *r, *c1, *xb;
    int *elite;
    double sigma, gamma, chol_eps;
    double *mu, *cov, *mu_new, *L;
    unsigned *counter;
    int *status;
    double *best_out;
};

// One run of the standard-normal stream: `count` values of the stream seeded
// with `seed`, written to `out` (device).  The same launch zeroes `status`
// and `counter` when they are not null (the status word and refit counter of
// a request that starts its solve).
struct GaussJob {
    unsigned long long seed;
    long long count;
    double *out;
    int *status;
    unsigned *counter;
};

// Inputs and HBM workspace of the plain per-problem FP32 path (plain.cu).
struct PlainParams {
    int dims, nv, nf, n_p, np4, n_obs, use_bounds, N, K, mode;  // mode 0: xi_in given; 1: xi = mu + L z
    float rho, vmax, amax, smin[3], smax[3];
    CostParams<float> cost;
    const float *tab;
    TableLayout lay;
    const double *cB;
    const double *xi_in, *mu, *Lc, *z, *lam_in;
    double *xi_bar, *lam_out, *r_out, *c1_out;
    float *c, *xiF, *lam, *pos, *vel, *acc, *so, *rv, *ra;  // workspace (plain_carve)
};

// ---- launchers (defined in the .cu files) --------------------------------
size_t plain_work_floats(int dims, int nv, int nf, int n_p, int N);
void plain_carve(PlainParams &p, float *work);
cudaError_t launch_plain_project(const PlainParams &p, cudaStream_t st, int64_t *launches);
cudaError_t launch_normal_batch(const GaussJob *jobs_dev, int n_jobs, long long max_count, cudaStream_t st);
cudaError_t launch_normal(unsigned long long seed, long long count, double *out_dev, cudaStream_t st);
cudaError_t launch_setup(const SetupParams &p, cudaStream_t st);
cudaError_t launch_setup_batch(const SetupParams *ps_dev, int n, size_t smem, cudaStream_t st);
size_t setup_smem_bytes(const Shape &sh);
cudaError_t launch_select_batch(const CemArgs *args_dev, int n, size_t smem, cudaStream_t st);
cudaError_t launch_refit_batch(const CemArgs *args_dev, int n, int D_max, size_t smem, cudaStream_t st);
size_t select_smem_bytes(int N);
size_t refit_smem_bytes(int D, int n_elite);

// Persistent batched projection over the (problem, first sample) items; kind
// selects the chunked (0) or point-owner FP32 (1) kernel.
template <typename Real>
cudaError_t launch_project_batch(const ProjParams<Real> *params_dev, const int2 *items_dev, int n_items,
                                 int *counter_dev, int dims, int R, int threads, int nf, int nv, int want_lambda,
                                 size_t smem, int grid, cudaStream_t st, int kind = 0);


template <typename Real>
size_t project_smem_bytes(const Shape &sh, int S, int C);

template <typename Real>
cudaError_t launch_project(const ProjParams<Real> &p, const Tiling &t, cudaStream_t st);
cudaError_t launch_project_pts(const ProjParams<float> &p, const Tiling &t, cudaStream_t st);
cudaError_t launch_project_pts_batch(const ProjParams<float> *params, const int2 *items, int n_items, int *counter,
                                     int dims, int nf, int R, int want_lambda, size_t smem, int grid, cudaStream_t st);

template <typename Real>
Tiling choose_tiling(const Shape &sh, int n_samples, int n_sm);

template <typename Real>
std::vector<Tiling> tiling_candidates(const Shape &sh, int n_samples, int n_sm);

// Tiling of one problem inside a batched (persistent) launch: the batched
// variant's CTA size, warp groups of two (2-D FP32) or one warp, chunk count
// from the cost model.  smem == 0 signals a problem too large for one CTA.
template <typename Real>
Tiling batch_tiling(const Shape &sh);
template <typename Real>
std::vector<Tiling> batch_candidates(const Shape &sh);

// One compiled kernel variant (explicitly instantiated in project_f32_*.cu /
// project_f64.cu).
template <typename Real, int DIMS, int R, int THREADS>
cudaError_t launch_variant(const ProjParams<Real> &p, const Tiling &t, cudaStream_t st);
template <typename Real, int DIMS, int R, int THREADS>
cudaError_t launch_variant_batch(const ProjParams<Real> *params, const int2 *items, int n_items, int *counter,
                                 int nf, int nv, int want_lambda, size_t smem, int grid, cudaStream_t st);

cudaError_t launch_select(int N, const double *r, const double *c1, int n_proj, int n_elite,
                          int *elite_idx, cudaStream_t st);

cudaError_t launch_refit(int D, const double *xb, const double *r, const double *c1,
                         const int *elite, int n_elite, double sigma, double gamma, double chol_eps,
                         double *mu, double *cov, double *mu_new, double *L, unsigned *counter,
                         int *status, double *best_out, cudaStream_t st);

}  // namespace priest
