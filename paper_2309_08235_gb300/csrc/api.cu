// api.cu -- the C ABI of priest.h: contexts, validation, device-resident
// problems, the plan / project pipelines (Alg. 1 as a sequence of kernel
// launches on one stream), the host Gaussian stream and the serving worker.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "host_internal.h"

using namespace priest;
using namespace priest::host;

// Descriptors and recorded launch sequence of one batched solve.
namespace priest {
struct BatchPlan {
    void *dev = nullptr;            // one allocation: params, setup params, CEM args, items, counters
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n = 0, n_items = 0, L = 0, D_max = 0;
    size_t smem_proj = 0, smem_setup = 0, smem_select = 0, smem_refit = 0;
    SetupParams *setup_dev = nullptr, *setup_dev_ready = nullptr;
    void *params_dev = nullptr;     // L x n ProjParams<Real>
    CemArgs *cem_dev = nullptr;
    int2 *items_dev = nullptr;
    int *counters_dev = nullptr;    // L
    int dims = 0, nf = 0, nv = 0, dbl = 0;
    int kind = 0, R = 4;            // projection kernel of the batch (Tiling::kind) and its points per item
    std::vector<int2> items_host;   // the uploaded items (a refresh must reproduce them)
    std::vector<cudaEvent_t> ev;    // 2 L events recorded around the projection launches of the graph
    std::vector<cudaGraphNode_t> ev_nodes;  // their record nodes, in the same order
    bool ev_swapped = false;        // the nodes point at events of the context's pool
    cudaEvent_t zwait = nullptr;    // not owned: recorded once the draws of CEM iterations >= 1 are
                                    // in place (host-buffer solves); the second projection waits on it
};

// One piece of a transfer for xfer_kernel: count doubles from src to dst
// (either may be the device view of pinned host memory).
struct XferChunk {
    const double *src;
    double *dst;
    long long count;
};

// Resident problems, draws and results of the batched solve through host
// buffers (priest_plan_batch_host).
struct HostBatch {
    std::vector<double> key;                // layout of every problem (host_layout_key)
    std::vector<priest_loaded *> h;
    int n = 0;
    double *zdev = nullptr;                 // draws of all problems
    double *odev = nullptr;                 // results, ostride doubles per problem
    size_t ostride = 0;
    char *stage = nullptr;                  // pinned: obstacle spans, then results, then means
    char *stage_dev = nullptr;              // the stage's device view (nullptr: copies instead)
    size_t out_off = 0, mu_off = 0;
    std::vector<size_t> z_off, ob_off, ob_bytes;
    XferChunk *xin = nullptr, *xout = nullptr;  // pinned chunk tables of the two gathers
    XferChunk *xin_dev = nullptr, *xout_dev = nullptr, *xside = nullptr, *xside_dev = nullptr;
    size_t xin_cap = 0, xout_cap = 0, xside_cap = 0;
    cudaStream_t cstream = nullptr;         // transfer of the draws of CEM iterations >= 1, beside the solve
    cudaEvent_t zev = nullptr;              // recorded on cstream after those copies
};
}  // namespace priest

namespace priest {
namespace host {

priest_status fail(priest_ctx *ctx, priest_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

priest_status cuda_fail(priest_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, PRIEST_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Resolves the shape of a problem against the context defaults and checks it.
priest_status resolve(const priest_config &c, const priest_problem *pr, int n_override, Shape &sh, std::string &why)
{
    auto fail = [&why](priest_status st, const char *msg) {
        why = msg;
        return st;
    };
    if (!pr) return fail(PRIEST_ERR_INVALID, "problem is NULL");
    std::memset(&sh, 0, sizeof(sh));
    sh.dims = pr->dims ? pr->dims : c.dims;
    sh.degree = c.degree;
    sh.nv = sh.degree + 1;
    sh.n_p = pr->n_p ? pr->n_p : c.n_p;
    sh.horizon = pr->horizon > 0 ? pr->horizon : c.horizon;
    sh.rho = c.rho;
    sh.vmax = pr->vmax > 0 ? pr->vmax : c.vmax;
    sh.amax = pr->amax > 0 ? pr->amax : c.amax;
    sh.use_bounds = c.use_bounds ? 1 : 0;
    sh.bc_mask = pr->bc_final_mask;
    sh.n_obs = pr->n_obs;
    if (sh.dims != 2 && sh.dims != 3) return fail(PRIEST_ERR_INVALID, "dims must be 2 or 3");
    if (sh.degree < 5 || sh.degree > 15) return fail(PRIEST_ERR_INVALID, "degree must be in [5, 15]");
    if (sh.n_p < 2 || sh.n_p > PRIEST_MAX_NP) return fail(PRIEST_ERR_INVALID, "n_p out of range");
    if (!(sh.horizon > 0) || !std::isfinite(sh.horizon)) return fail(PRIEST_ERR_INVALID, "horizon must be > 0");
    if (!(sh.rho > 0) || !std::isfinite(sh.rho)) return fail(PRIEST_ERR_INVALID, "rho must be > 0");
    if (!(sh.vmax > 0) || !(sh.amax > 0) || !std::isfinite(sh.vmax) || !std::isfinite(sh.amax))
        return fail(PRIEST_ERR_INVALID, "vmax and amax must be > 0");
    if (sh.bc_mask != 0 && sh.bc_mask != 1 && sh.bc_mask != 3 && sh.bc_mask != 7)
        return fail(PRIEST_ERR_INVALID, "bc_final_mask must be 0, 1, 3 or 7");
    if (sh.n_obs < 0 || sh.n_obs > PRIEST_MAX_OBS) return fail(PRIEST_ERR_INVALID, "n_obs out of range");
    if (sh.n_obs > 0 && (!pr->center || !pr->semi))
        return fail(PRIEST_ERR_INVALID, "obstacle arrays are NULL");
    for (int ax = 0; ax < sh.dims; ++ax)
        for (int q = 0; q < 3; ++q) {
            if (!std::isfinite(pr->b0[ax][q]) || !std::isfinite(pr->bf[ax][q]))
                return fail(PRIEST_ERR_INVALID, "boundary values must be finite");
            sh.b0[ax][q] = pr->b0[ax][q];
            sh.bf[ax][q] = pr->bf[ax][q];
        }
    for (int ax = 0; ax < 3; ++ax) {
        sh.smin[ax] = c.smin[ax];
        sh.smax[ax] = c.smax[ax];
    }
    for (int j = 0; j < sh.n_obs; ++j) {
        const double a = pr->semi[2 * j], b = pr->semi[2 * j + 1];
        if (!(a > 0) || !std::isfinite(a) || (sh.dims == 3 && (!(b > 0) || !std::isfinite(b))))
            return fail(PRIEST_ERR_INVALID, "obstacle semi-axes must be finite and > 0");
        for (int ax = 0; ax < sh.dims; ++ax) {
            if (!std::isfinite(pr->center[j * sh.dims + ax]))
                return fail(PRIEST_ERR_INVALID, "obstacle centre is not finite");
            if (pr->vel && !std::isfinite(pr->vel[j * sh.dims + ax]))
                return fail(PRIEST_ERR_INVALID, "obstacle velocity is not finite");
        }
    }
    sh.cost_kind = pr->cost_kind;
    sh.w_acc = pr->w_acc;
    sh.w_curv = pr->w_curv;
    sh.w_path = pr->w_path;
    sh.curv_eps = pr->curv_eps;
    sh.list_delta = list_margin(sh.dims, sh.n_obs, pr->center, pr->semi);
    if (sh.cost_kind != 0 && sh.cost_kind != 1) return fail(PRIEST_ERR_INVALID, "cost_kind must be 0 or 1");
    if (sh.cost_kind == 1 &&
        (!(sh.w_acc >= 0) || !(sh.w_curv >= 0) || !(sh.w_path >= 0) || !std::isfinite(sh.w_acc) ||
         !std::isfinite(sh.w_curv) || !std::isfinite(sh.w_path) || !(sh.curv_eps > 0) || !std::isfinite(sh.curv_eps)))
        return fail(PRIEST_ERR_INVALID, "cost weights must be finite and >= 0, curv_eps > 0");
    sh.nf = sh.nv - kFree0 - final_fixed(sh.bc_mask);
    sh.D = sh.dims * sh.nv;
    sh.N = n_override >= 0 ? n_override : (pr->n_samples ? pr->n_samples : c.n_samples);
    if (sh.N < 0 || sh.N > PRIEST_MAX_SAMPLES) return fail(PRIEST_ERR_INVALID, "sample count out of range");
    if (n_override < 0) {
        if (sh.N < 1) return fail(PRIEST_ERR_INVALID, "n_samples must be >= 1");
        int np = pr->n_proj ? pr->n_proj : c.n_proj;
        int ne = pr->n_elite ? pr->n_elite : c.n_elite;
        if (np <= 0) np = std::max(1, (80 * sh.N) / 110);
        if (ne <= 0) ne = std::max(1, std::min(np, sh.N / 10));
        if (np > sh.N || ne > np || ne > PRIEST_MAX_ELITE)
            return fail(PRIEST_ERR_INVALID, "need n_elite <= n_proj <= n_samples");
        sh.n_proj = np;
        sh.n_elite = ne;
    }
    return PRIEST_OK;
}

// Stable static-first order of the obstacles (moving ones, |v| > 0, last).
void order_obstacles(const Shape &sh, const double *center, const double *vel, const double *semi,
                     std::vector<double> &c, std::vector<double> &v, std::vector<double> &s, int &n_static)
{
    const int n = sh.n_obs, d = sh.dims;
    c.assign(size_t(std::max(n, 1)) * d, 0.0);
    v.assign(size_t(std::max(n, 1)) * d, 0.0);
    s.assign(size_t(std::max(n, 1)) * 2, 1.0);
    std::vector<int> order;
    order.reserve(n);
    auto moving = [&](int j) {
        if (!vel) return false;
        for (int ax = 0; ax < d; ++ax)
            if (vel[j * d + ax] != 0.0) return true;
        return false;
    };
    for (int j = 0; j < n; ++j)
        if (!moving(j)) order.push_back(j);
    n_static = int(order.size());
    for (int j = 0; j < n; ++j)
        if (moving(j)) order.push_back(j);
    for (int k = 0; k < n; ++k) {
        const int j = order[k];
        for (int ax = 0; ax < d; ++ax) {
            c[k * d + ax] = center[j * d + ax];
            v[k * d + ax] = vel ? vel[j * d + ax] : 0.0;
        }
        s[2 * k] = semi[2 * j];
        s[2 * k + 1] = (d == 3) ? semi[2 * j + 1] : semi[2 * j];
    }
}

size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

Carve carve(const Shape &sh, bool fp32, int z_iters, bool proj_buffers)
{
    Carve k;
    size_t o = 0;
    const int nob = std::max(sh.n_obs, 1);
    const TableLayout lay = table_layout(sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs);
    const size_t N = size_t(std::max(sh.N, 1)), D = size_t(sh.D);
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = round_up(o + bytes);
        return at;
    };
    k.center = take(sizeof(double) * nob * sh.dims);
    k.vel = take(sizeof(double) * nob * sh.dims);
    k.semi = take(sizeof(double) * nob * 2);
    k.tab64 = take(sizeof(double) * lay.total);
    k.tab32 = take(fp32 ? sizeof(float) * lay.total32 : 0);
    k.cB = take(sizeof(double) * kAuxDoubles);
    k.mu = take(sizeof(double) * D);
    k.cov = take(sizeof(double) * D * D);
    k.L = take(sizeof(double) * D * D);
    k.mu_new = take(sizeof(double) * D);
    k.xb = take(sizeof(double) * N * D);
    k.r = take(sizeof(double) * N);
    k.c1 = take(sizeof(double) * N);
    k.elite = take(sizeof(int) * std::max(sh.n_elite, 1));
    k.out = take(sizeof(double) * (D + 5));
    k.counter = take(sizeof(unsigned));
    k.z = take(sizeof(double) * size_t(z_iters) * N * D);
    k.xi = take(proj_buffers ? sizeof(double) * N * D : 0);
    k.lam = take(proj_buffers ? sizeof(double) * N * D : 0);
    k.total = o;
    return k;
}

void carve_ptrs(priest_loaded *h, char *b, const Carve &k, bool fp32, int z_iters, bool proj_buffers)
{
    h->center = reinterpret_cast<double *>(b + k.center);
    h->vel = reinterpret_cast<double *>(b + k.vel);
    h->semi = reinterpret_cast<double *>(b + k.semi);
    h->tab64 = reinterpret_cast<double *>(b + k.tab64);
    h->tab32 = fp32 ? reinterpret_cast<float *>(b + k.tab32) : nullptr;
    h->cB = reinterpret_cast<double *>(b + k.cB);
    h->mu = reinterpret_cast<double *>(b + k.mu);
    h->cov = reinterpret_cast<double *>(b + k.cov);
    h->L = reinterpret_cast<double *>(b + k.L);
    h->mu_new = reinterpret_cast<double *>(b + k.mu_new);
    h->xb = reinterpret_cast<double *>(b + k.xb);
    h->r = reinterpret_cast<double *>(b + k.r);
    h->c1 = reinterpret_cast<double *>(b + k.c1);
    h->elite = reinterpret_cast<int *>(b + k.elite);
    h->out = reinterpret_cast<double *>(b + k.out);
    h->counter = reinterpret_cast<unsigned *>(b + k.counter);
    h->z = z_iters ? reinterpret_cast<double *>(b + k.z) : nullptr;
    h->xi = proj_buffers ? reinterpret_cast<double *>(b + k.xi) : nullptr;
    h->lam = proj_buffers ? reinterpret_cast<double *>(b + k.lam) : nullptr;
}

// PRIEST_NEIGHBOUR_LISTS=0 in the environment (read at every launch set-up)
// makes the point-owner kernel screen every obstacle in every iteration
// (comparisons); lists are on otherwise.
bool neighbour_lists()
{
    const char *v = getenv("PRIEST_NEIGHBOUR_LISTS");
    return !(v && std::string(v) == "0");
}

// PRIEST_LIST_GRID=0 (read at every launch set-up): neighbour-list builds
// screen every static obstacle instead of the grid's cell (comparisons; the
// lists, and so the results, are the same).
bool list_grid()
{
    const char *v = getenv("PRIEST_LIST_GRID");
    return !(v && std::string(v) == "0");
}

template <typename Real>
ProjParams<Real> proj_params(const priest_ctx *ctx, const priest_loaded *h, const Tiling &t)
{
    const Shape &sh = h->sh;
    ProjParams<Real> p;
    std::memset(&p, 0, sizeof(p));
    p.dims = sh.dims;
    p.nv = sh.nv;
    p.nf = sh.nf;
    p.n_p = sh.n_p;
    p.n_obs = sh.n_obs;
    p.n_static = sh.n_static;
    p.use_bounds = sh.use_bounds;
    p.K = ctx->cfg.proj_iters;
    p.S = t.S;
    p.C = t.C;
    p.WS = t.ws;
    p.rho = Real(sh.rho);
    p.vmax = Real(sh.vmax);
    p.amax = Real(sh.amax);
    for (int ax = 0; ax < 3; ++ax) {
        p.smin[ax] = Real(sh.smin[ax]);
        p.smax[ax] = Real(sh.smax[ax]);
    }
    p.tab = std::is_same<Real, double>::value ? reinterpret_cast<const Real *>(h->tab64)
                                              : reinterpret_cast<const Real *>(h->tab32);
    p.lay = table_layout(sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs);
    p.cB = h->cB;
    p.seg_len = h->seg_len;
    p.cost = make_cost<Real>(sh);
    p.list_delta = neighbour_lists() ? Real(sh.list_delta) : Real(0);
    p.list_grid = list_grid() ? 1 : 0;
    return p;
}

SetupParams setup_params(const priest_ctx *ctx, const priest_loaded *h, bool plan_mode, int *status)
{
    SetupParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.sh = h->sh;
    sp.center = h->center;
    sp.vel = h->vel;
    sp.semi = h->semi;
    sp.tab64 = h->tab64;
    sp.tab = h->tab32 ? static_cast<void *>(h->tab32) : static_cast<void *>(h->tab64);
    sp.real_is_double = h->tab32 ? 0 : 1;
    sp.cB = h->cB;
    if (plan_mode) {
        sp.mu = h->mu;
        sp.cov = h->cov;
        sp.L = h->L;
        sp.default_mu = h->default_mu;
        sp.default_cov = h->default_cov;
    }
    sp.init_std = ctx->cfg.init_std;
    sp.chol_eps = ctx->cfg.chol_eps;
    sp.status = status;
    sp.shape_ready = h->shape_ready ? 1 : 0;
    return sp;
}

CemArgs cem_args(const priest_ctx *ctx, const priest_loaded *h, int *status, double *best_out)
{
    const Shape &sh = h->sh;
    CemArgs a;
    std::memset(&a, 0, sizeof(a));
    a.N = sh.N;
    a.n_proj = sh.n_proj;
    a.n_elite = sh.n_elite;
    a.D = sh.D;
    a.r = h->r;
    a.c1 = h->c1;
    a.xb = h->xb;
    a.elite = h->elite;
    a.sigma = ctx->cfg.sigma_lr;
    a.gamma = ctx->cfg.gamma;
    a.chol_eps = ctx->cfg.chol_eps;
    a.mu = h->mu;
    a.cov = h->cov;
    a.mu_new = h->mu_new;
    a.L = h->L;
    a.counter = h->counter;
    a.status = status;
    a.best_out = best_out;
    return a;
}

void fill_result(const Shape &sh, const double *host_out, const double *host_mu, priest_result *res)
{
    std::memset(res, 0, sizeof(*res));
    res->status = PRIEST_OK;
    res->D = sh.D;
    for (int d = 0; d < sh.D; ++d) {
        res->xi_best[d] = host_out[d];
        res->mu[d] = host_mu[d];
    }
    res->resid = host_out[sh.D];
    res->cost = host_out[sh.D + 1];
    res->c_aug = host_out[sh.D + 2];
    res->best_index = int(host_out[sh.D + 3]);
}

template ProjParams<float> proj_params<float>(const priest_ctx *, const priest_loaded *, const Tiling &);
template ProjParams<double> proj_params<double>(const priest_ctx *, const priest_loaded *, const Tiling &);

}  // namespace host
}  // namespace priest

namespace {

#define PRIEST_CUDA(ctx, call)                                      \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);  \
    } while (0)

bool is_fin(double x) { return std::isfinite(x); }

priest_status resolve(priest_ctx *ctx, const priest_problem *pr, int n_override, Shape &sh)
{
    std::string why;
    const priest_status s = host::resolve(ctx->cfg, pr, n_override, sh, why);
    if (s != PRIEST_OK) return fail(ctx, s, why);
    return PRIEST_OK;
}

void free_loaded(priest_loaded *h)
{
    if (!h) return;
    if (h->block) cudaFree(h->block);
    delete h;
}

// Allocates and fills a loaded problem (obstacles uploaded on `st`).
priest_status make_loaded(priest_ctx *ctx, const Shape &sh_in, const double *center, const double *vel,
                          const double *semi, int z_iters, bool proj_buffers, cudaStream_t st,
                          priest_loaded **out)
{
    Shape sh = sh_in;
    std::vector<double> c, v, s;
    order_obstacles(sh, center, vel, semi, c, v, s, sh.n_static);
    const bool fp32 = ctx->cfg.precision != PRIEST_FP64_CHECK;
    const Carve k = carve(sh, fp32, z_iters, proj_buffers);
    priest_loaded *h = new (std::nothrow) priest_loaded();
    if (!h) return fail(ctx, PRIEST_ERR_NOMEM, "host allocation failed");
    h->sh = sh;
    cudaError_t e = cudaMalloc(&h->block, k.total);
    if (e != cudaSuccess) {
        delete h;
        cudaGetLastError();
        return fail(ctx, PRIEST_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->bytes = k.total;
    carve_ptrs(h, static_cast<char *>(h->block), k, fp32, z_iters, proj_buffers);
    const size_t ob = sizeof(double) * c.size();
    e = cudaMemcpyAsync(h->center, c.data(), ob, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->vel, v.data(), ob, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->semi, s.data(), sizeof(double) * s.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->counter, 0, sizeof(unsigned), st);
    // the vectors above must outlive the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_loaded(h);
        return cuda_fail(ctx, e, "upload of the problem");
    }
    *out = h;
    return PRIEST_OK;
}

// Host-pointer entry points reuse one scratch problem while it is big enough.
priest_status scratch_for(priest_ctx *ctx, const Shape &sh, const priest_problem *pr, int z_iters,
                          bool proj_buffers, priest_loaded **out)
{
    priest_loaded *h = ctx->scratch;
    const bool fp32 = ctx->cfg.precision != PRIEST_FP64_CHECK;
    if (h && carve(sh, fp32, z_iters, proj_buffers).total <= h->bytes && sh.dims == h->sh.dims) {
        // re-carve in place with the new shape
        const Carve k = carve(sh, fp32, z_iters, proj_buffers);
        char *b = static_cast<char *>(h->block);
        Shape s2 = sh;
        std::vector<double> c, v, s;
        order_obstacles(s2, pr->center, pr->vel, pr->semi, c, v, s, s2.n_static);
        // the basis, time stamps and Gram blocks stay valid (and in place)
        // while the table layout and the basis inputs are unchanged
        const Shape &o = h->sh;
        const bool same_tables = o.dims == s2.dims && o.degree == s2.degree && o.nf == s2.nf && o.n_p == s2.n_p &&
                                 o.n_obs == s2.n_obs && o.horizon == s2.horizon;
        h->shape_ready = h->shape_ready && same_tables;
        h->sh = s2;
        carve_ptrs(h, b, k, fp32, z_iters, proj_buffers);
        const size_t ob = sizeof(double) * c.size();
        cudaError_t e = cudaMemcpyAsync(h->center, c.data(), ob, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->vel, v.data(), ob, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->semi, s.data(), sizeof(double) * s.size(), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->counter, 0, sizeof(unsigned), ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "upload of the problem");
        *out = h;
        return PRIEST_OK;
    }
    if (h) {
        cudaStreamSynchronize(ctx->stream);
        free_loaded(h);
        ctx->scratch = nullptr;
    }
    priest_status st = make_loaded(ctx, sh, pr->center, pr->vel, pr->semi, z_iters, proj_buffers, ctx->stream, &h);
    if (st != PRIEST_OK) return st;
    ctx->scratch = h;
    *out = h;
    return PRIEST_OK;
}

priest_status enqueue_setup(priest_ctx *ctx, priest_loaded *h, bool plan_mode, cudaStream_t st, int *status)
{
    const SetupParams sp = setup_params(ctx, h, plan_mode, status);
    cudaError_t e = launch_setup(sp, st);
    ctx->launches++;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "setup kernel");
    h->shape_ready = true;
    return PRIEST_OK;
}

// Optional persistent record of tuned tilings: the file named by the
// environment variable PRIEST_TUNE_CACHE holds one line per shape class,
// "<key integers> S C R threads ws kind" (10 key integers for a single
// launch's shape, 11 starting with -1 for a batched launch's class).  Read
// once per context, appended to after each new tuning.
void load_tune_cache(priest_ctx *ctx)
{
    const char *path = getenv("PRIEST_TUNE_CACHE");
    if (!path || ctx->tune_cache_loaded) return;
    ctx->tune_cache_loaded = true;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        std::vector<int> v;
        char *c = line, *end = nullptr;
        for (long x = strtol(c, &end, 10); end != c; x = strtol(c, &end, 10)) {
            v.push_back(int(x));
            c = end;
        }
        const size_t nk = v.size() >= 6 ? v.size() - 6 : 0;
        if (nk != 10 && !(nk == 11 && v[0] == -1)) continue;  // lines of another format are ignored
        Tiling t;
        t.S = v[nk];
        t.C = v[nk + 1];
        t.R = v[nk + 2];
        t.threads = v[nk + 3];
        t.ws = v[nk + 4];
        t.kind = v[nk + 5];
        t.smem = 0;
        ctx->tuned[std::vector<int>(v.begin(), v.begin() + nk)] = t;
    }
    fclose(f);
}

void save_tune_entry(const std::vector<int> &key, const Tiling &t)
{
    const char *path = getenv("PRIEST_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    for (int k : key) fprintf(f, "%d ", k);
    fprintf(f, "%d %d %d %d %d %d\n", t.S, t.C, t.R, t.threads, t.ws, t.kind);
    fclose(f);
}

// Autotuner: on the first call of a problem shape, time every candidate
// tiling for a few iterations on the actual inputs (outputs are rewritten by
// the real launch that follows; multipliers are not written back) and keep
// the fastest.  Blocks while it runs.
template <typename Real>
Tiling pick_tiling(priest_ctx *ctx, const Shape &sh, int N, ProjParams<Real> p, cudaStream_t st)
{
    const Tiling model = choose_tiling<Real>(sh, N, ctx->n_sm);
    if (!ctx->cfg.autotune) return model;
    const std::vector<int> key = {int(sizeof(Real)), sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs, sh.n_static,
                                  N, p.want_lambda, sh.use_bounds};
    load_tune_cache(ctx);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
        Tiling t = it->second;
        if (t.smem == 0) t.smem = t.kind == 1 ? pts_smem_bytes(sh, t.S, t.R) : project_smem_bytes<Real>(sh, t.S, t.C);
        return t;
    }
    std::vector<Tiling> cands = tiling_candidates<Real>(sh, N, ctx->n_sm);
    cands.push_back(model);
    // marginal cost per iteration: the fastest of two launches at K = 2 and at
    // K = 22, differenced (a warm-up launch first)
    const int k_lo = 2, k_hi = 22;
    p.lam_out = nullptr;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Tiling best = model;
    float best_ms = 1e30f;
    for (const Tiling &t : cands) {
        if (t.smem > size_t(227) * 1024) continue;
        p.S = t.S;
        p.C = t.C;
        p.WS = t.ws;
        float t_k[2] = {1e30f, 1e30f};
        bool ok = true;
        for (int rep = 0; rep < 5 && ok; ++rep) {
            const int slot = rep == 0 ? -1 : (rep - 1) & 1;  // rep 0 warms up
            p.K = slot == 1 ? k_hi : k_lo;
            cudaEventRecord(e0, st);
            cudaError_t e = launch_project<Real>(p, t, st);
            cudaEventRecord(e1, st);
            ctx->launches++;
            if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                cudaGetLastError();
                ok = false;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (slot >= 0) t_k[slot] = std::min(t_k[slot], ms);
        }
        float ms = ok ? (t_k[1] - t_k[0]) / float(k_hi - k_lo) : 1e30f;
        if (!(ms > 0.f)) ms = ok ? t_k[1] / float(k_hi + 1) : 1e30f;  // timing noise: fall back to the plain ratio
        if (const char *lv = getenv("PRIEST_AUTOTUNE_LOG"))
            if (atoi(lv) >= 2)
                fprintf(stderr, "priest autotune candidate: kind=%d S=%d C=%d R=%d threads=%d ws=%d smem=%zu -> %.2f us / iteration\n",
                        t.kind, t.S, t.C, t.R, t.threads, t.ws, t.smem, 1e3f * ms);
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (getenv("PRIEST_AUTOTUNE_LOG"))
        fprintf(stderr, "priest autotune: %zu candidates, best kind=%d S=%d C=%d R=%d threads=%d ws=%d (%.2f us / iteration)\n",
                cands.size(), best.kind, best.S, best.C, best.R, best.threads, best.ws, 1e3f * best_ms);
    ctx->tuned[key] = best;
    save_tune_entry(key, best);
    return best;
}

// PRIEST_MIXED_BF16: the projection with the pair tests on the tensor core
// (project_tc.cu).  tc_params fills the launch's parameters; it and
// enqueue_project_tc return false when the shape does not fit that kernel
// (too many obstacles for tensor memory, or shared memory); the caller then
// runs the FMA kernel.
bool tc_params(priest_ctx *ctx, priest_loaded *h, int N, int mode, const double *xi, const double *z,
               const double *lam_in, double *lam_out, double *xb, double *r, double *c1, TcParams &q)
{
    Shape sh = h->sh;
    sh.N = N;
    int S = 0;
    const TcPlan tp = tc_choose(sh, N, ctx->n_sm, &S);
    if (!tp.smem || S < 1) return false;
    Tiling t;
    std::memset(&t, 0, sizeof(t));
    t.S = S;
    t.C = tp.nseg;
    t.ws = 1;
    std::memset(&q, 0, sizeof(q));
    q.p = proj_params<float>(ctx, h, t);
    q.p.N = N;
    q.p.mode = mode;
    q.p.xi_in = xi;
    q.p.mu = h->mu;
    q.p.Lc = h->L;
    q.p.z = z;
    q.p.lam_in = lam_in;
    q.p.lam_out = lam_out;
    q.p.want_lambda = lam_out != nullptr;
    q.p.xi_bar = xb;
    q.p.r_out = r;
    q.p.c1_out = c1;
    q.center = h->center;
    q.vel = h->vel;
    q.semi = h->semi;
    q.origin64 = h->tab64 + table_layout(sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs).origin;
    q.status = ctx->d_status;
    q.tp = tp;
    return true;
}

bool enqueue_project_tc(priest_ctx *ctx, priest_loaded *h, int N, int mode, const double *xi, const double *z,
                        const double *lam_in, double *lam_out, double *xb, double *r, double *c1, cudaStream_t st,
                        priest_status *out)
{
    TcParams q;
    if (!tc_params(ctx, h, N, mode, xi, z, lam_in, lam_out, xb, r, c1, q)) return false;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (ctx->profile && st == ctx->stream) {
        if (!ctx->prof_free.empty()) {
            ev = ctx->prof_free.back();
            ctx->prof_free.pop_back();
        } else {
            cudaEventCreate(&ev.first);
            cudaEventCreate(&ev.second);
        }
        cudaEventRecord(ev.first, st);
    }
    cudaError_t e = launch_project_tc(q, st);
    ctx->launches++;
    ctx->last_kind = 2;
    if (ev.first) {
        cudaEventRecord(ev.second, st);
        ctx->prof_used.push_back(ev);
    }
    *out = e == cudaSuccess ? PRIEST_OK : cuda_fail(ctx, e, "tensor-core projection kernel");
    return true;
}

// Marginal device time of one projection iteration of a launch: the fastest
// of two launches at K = 22 minus the fastest of two at K = 2, over 20 (a
// warm-up launch first); +inf when a launch fails.
template <typename Launch>
float marginal_iteration_ms(priest_ctx *ctx, cudaStream_t st, Launch launch)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float t_k[2] = {1e30f, 1e30f};
    bool ok = true;
    for (int rep = 0; rep < 5 && ok; ++rep) {
        const int slot = rep == 0 ? -1 : (rep - 1) & 1;
        cudaEventRecord(e0, st);
        const cudaError_t e = launch(slot == 1 ? 22 : 2);
        cudaEventRecord(e1, st);
        ctx->launches++;
        if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (slot >= 0) t_k[slot] = std::min(t_k[slot], ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return 1e30f;
    const float ms = (t_k[1] - t_k[0]) / 20.f;
    return ms > 0.f ? ms : t_k[1] / 23.f;
}

// PRIEST_MIXED_BF16: which kernel runs a projection shape.  With the
// autotuner on, the tensor-core kernel and the FP32 kernel are timed once per
// shape on the actual inputs and the faster one is kept (their results agree
// to FP32 summation order); with it off, or with PRIEST_MIXED_KERNEL=tensor in
// the environment, the tensor-core kernel runs.  Returns true for the
// tensor-core kernel.
bool mixed_uses_tensor(priest_ctx *ctx, priest_loaded *h, int N, int mode, const double *xi, const double *z,
                       const double *lam_in, double *xb, double *r, double *c1, const Tiling &t_fp32,
                       const ProjParams<float> &p_fp32, cudaStream_t st)
{
    static const bool forced = [] {
        const char *v = getenv("PRIEST_MIXED_KERNEL");
        return v && std::string(v) == "tensor";
    }();
    if (forced || !ctx->cfg.autotune) return true;
    const Shape &sh = h->sh;
    const std::vector<int> key = {3, sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs, sh.n_static, N, sh.use_bounds};
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) return it->second.kind == 2;
    TcParams q;
    float ms_tc = 1e30f;
    if (tc_params(ctx, h, N, mode, xi, z, lam_in, nullptr, xb, r, c1, q)) {
        q.p.want_lambda = 0;
        ms_tc = marginal_iteration_ms(ctx, st, [&](int k) {
            TcParams qk = q;
            qk.p.K = k;
            return launch_project_tc(qk, st);
        });
    }
    ProjParams<float> pf = p_fp32;
    pf.lam_out = nullptr;
    pf.want_lambda = 0;
    const float ms_fp32 = marginal_iteration_ms(ctx, st, [&](int k) {
        ProjParams<float> pk = pf;
        pk.K = k;
        return launch_project<float>(pk, t_fp32, st);
    });
    Tiling choice = t_fp32;
    if (ms_tc < ms_fp32) choice.kind = 2;
    ctx->tuned[key] = choice;
    if (getenv("PRIEST_AUTOTUNE_LOG"))
        fprintf(stderr, "priest mixed precision: n_p=%d n_obs=%d N=%d tensor %.4f ms / FP32 kernel %.4f ms per iteration -> %s\n",
                sh.n_p, sh.n_obs, N, ms_tc, ms_fp32, ms_tc < ms_fp32 ? "tensor" : "FP32");
    return ms_tc < ms_fp32;
}

template <typename Real>
priest_status enqueue_project(priest_ctx *ctx, priest_loaded *h, int N, int mode, const double *xi,
                              const double *z, const double *lam_in, double *lam_out, double *xb, double *r,
                              double *c1, cudaStream_t st)
{
    const bool mixed = sizeof(Real) == 4 && ctx->cfg.precision == PRIEST_MIXED_BF16;
    Shape sh = h->sh;
    sh.N = N;
    Tiling t = choose_tiling<Real>(sh, N, ctx->n_sm);
    if (t.smem > size_t(227) * 1024)
        return fail(ctx, PRIEST_ERR_INVALID, "problem too large for one CTA's shared memory (reduce n_p / n_obs)");
    ProjParams<Real> p = proj_params<Real>(ctx, h, t);
    p.N = N;
    p.mode = mode;
    p.xi_in = xi;
    p.mu = h->mu;
    p.Lc = h->L;
    p.z = z;
    p.lam_in = lam_in;
    p.lam_out = lam_out;
    p.want_lambda = lam_out != nullptr;
    p.xi_bar = xb;
    p.r_out = r;
    p.c1_out = c1;
    t = pick_tiling<Real>(ctx, sh, N, p, st);
    p.S = t.S;
    p.C = t.C;
    p.WS = t.ws;
    if constexpr (sizeof(Real) == 4) {
        priest_status ts;
        if (mixed && mixed_uses_tensor(ctx, h, N, mode, xi, z, lam_in, xb, r, c1, t, p, st) &&
            enqueue_project_tc(ctx, h, N, mode, xi, z, lam_in, lam_out, xb, r, c1, st, &ts))
            return ts;
    }
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (ctx->profile && st == ctx->stream) {
        if (!ctx->prof_free.empty()) {
            ev = ctx->prof_free.back();
            ctx->prof_free.pop_back();
        } else {
            cudaEventCreate(&ev.first);
            cudaEventCreate(&ev.second);
        }
        cudaEventRecord(ev.first, st);
    }
    cudaError_t e = launch_project<Real>(p, t, st);
    ctx->launches++;
    ctx->last_kind = t.kind;
    if (ev.first) {
        cudaEventRecord(ev.second, st);
        ctx->prof_used.push_back(ev);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "projection kernel");
    return PRIEST_OK;
}

priest_status enqueue_project_any(priest_ctx *ctx, priest_loaded *h, int N, int mode, const double *xi,
                                  const double *z, const double *lam_in, double *lam_out, double *xb, double *r,
                                  double *c1, cudaStream_t st)
{
    if (ctx->cfg.precision == PRIEST_FP64_CHECK)
        return enqueue_project<double>(ctx, h, N, mode, xi, z, lam_in, lam_out, xb, r, c1, st);
    return enqueue_project<float>(ctx, h, N, mode, xi, z, lam_in, lam_out, xb, r, c1, st);
}

// Alg. 1 on a loaded problem: setup, then per CEM iteration
// project(sample) -> select -> refit(+Cholesky).  z: L x N x D (device).
priest_status enqueue_plan(priest_ctx *ctx, priest_loaded *h, const double *z, double *out, cudaStream_t st,
                           int *status)
{
    const Shape &sh = h->sh;
    priest_status s = enqueue_setup(ctx, h, true, st, status);
    if (s != PRIEST_OK) return s;
    const size_t step = size_t(sh.N) * sh.D;
    for (int l = 0; l < ctx->cfg.cem_iters; ++l) {
        s = enqueue_project_any(ctx, h, sh.N, 1, nullptr, z + l * step, nullptr, nullptr, h->xb, h->r, h->c1, st);
        if (s != PRIEST_OK) return s;
        cudaError_t e = launch_select(sh.N, h->r, h->c1, sh.n_proj, sh.n_elite, h->elite, st);
        ctx->launches++;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "select kernel");
        e = launch_refit(sh.D, h->xb, h->r, h->c1, h->elite, sh.n_elite, ctx->cfg.sigma_lr, ctx->cfg.gamma,
                         ctx->cfg.chol_eps, h->mu, h->cov, h->mu_new, h->L, h->counter, status,
                         out ? out : h->out, st);
        ctx->launches++;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "refit kernel");
    }
    return PRIEST_OK;
}

priest_status check_status(priest_ctx *ctx, int *d_status, cudaStream_t st)
{
    int hs = 0;
    PRIEST_CUDA(ctx, cudaMemcpyAsync(&hs, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PRIEST_CUDA(ctx, cudaStreamSynchronize(st));
    if (hs) {
        PRIEST_CUDA(ctx, cudaMemsetAsync(d_status, 0, sizeof(int), st));
        PRIEST_CUDA(ctx, cudaStreamSynchronize(st));
        if (hs & kStatusCholesky) return fail(ctx, PRIEST_ERR_NUMERIC, "covariance Cholesky met a non-positive pivot");
        if (hs & kStatusKkt) return fail(ctx, PRIEST_ERR_NUMERIC, "KKT block met a non-positive pivot");
        if (hs & kStatusTensor) return fail(ctx, PRIEST_ERR_TIMEOUT, "tensor-core completion wait timed out");
        return fail(ctx, PRIEST_ERR_NUMERIC, "numerical failure on the device");
    }
    return PRIEST_OK;
}

uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void gaussian_stream(uint64_t seed, int64_t count, double *out)
{
    const double two_pi = 6.283185307179586476925286766559;
    uint64_t s = seed;
    int64_t i = 0;
    while (i < count) {
        const double u1 = double(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
        const double u2 = double(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
        const double rad = std::sqrt(-2.0 * std::log(1.0 - u1));
        const double th = two_pi * u2;
        out[i++] = rad * std::cos(th);
        if (i < count) out[i++] = rad * std::sin(th);
    }
}

// ---------------------------------------------------------------------------
// Plain per-problem FP32 path (plain.cu): the comparison point of the fused
// kernel, one launch per step with HBM intermediates.
// ---------------------------------------------------------------------------
priest_status plain_workspace(priest_ctx *ctx, const Shape &sh, int N, float **out)
{
    if (ctx->cfg.precision == PRIEST_FP64_CHECK) return fail(ctx, PRIEST_ERR_INVALID, "the plain path runs in FP32 only");
    const size_t need = plain_work_floats(sh.dims, sh.nv, sh.nf, sh.n_p, std::max(N, 1));
    if (need > ctx->plain_cap) {
        PRIEST_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->plain_work) cudaFree(ctx->plain_work);
        ctx->plain_work = nullptr;
        ctx->plain_cap = 0;
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&ctx->plain_work), need * sizeof(float));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, PRIEST_ERR_NOMEM, "plain-path workspace");
        }
        ctx->plain_cap = need;
    }
    *out = ctx->plain_work;
    return PRIEST_OK;
}

PlainParams plain_params(priest_ctx *ctx, const priest_loaded *h, int N, float *work)
{
    const Shape &sh = h->sh;
    PlainParams p;
    std::memset(&p, 0, sizeof(p));
    p.dims = sh.dims;
    p.nv = sh.nv;
    p.nf = sh.nf;
    p.n_p = sh.n_p;
    p.np4 = (sh.n_p + 3) / 4 * 4;
    p.n_obs = sh.n_obs;
    p.use_bounds = sh.use_bounds;
    p.N = N;
    p.K = ctx->cfg.proj_iters;
    p.rho = float(sh.rho);
    p.vmax = float(sh.vmax);
    p.amax = float(sh.amax);
    for (int ax = 0; ax < 3; ++ax) {
        p.smin[ax] = float(sh.smin[ax]);
        p.smax[ax] = float(sh.smax[ax]);
    }
    p.tab = h->tab32;
    p.lay = table_layout(sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs);
    p.cB = h->cB;
    p.cost = make_cost<float>(sh);
    plain_carve(p, work);
    return p;
}

// Alg. 1 on a loaded problem through the plain projection.
priest_status enqueue_plan_plain(priest_ctx *ctx, priest_loaded *h, const double *z, double *out, cudaStream_t st,
                                 int *status)
{
    const Shape &sh = h->sh;
    float *work = nullptr;
    priest_status s = plain_workspace(ctx, sh, sh.N, &work);
    if (s != PRIEST_OK) return s;
    s = enqueue_setup(ctx, h, true, st, status);
    if (s != PRIEST_OK) return s;
    const size_t step = size_t(sh.N) * sh.D;
    PlainParams p = plain_params(ctx, h, sh.N, work);
    p.mode = 1;
    p.mu = h->mu;
    p.Lc = h->L;
    p.xi_bar = h->xb;
    p.r_out = h->r;
    p.c1_out = h->c1;
    for (int l = 0; l < ctx->cfg.cem_iters; ++l) {
        p.z = z + l * step;
        int64_t n = 0;
        cudaError_t e = launch_plain_project(p, st, &n);
        ctx->launches += n;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "plain projection");
        e = launch_select(sh.N, h->r, h->c1, sh.n_proj, sh.n_elite, h->elite, st);
        ctx->launches++;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "select kernel");
        e = launch_refit(sh.D, h->xb, h->r, h->c1, h->elite, sh.n_elite, ctx->cfg.sigma_lr, ctx->cfg.gamma,
                         ctx->cfg.chol_eps, h->mu, h->cov, h->mu_new, h->L, h->counter, status,
                         out ? out : h->out, st);
        ctx->launches++;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "refit kernel");
    }
    return PRIEST_OK;
}

priest_status plan_host(priest_ctx *ctx, const priest_problem *pr, const double *mu0, const double *cov0,
                        const double *z_host, priest_result *out, bool plain = false)
{
    if (!ctx || !out) return fail(ctx, PRIEST_ERR_INVALID, "NULL argument");
    Shape sh;
    priest_status s = resolve(ctx, pr, -1, sh);
    if (s != PRIEST_OK) return s;
    const int L = ctx->cfg.cem_iters;
    priest_loaded *h = nullptr;
    s = scratch_for(ctx, sh, pr, L, false, &h);
    if (s != PRIEST_OK) return s;
    const size_t nz = size_t(L) * sh.N * sh.D;
    std::vector<double> zbuf;
    if (!z_host) {
        zbuf.resize(nz);
        gaussian_stream(pr->seed, int64_t(nz), zbuf.data());
        z_host = zbuf.data();
    }
    PRIEST_CUDA(ctx, cudaMemcpyAsync(h->z, z_host, nz * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    h->default_mu = mu0 == nullptr;
    h->default_cov = cov0 == nullptr;
    if (mu0) PRIEST_CUDA(ctx, cudaMemcpyAsync(h->mu, mu0, sh.D * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (cov0)
        PRIEST_CUDA(ctx, cudaMemcpyAsync(h->cov, cov0, size_t(sh.D) * sh.D * sizeof(double), cudaMemcpyHostToDevice,
                                         ctx->stream));
    s = plain ? enqueue_plan_plain(ctx, h, h->z, h->out, ctx->stream, ctx->d_status)
              : enqueue_plan(ctx, h, h->z, h->out, ctx->stream, ctx->d_status);
    if (s != PRIEST_OK) return s;
    std::vector<double> ho(sh.D + 4), hm(sh.D);
    PRIEST_CUDA(ctx, cudaMemcpyAsync(ho.data(), h->out, ho.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(hm.data(), h->mu, hm.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    s = check_status(ctx, ctx->d_status, ctx->stream);
    if (s != PRIEST_OK) return s;
    fill_result(sh, ho.data(), hm.data(), out);
    return PRIEST_OK;
}

// ---------------------------------------------------------------------------
// Batched solves.
// ---------------------------------------------------------------------------
void free_batch(BatchPlan *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->dev) cudaFree(b->dev);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    delete b;
}

// A pair of timing events from the context's pool (created on demand).
std::pair<cudaEvent_t, cudaEvent_t> prof_pair(priest_ctx *ctx)
{
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (!ctx->prof_free.empty()) {
        ev = ctx->prof_free.back();
        ctx->prof_free.pop_back();
    } else {
        cudaEventCreate(&ev.first);
        cudaEventCreate(&ev.second);
    }
    return ev;
}

// Autotuner of the batched launch: per class of problem shape (dims,
// degree, mask, n_p, obstacles rounded up to a multiple of 32, moving ones
// present, bounds), every candidate tiling is timed on a representative
// problem of the batch.  The trial launch is the batched kernel itself over
// that problem's items, repeated until they fill the GPU twice, so the
// measure is throughput (per-iteration marginal time: K = 22 minus K = 2,
// the fastest of two launches each).
std::vector<int> batch_class(const Shape &sh, int dbl)
{
    return {-1, dbl, sh.dims, sh.nv, sh.nf, sh.bc_mask, sh.n_p, (sh.n_obs + 31) / 32, sh.n_obs > sh.n_static,
            sh.use_bounds, std::min(sh.N, 16)};
}

template <typename Real>
Tiling batch_tiling_for(priest_ctx *ctx, const Shape &sh)
{
    auto it = ctx->tuned.find(batch_class(sh, sizeof(Real) == 8));
    if (it == ctx->tuned.end()) return batch_tiling<Real>(sh);
    Tiling t = it->second;
    t.S = std::max(1, std::min(t.S, sh.N));
    t.smem = t.kind == 1 ? pts_smem_bytes(sh, t.S, t.R) : project_smem_bytes<Real>(sh, t.S, t.C);
    if (t.smem > size_t(227) * 1024) return batch_tiling<Real>(sh);
    // an entry from a cache file written for another CTA size
    if (t.kind == 1 && (t.R != 2 || pts_threads(sh, t.S, 2) > pts_batch_threads(sh))) return batch_tiling<Real>(sh);
    return t;
}

// shapes[i]: problem i's shape with the sample count of the launch; base[i]:
// its projection parameters (inputs, outputs, mode) -- the trials write its
// outputs, which the real launch rewrites, and never its multipliers.
// setups != null: the tables are formed first (one setup launch, waited for),
// only when some class needs tuning; *formed tells whether that launch ran.
template <typename Real>
priest_status tune_batch(priest_ctx *ctx, int n, const std::vector<Shape> &shapes,
                         const std::vector<ProjParams<Real>> &base, const std::vector<SetupParams> *setups,
                         bool *formed = nullptr)
{
    if (formed) *formed = false;
    std::vector<int> reps;  // one representative problem per untuned class
    {
        std::map<std::vector<int>, int> seen;
        for (int i = 0; i < n; ++i) {
            if (shapes[i].N < 1) continue;
            const std::vector<int> key = batch_class(shapes[i], sizeof(Real) == 8);
            if (ctx->tuned.count(key) || seen.count(key)) continue;
            seen[key] = i;
            reps.push_back(i);
        }
    }
    load_tune_cache(ctx);
    for (size_t k = 0; k < reps.size();)  // classes a cache file already holds
        if (ctx->tuned.count(batch_class(shapes[reps[k]], sizeof(Real) == 8)))
            reps.erase(reps.begin() + k);
        else
            ++k;
    if (reps.empty()) return PRIEST_OK;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (setups) {
        void *dsetup = nullptr;
        PRIEST_CUDA(ctx, cudaMalloc(&dsetup, sizeof(SetupParams) * n));
        size_t smem_setup = 0;
        for (int i = 0; i < n; ++i) smem_setup = std::max(smem_setup, setup_smem_bytes(shapes[i]));
        e = cudaMemcpyAsync(dsetup, setups->data(), sizeof(SetupParams) * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_setup_batch(static_cast<SetupParams *>(dsetup), n, smem_setup, st);
        ctx->launches++;
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(dsetup);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "setup before tuning");
        if (formed) *formed = true;
    }
    const int fill = 2 * ctx->n_sm;
    void *dbuf = nullptr;
    size_t dcap = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int i : reps) {
        const Shape &sh = shapes[i];
        Tiling best = batch_tiling<Real>(sh);
        float best_us = 1e30f;
        for (const Tiling &t : batch_candidates<Real>(sh)) {
            ProjParams<Real> p = base[i];
            p.S = t.S;
            p.C = t.C;
            p.WS = t.ws;
            p.N = sh.N;
            p.lam_out = nullptr;
            p.want_lambda = 0;
            std::vector<int2> it;
            while (int(it.size()) < fill)
                for (int s = 0; s < sh.N; s += t.S) it.push_back(make_int2(0, s));
            const size_t need = 2 * sizeof(ProjParams<Real>) + sizeof(int2) * it.size() + 256;
            if (need > dcap) {
                if (dbuf) cudaFree(dbuf);
                dbuf = nullptr;
                dcap = 0;
                if (cudaMalloc(&dbuf, need) != cudaSuccess) {
                    cudaGetLastError();
                    break;
                }
                dcap = need;
            }
            ProjParams<Real> pk[2] = {p, p};
            pk[0].K = 2;
            pk[1].K = 22;
            char *d = static_cast<char *>(dbuf);
            int *cnt = reinterpret_cast<int *>(d);
            ProjParams<Real> *dp = reinterpret_cast<ProjParams<Real> *>(d + 256);
            int2 *di = reinterpret_cast<int2 *>(d + 256 + 2 * sizeof(ProjParams<Real>));
            e = cudaMemcpyAsync(dp, pk, sizeof(pk), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(di, it.data(), sizeof(int2) * it.size(), cudaMemcpyHostToDevice, st);
            float ms[2] = {1e30f, 1e30f};
            for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
                const int k = rep == 0 ? 0 : (rep - 1) & 1;  // rep 0 warms up; then the fastest of two each
                e = cudaMemsetAsync(cnt, 0, sizeof(int), st);
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                if (e == cudaSuccess)
                    e = launch_project_batch<Real>(dp + k, di, int(it.size()), cnt, sh.dims, t.R, 0, sh.nf, sh.nv, 0,
                                                   t.smem, 0, st, t.kind);
                ctx->launches++;
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float t_ms = 0.f;
                if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&t_ms, e0, e1) == cudaSuccess)
                    ms[k] = std::min(ms[k], t_ms);
            }
            if (e != cudaSuccess) {
                cudaGetLastError();
                e = cudaSuccess;
                continue;
            }
            // marginal time per iteration per sample processed
            float us = 1e3f * (ms[1] - ms[0]) / 20.f / float(it.size() * t.S);
            if (!(us > 0.f)) us = 1e3f * ms[1] / 23.f / float(it.size() * t.S);  // timing noise
            if (const char *lv = getenv("PRIEST_AUTOTUNE_LOG"))
                if (atoi(lv) >= 2)
                    fprintf(stderr, "priest batch autotune candidate: n_p=%d n_obs=%d kind=%d S=%d C=%d ws=%d -> %.5f us\n",
                            sh.n_p, sh.n_obs, t.kind, t.S, t.C, t.ws, us);
            if (us < best_us) {
                best_us = us;
                best = t;
            }
        }
        ctx->tuned[batch_class(sh, sizeof(Real) == 8)] = best;
        save_tune_entry(batch_class(sh, sizeof(Real) == 8), best);
        if (getenv("PRIEST_AUTOTUNE_LOG"))
            fprintf(stderr, "priest batch autotune: n_p=%d n_obs=%d -> kind=%d S=%d C=%d ws=%d (%.4f us / sample-iteration)\n",
                    sh.n_p, sh.n_obs, best.kind, best.S, best.C, best.ws, best_us);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (dbuf) cudaFree(dbuf);
    return PRIEST_OK;
}

// Per-problem tilings of one persistent launch and the kernel they share:
// the point-owner kernel when every problem's tiling uses it, the chunked one
// otherwise (one kernel kind per launch).
template <typename Real>
priest_status batch_tiles(priest_ctx *ctx, const std::vector<Shape> &shapes, std::vector<Tiling> &tiles, int &kind,
                          int &R)
{
    const int n = int(shapes.size());
    tiles.resize(n);
    bool all_pts = true;
    for (int i = 0; i < n; ++i) {
        tiles[i] = batch_tiling_for<Real>(ctx, shapes[i]);
        all_pts = all_pts && tiles[i].kind == 1;
    }
    for (int i = 0; i < n && !all_pts; ++i)
        if (tiles[i].kind == 1) {
            for (const Tiling &c : batch_candidates<Real>(shapes[i]))
                if (c.kind == 0) {
                    tiles[i] = c;
                    break;
                }
        }
    kind = all_pts ? 1 : 0;
    R = all_pts ? tiles[0].R : 4;
    for (int i = 0; i < n; ++i)
        if (tiles[i].smem == 0 || tiles[i].kind != kind)
            return fail(ctx, PRIEST_ERR_INVALID, "problem too large for one CTA's shared memory");
    return PRIEST_OK;
}

// Host-side descriptors of one batched solve (Alg. 1 for every problem).
template <typename Real>
struct BatchDesc {
    std::vector<ProjParams<Real>> params;  // L x n
    std::vector<SetupParams> setups, setups_ready;
    std::vector<CemArgs> cem;
    std::vector<int2> items;               // (problem, first sample), most expensive first
    int kind = 0, R = 4, D_max = 0;
    size_t smem_proj = 0, smem_setup = 0, smem_select = 0, smem_refit = 0;
};

template <typename Real>
priest_status batch_describe(priest_ctx *ctx, int n, priest_loaded *const *probs, const double *const *z,
                             double *const *out, BatchDesc<Real> &d, bool with_items = true)
{
    const int L = ctx->cfg.cem_iters;
    const Shape &s0 = probs[0]->sh;
    std::vector<Shape> shapes(n);
    for (int i = 0; i < n; ++i) {
        shapes[i] = probs[i]->sh;
        if (shapes[i].dims != s0.dims || shapes[i].nv != s0.nv || shapes[i].bc_mask != s0.bc_mask)
            return fail(ctx, PRIEST_ERR_INVALID, "batched problems must share dims, degree and bc_final_mask");
    }
    std::vector<Tiling> tiles;
    priest_status s = batch_tiles<Real>(ctx, shapes, tiles, d.kind, d.R);
    if (s != PRIEST_OK) return s;
    d.params.assign(size_t(L) * n, ProjParams<Real>{});
    d.setups.resize(n);
    d.setups_ready.resize(n);
    d.cem.resize(n);
    std::vector<std::pair<double, int2>> items;
    for (int i = 0; i < n; ++i) {
        priest_loaded *h = probs[i];
        const Shape &sh = h->sh;
        const Tiling t = tiles[i];
        d.smem_proj = std::max(d.smem_proj, t.smem);
        ProjParams<Real> p = proj_params<Real>(ctx, h, t);
        p.N = sh.N;
        p.mode = 1;
        p.mu = h->mu;
        p.Lc = h->L;
        p.want_lambda = 0;
        p.xi_bar = h->xb;
        p.r_out = h->r;
        p.c1_out = h->c1;
        for (int l = 0; l < L; ++l) {
            p.z = z[i] + size_t(l) * sh.N * sh.D;
            d.params[size_t(l) * n + i] = p;
        }
        const double cost = double(sh.n_p) * (double(sh.n_obs) + 12.0);
        if (with_items)
            for (int s0i = 0; s0i < sh.N; s0i += t.S)
                items.push_back({cost * std::min(t.S, sh.N - s0i), make_int2(i, s0i)});
        SetupParams sp = setup_params(ctx, h, true, ctx->d_status);
        sp.default_mu = 1;
        sp.default_cov = 1;
        sp.shape_ready = 0;
        d.setups[i] = sp;
        sp.shape_ready = 1;
        d.setups_ready[i] = sp;
        d.smem_setup = std::max(d.smem_setup, setup_smem_bytes(sh));
        d.cem[i] = cem_args(ctx, h, ctx->d_status, out[i]);
        d.smem_select = std::max(d.smem_select, select_smem_bytes(sh.N));
        d.smem_refit = std::max(d.smem_refit, refit_smem_bytes(sh.D, sh.n_elite));
        d.D_max = std::max(d.D_max, sh.D);
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int2> &x, const std::pair<double, int2> &y) { return x.first > y.first; });
    d.items.resize(items.size());
    for (size_t k = 0; k < items.size(); ++k) d.items[k] = items[k].second;
    return PRIEST_OK;
}

// Offsets of the descriptor block of a batched solve.
struct BatchOffsets {
    size_t params, setup, setup_r, cem, items, cnt, total;
};

template <typename Real>
BatchOffsets batch_offsets(const BatchDesc<Real> &d, int n, int L)
{
    BatchOffsets o;
    size_t at = 0;
    auto take = [&](size_t bytes) {
        const size_t here = at;
        at = round_up(at + bytes);
        return here;
    };
    o.params = take(sizeof(ProjParams<Real>) * d.params.size());
    o.setup = take(sizeof(SetupParams) * n);
    o.setup_r = take(sizeof(SetupParams) * n);
    o.cem = take(sizeof(CemArgs) * n);
    o.items = take(sizeof(int2) * d.items.size());
    o.cnt = take(sizeof(int) * L);
    o.total = at;
    return o;
}

template <typename Real>
priest_status batch_upload(priest_ctx *ctx, BatchPlan *b, const BatchDesc<Real> &d, bool with_items = true)
{
    cudaStream_t st = ctx->stream;
    PRIEST_CUDA(ctx, cudaMemcpyAsync(b->params_dev, d.params.data(), sizeof(ProjParams<Real>) * d.params.size(),
                                     cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(b->setup_dev, d.setups.data(), sizeof(SetupParams) * b->n,
                                     cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(b->setup_dev_ready, d.setups_ready.data(), sizeof(SetupParams) * b->n,
                                     cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(b->cem_dev, d.cem.data(), sizeof(CemArgs) * b->n, cudaMemcpyHostToDevice, st));
    if (with_items)
        PRIEST_CUDA(ctx, cudaMemcpyAsync(b->items_dev, d.items.data(), sizeof(int2) * d.items.size(),
                                         cudaMemcpyHostToDevice, st));
    // the host vectors are released when the caller returns
    PRIEST_CUDA(ctx, cudaStreamSynchronize(st));
    return PRIEST_OK;
}

template <typename Real>
priest_status batch_build(priest_ctx *ctx, int n, priest_loaded *const *probs, const double *const *z,
                          double *const *out, BatchPlan *b)
{
    const int L = ctx->cfg.cem_iters;
    const Shape &s0 = probs[0]->sh;
    b->n = n;
    b->L = L;
    b->dims = s0.dims;
    b->nf = s0.nf;
    b->nv = s0.nv;
    b->dbl = sizeof(Real) == 8;
    if (ctx->cfg.autotune) {
        std::vector<Shape> shapes(n);
        std::vector<SetupParams> sps(n);
        std::vector<ProjParams<Real>> base(n);
        Tiling t0;
        std::memset(&t0, 0, sizeof(t0));
        t0.S = t0.C = t0.ws = 1;
        for (int i = 0; i < n; ++i) {
            priest_loaded *h = probs[i];
            shapes[i] = h->sh;
            sps[i] = setup_params(ctx, h, true, ctx->d_status);
            sps[i].default_mu = 1;
            sps[i].default_cov = 1;
            ProjParams<Real> p = proj_params<Real>(ctx, h, t0);
            p.N = h->sh.N;
            p.mode = 1;
            p.mu = h->mu;
            p.Lc = h->L;
            p.z = z[i];
            p.xi_bar = h->xb;
            p.r_out = h->r;
            p.c1_out = h->c1;
            base[i] = p;
        }
        bool formed = false;
        const priest_status ts = tune_batch<Real>(ctx, n, shapes, base, &sps, &formed);
        if (ts != PRIEST_OK) return ts;
        // the tables exist only if the tuner ran the setup launch
        if (formed)
            for (int i = 0; i < n; ++i) probs[i]->shape_ready = true;
    }
    BatchDesc<Real> d;
    priest_status s = batch_describe<Real>(ctx, n, probs, z, out, d);
    if (s != PRIEST_OK) return s;
    b->kind = d.kind;
    b->R = d.R;
    b->D_max = d.D_max;
    b->smem_proj = d.smem_proj;
    b->smem_setup = d.smem_setup;
    b->smem_select = d.smem_select;
    b->smem_refit = d.smem_refit;
    b->n_items = int(d.items.size());
    const BatchOffsets o = batch_offsets(d, n, L);
    cudaError_t e = cudaMalloc(&b->dev, o.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PRIEST_ERR_NOMEM, "batch descriptors");
    }
    char *dv = static_cast<char *>(b->dev);
    b->params_dev = dv + o.params;
    b->setup_dev = reinterpret_cast<SetupParams *>(dv + o.setup);
    b->setup_dev_ready = reinterpret_cast<SetupParams *>(dv + o.setup_r);
    b->cem_dev = reinterpret_cast<CemArgs *>(dv + o.cem);
    b->items_dev = reinterpret_cast<int2 *>(dv + o.items);
    b->counters_dev = reinterpret_cast<int *>(dv + o.cnt);
    b->items_host = d.items;
    return batch_upload<Real>(ctx, b, d);
}

// New problem data (obstacles, boundary values, bounds) behind the same
// handles, every problem keeping its layout (the host-buffer path checks its
// layout key first): the per-problem descriptors are formed again and
// uploaded in place, the work items stay, and the recorded graph stays
// valid.  Returns false when the launch layout changed (kernel, shared
// memory), which needs a new plan.
template <typename Real>
bool batch_refresh(priest_ctx *ctx, int n, priest_loaded *const *probs, const double *const *z,
                   double *const *out, BatchPlan *b, priest_status *st)
{
    // the caller keeps every problem's layout (sample count, shape class and
    // so tiling), so the work items are the recorded ones: only the
    // per-problem parameters are formed again
    BatchDesc<Real> d;
    *st = batch_describe<Real>(ctx, n, probs, z, out, d, false);
    if (*st != PRIEST_OK) return false;
    if (d.kind != b->kind || d.R != b->R || d.smem_proj != b->smem_proj || d.smem_setup > b->smem_setup ||
        d.smem_select > b->smem_select || d.smem_refit > b->smem_refit || d.D_max != b->D_max)
        return false;
    *st = batch_upload<Real>(ctx, b, d, false);
    return *st == PRIEST_OK;
}

// The launch sequence of one batched solve.  When `capture` is set the
// projection launches are bracketed by external event-record nodes (the
// plan's own events), so that a replay can be timed per projection launch;
// a direct run while profiling brackets them with the context's events.
template <typename Real>
priest_status batch_enqueue(priest_ctx *ctx, BatchPlan *b, bool shape_ready, cudaStream_t st, bool capture)
{
    cudaError_t e = cudaMemsetAsync(b->counters_dev, 0, sizeof(int) * b->L, st);
    if (e == cudaSuccess)
        e = launch_setup_batch(shape_ready ? b->setup_dev_ready : b->setup_dev, b->n, b->smem_setup, st);
    ctx->launches++;
    const ProjParams<Real> *params = static_cast<const ProjParams<Real> *>(b->params_dev);
    const bool mark = capture && int(b->ev.size()) == 2 * b->L;
    for (int l = 0; l < b->L && e == cudaSuccess; ++l) {
        std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
        if (l == 1 && b->zwait) e = cudaStreamWaitEvent(st, b->zwait, capture ? cudaEventWaitExternal : 0);
        if (e != cudaSuccess) break;
        if (mark) {
            e = cudaEventRecordWithFlags(b->ev[2 * l], st, cudaEventRecordExternal);
        } else if (!capture && ctx->profile && st == ctx->stream) {
            ev = prof_pair(ctx);
            cudaEventRecord(ev.first, st);
        }
        if (e == cudaSuccess)
            e = launch_project_batch<Real>(params + size_t(l) * b->n, b->items_dev, b->n_items, b->counters_dev + l,
                                           b->dims, b->R, 0, b->nf, b->nv, 0, b->smem_proj, 0, st, b->kind);
        if (mark && e == cudaSuccess) e = cudaEventRecordWithFlags(b->ev[2 * l + 1], st, cudaEventRecordExternal);
        if (ev.first) {
            cudaEventRecord(ev.second, st);
            ctx->prof_used.push_back(ev);
        }
        if (e == cudaSuccess) e = launch_select_batch(b->cem_dev, b->n, b->smem_select, st);
        if (e == cudaSuccess) e = launch_refit_batch(b->cem_dev, b->n, b->D_max, b->smem_refit, st);
        ctx->launches += 3;
    }
    ctx->last_kind = b->kind;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched launch");
    return PRIEST_OK;
}

// Replay of a recorded batched solve.  While profiling, the event-record
// nodes around the projection launches are pointed at fresh events of the
// context's pool (read back by priest_profile_read); otherwise at the plan's
// own events.
priest_status batch_replay(priest_ctx *ctx, BatchPlan *b)
{
    const bool timed = ctx->profile && int(b->ev_nodes.size()) == 2 * b->L;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
    if (timed || b->ev_swapped) {
        for (int l = 0; l < b->L; ++l) {
            std::pair<cudaEvent_t, cudaEvent_t> ev{b->ev[2 * l], b->ev[2 * l + 1]};
            if (timed) ev = prof_pair(ctx);
            if (cudaGraphExecEventRecordNodeSetEvent(b->exec, b->ev_nodes[2 * l], ev.first) != cudaSuccess ||
                cudaGraphExecEventRecordNodeSetEvent(b->exec, b->ev_nodes[2 * l + 1], ev.second) != cudaSuccess)
                return cuda_fail(ctx, cudaGetLastError(), "graph event node update");
            if (timed) evs.push_back(ev);
        }
        b->ev_swapped = timed;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, ctx->stream);
    ctx->launches += 1 + 3 * b->L;
    ctx->last_kind = b->kind;
    ctx->prof_used.insert(ctx->prof_used.end(), evs.begin(), evs.end());
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    return PRIEST_OK;
}

std::vector<uintptr_t> batch_key(int n, priest_loaded *const *probs, const double *const *z, double *const *out)
{
    std::vector<uintptr_t> key;
    key.reserve(3 * size_t(n) + 1);
    key.push_back(uintptr_t(n));
    for (int i = 0; i < n; ++i) {
        key.push_back(reinterpret_cast<uintptr_t>(probs[i]));
        key.push_back(reinterpret_cast<uintptr_t>(z[i]));
        key.push_back(reinterpret_cast<uintptr_t>(out[i]));
    }
    return key;
}

// refresh: the problems behind the handles may have new data (see
// batch_refresh); otherwise a recorded plan is replayed as it is.
template <typename Real>
priest_status plan_batch(priest_ctx *ctx, int n, priest_loaded *const *probs, const double *const *z,
                         double *const *out, bool refresh = false, cudaEvent_t zwait = nullptr)
{
    const std::vector<uintptr_t> key = batch_key(n, probs, z, out);
    auto it = ctx->batches.find(key);
    if (it != ctx->batches.end() && it->second->exec) {
        priest_status s = PRIEST_OK;
        if (!refresh || batch_refresh<Real>(ctx, n, probs, z, out, it->second, &s)) return batch_replay(ctx, it->second);
        if (s != PRIEST_OK) return s;
    }
    if (it != ctx->batches.end()) {
        cudaStreamSynchronize(ctx->stream);
        free_batch(it->second);
        ctx->batches.erase(it);
    }
    BatchPlan *b = new BatchPlan();
    b->zwait = zwait;
    priest_status s = batch_build<Real>(ctx, n, probs, z, out, b);
    if (s != PRIEST_OK) {
        free_batch(b);
        return s;
    }
    bool ready = true;
    for (int i = 0; i < n; ++i) ready = ready && probs[i]->shape_ready;
    s = batch_enqueue<Real>(ctx, b, ready, ctx->stream, false);  // direct run (also sets kernel attributes)
    if (s != PRIEST_OK) {
        free_batch(b);
        return s;
    }
    for (int i = 0; i < n; ++i) probs[i]->shape_ready = true;
    // record the sequence for replay, with timing events around the projections
    b->ev.assign(2 * size_t(b->L), nullptr);
    for (cudaEvent_t &ev : b->ev)
        if (cudaEventCreate(&ev) != cudaSuccess) {
            cudaGetLastError();
            for (cudaEvent_t &x : b->ev)
                if (x) cudaEventDestroy(x);
            b->ev.clear();
            break;
        }
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess) {
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int64_t before = ctx->launches.load();
            const priest_status ok = batch_enqueue<Real>(ctx, b, true, cap, true);
            ctx->launches = before;
            cudaGraph_t g = nullptr;
            if (cudaStreamEndCapture(cap, &g) == cudaSuccess && ok == PRIEST_OK && g) {
                b->graph = g;
                if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) b->exec = nullptr;
            } else if (g) {
                cudaGraphDestroy(g);
            }
        }
        cudaGetLastError();
        cudaStreamDestroy(cap);
    }
    // the record nodes of the timing events, in the order of b->ev
    if (b->graph && !b->ev.empty()) {
        size_t count = 0;
        if (cudaGraphGetNodes(b->graph, nullptr, &count) == cudaSuccess && count > 0) {
            std::vector<cudaGraphNode_t> nodes(count);
            std::vector<cudaGraphNode_t> found(b->ev.size(), nullptr);
            if (cudaGraphGetNodes(b->graph, nodes.data(), &count) == cudaSuccess) {
                for (cudaGraphNode_t nd : nodes) {
                    cudaGraphNodeType ty;
                    cudaEvent_t ev = nullptr;
                    if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord) continue;
                    if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
                    for (size_t k = 0; k < b->ev.size(); ++k)
                        if (b->ev[k] == ev) found[k] = nd;
                }
                bool all = true;
                for (cudaGraphNode_t nd : found) all = all && nd != nullptr;
                if (all) b->ev_nodes = found;
            }
        }
        cudaGetLastError();
    }
    ctx->batches[key] = b;
    return PRIEST_OK;
}

// ---------------------------------------------------------------------------
// Batched projection of caller-given samples: one setup launch for all
// problems, then one persistent projection launch over every problem's
// (problem, first sample) items, with the tilings of the batched solves.
// ---------------------------------------------------------------------------

// Grows the context's descriptor block (device) and its pinned staging copy
// to at least `bytes`; waits for the previous user of the staging first.
priest_status descriptor_block(priest_ctx *ctx, size_t bytes)
{
    if (ctx->pb_done) PRIEST_CUDA(ctx, cudaEventSynchronize(ctx->pb_done));
    if (bytes <= ctx->pb_cap) return PRIEST_OK;
    PRIEST_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->pb_dev) cudaFree(ctx->pb_dev);
    if (ctx->pb_host) cudaFreeHost(ctx->pb_host);
    ctx->pb_dev = ctx->pb_host = nullptr;
    ctx->pb_cap = 0;
    const size_t cap = round_up(bytes + bytes / 2);
    if (cudaMalloc(&ctx->pb_dev, cap) != cudaSuccess || cudaMallocHost(&ctx->pb_host, cap) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->pb_dev) cudaFree(ctx->pb_dev);
        ctx->pb_dev = nullptr;
        return fail(ctx, PRIEST_ERR_NOMEM, "batched projection descriptors");
    }
    if (!ctx->pb_done) PRIEST_CUDA(ctx, cudaEventCreateWithFlags(&ctx->pb_done, cudaEventDisableTiming));
    ctx->pb_cap = cap;
    return PRIEST_OK;
}

template <typename Real>
priest_status project_batch(priest_ctx *ctx, int n, priest_loaded *const *probs, const int *rows,
                            const double *const *xi, double *const *lam, double *const *xb, double *const *r,
                            double *const *c1)
{
    cudaStream_t st = ctx->stream;
    std::vector<Shape> shapes(n);
    std::vector<SetupParams> sps(n);
    std::vector<ProjParams<Real>> base(n);
    Tiling t0;
    std::memset(&t0, 0, sizeof(t0));
    t0.S = t0.C = t0.ws = 1;
    size_t smem_setup = 0, n_rows = 0;
    int want_lambda = 0;
    for (int i = 0; i < n; ++i) {
        priest_loaded *h = probs[i];
        shapes[i] = h->sh;
        shapes[i].N = rows[i];
        sps[i] = setup_params(ctx, h, false, ctx->d_status);
        smem_setup = std::max(smem_setup, setup_smem_bytes(h->sh));
        ProjParams<Real> p = proj_params<Real>(ctx, h, t0);
        p.N = rows[i];
        p.mode = 0;
        p.xi_in = xi[i];
        p.lam_in = lam ? lam[i] : nullptr;
        p.lam_out = p.lam_in ? lam[i] : nullptr;
        p.want_lambda = p.lam_out != nullptr;
        want_lambda |= p.want_lambda;
        p.xi_bar = xb[i];
        p.r_out = r[i];
        p.c1_out = c1[i];
        base[i] = p;
        n_rows += size_t(rows[i]);
    }
    // descriptor block: counter | setups | params | items (at most one per row)
    const size_t o_set = 256, o_par = round_up(o_set + sizeof(SetupParams) * n),
                 o_it = round_up(o_par + sizeof(ProjParams<Real>) * n), total = o_it + sizeof(int2) * (n_rows + 1);
    priest_status s = descriptor_block(ctx, total);
    if (s != PRIEST_OK) return s;
    char *hb = static_cast<char *>(ctx->pb_host), *db = static_cast<char *>(ctx->pb_dev);
    std::memcpy(hb + o_set, sps.data(), sizeof(SetupParams) * n);
    PRIEST_CUDA(ctx, cudaMemcpyAsync(db + o_set, hb + o_set, sizeof(SetupParams) * n, cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, launch_setup_batch(reinterpret_cast<SetupParams *>(db + o_set), n, smem_setup, st));
    ctx->launches++;
    for (int i = 0; i < n; ++i) probs[i]->shape_ready = true;
    if (ctx->cfg.autotune) {
        s = tune_batch<Real>(ctx, n, shapes, base, nullptr);
        if (s != PRIEST_OK) return s;
    }
    std::vector<Tiling> tiles;
    int kind = 0, R = 4;
    s = batch_tiles<Real>(ctx, shapes, tiles, kind, R);
    if (s != PRIEST_OK) return s;
    size_t smem = 0;
    std::vector<std::pair<double, int2>> items;
    ProjParams<Real> *hp = reinterpret_cast<ProjParams<Real> *>(hb + o_par);
    for (int i = 0; i < n; ++i) {
        ProjParams<Real> p = base[i];
        p.S = tiles[i].S;
        p.C = tiles[i].C;
        p.WS = tiles[i].ws;
        hp[i] = p;
        smem = std::max(smem, tiles[i].smem);
        const double cost = double(shapes[i].n_p) * (double(shapes[i].n_obs) + 12.0);
        for (int s0 = 0; s0 < rows[i]; s0 += tiles[i].S)
            items.push_back({cost * std::min(tiles[i].S, rows[i] - s0), make_int2(i, s0)});
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int2> &x, const std::pair<double, int2> &y) { return x.first > y.first; });
    int2 *hi = reinterpret_cast<int2 *>(hb + o_it);
    for (size_t k = 0; k < items.size(); ++k) hi[k] = items[k].second;
    std::memset(hb, 0, sizeof(int));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(db, hb, sizeof(int), cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(db + o_par, hb + o_par, o_it - o_par + sizeof(int2) * items.size(),
                                     cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, cudaEventRecord(ctx->pb_done, st));
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (ctx->profile) {
        ev = prof_pair(ctx);
        cudaEventRecord(ev.first, st);
    }
    const Shape &s0 = shapes[0];
    cudaError_t e = launch_project_batch<Real>(reinterpret_cast<const ProjParams<Real> *>(db + o_par),
                                               reinterpret_cast<const int2 *>(db + o_it), int(items.size()),
                                               reinterpret_cast<int *>(db), s0.dims, R, 0, s0.nf, s0.nv, want_lambda,
                                               smem, 0, st, kind);
    ctx->launches++;
    ctx->last_kind = kind;
    if (ev.first) {
        cudaEventRecord(ev.second, st);
        ctx->prof_used.push_back(ev);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched projection");
    return PRIEST_OK;
}

// ---------------------------------------------------------------------------
// Batched solves through host buffers: the problems stay resident behind
// handles the context owns while their layout (sizes, obstacle counts, the
// tilings they imply) is unchanged; each call uploads the problems' data and
// draws, replays the recorded solve and copies the results back.
// ---------------------------------------------------------------------------

// Layout of a problem as far as the resident buffers and recorded launches
// depend on it (the rest -- obstacle values, boundary values, bounds, costs
// -- is uploaded by every call).
std::vector<double> host_layout_key(const Shape &sh)
{
    return {double(sh.dims), double(sh.nv), double(sh.nf), double(sh.n_p), double(sh.n_obs), double(sh.n_static),
            double(sh.N), double(sh.n_proj), double(sh.n_elite), double(sh.use_bounds), sh.horizon};
}

// ---- transfers of the host-buffer batched solve: every piece of one
//      direction in a single launch instead of one copy call per problem
constexpr int kXferThreads = 256;
constexpr long long kXferChunk = 32768;  // doubles per CTA (256 KB), even: chunks keep 16-byte alignment
constexpr int kSideCtas = 16;            // CTAs of a transfer that runs beside the solve

// Chunks n_chunks apart per CTA (one each when the grid covers them), plain
// loads and stores (16 bytes when both ends are 16-byte aligned, four in
// flight per thread), so pinned host memory is read or written over the host
// link directly.
__global__ void __launch_bounds__(kXferThreads) xfer_kernel(const XferChunk *chunks, int n_chunks)
{
    const int t = threadIdx.x;
    for (int k = blockIdx.x; k < n_chunks; k += gridDim.x) {
        const XferChunk c = chunks[k];
        if (((reinterpret_cast<uintptr_t>(c.src) | reinterpret_cast<uintptr_t>(c.dst)) & 15) == 0) {
            const long long n2 = c.count >> 1;
            const double2 *src = reinterpret_cast<const double2 *>(c.src);
            double2 *dst = reinterpret_cast<double2 *>(c.dst);
            long long i = t;
            for (; i + 3 * kXferThreads < n2; i += 4 * kXferThreads) {
                const double2 a = src[i], b = src[i + kXferThreads], e = src[i + 2 * kXferThreads],
                              f = src[i + 3 * kXferThreads];
                dst[i] = a;
                dst[i + kXferThreads] = b;
                dst[i + 2 * kXferThreads] = e;
                dst[i + 3 * kXferThreads] = f;
            }
            for (; i < n2; i += kXferThreads) dst[i] = src[i];
            if (t == 0 && (c.count & 1)) c.dst[c.count - 1] = c.src[c.count - 1];
        } else {
            for (long long i = t; i < c.count; i += kXferThreads) c.dst[i] = c.src[i];
        }
    }
}

// The device view of host memory a kernel may access: page-locked, mapped
// memory only (cudaMallocHost, cudaHostAlloc, cudaHostRegister); nullptr for
// pageable memory, which is then copied by DMA instead.
double *device_view(const void *p)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return static_cast<double *>(a.devicePointer);
}

size_t xfer_chunks(size_t count) { return (count + size_t(kXferChunk) - 1) / size_t(kXferChunk); }

void add_xfer(std::vector<XferChunk> &v, const double *src, double *dst, size_t count)
{
    for (size_t o = 0; o < count; o += size_t(kXferChunk))
        v.push_back({src + o, dst + o, (long long)std::min(size_t(kXferChunk), count - o)});
}

// Writes the chunk list into its pinned table (grown when needed) and
// launches one transfer over it on st, with at most max_ctas CTAs (0: one
// per chunk).
cudaError_t run_xfer(const std::vector<XferChunk> &v, XferChunk *&table, XferChunk *&table_dev, size_t &cap,
                     cudaStream_t st, int max_ctas = 0)
{
    if (v.empty()) return cudaSuccess;
    if (v.size() > cap) {
        cudaError_t e = cudaStreamSynchronize(st);  // the old table may still be read
        if (e != cudaSuccess) return e;
        if (table) cudaFreeHost(table);
        table = nullptr;
        table_dev = nullptr;
        cap = 0;
        e = cudaMallocHost(&table, sizeof(XferChunk) * v.size());
        if (e != cudaSuccess) return e;
        table_dev = reinterpret_cast<XferChunk *>(device_view(table));
        if (!table_dev) return cudaErrorInvalidValue;
        cap = v.size();
    }
    std::memcpy(table, v.data(), sizeof(XferChunk) * v.size());
    const int n = int(v.size());
    xfer_kernel<<<unsigned(max_ctas > 0 ? std::min(n, max_ctas) : n), kXferThreads, 0, st>>>(table_dev, n);
    return cudaGetLastError();
}

void free_host_batch(priest_ctx *ctx)
{
    HostBatch *hb = ctx->hbatch;
    if (!hb) return;
    cudaStreamSynchronize(ctx->stream);
    std::vector<double *> zp(hb->n), op(hb->n);
    for (int i = 0; i < hb->n; ++i) {
        zp[i] = hb->zdev + hb->z_off[i];
        op[i] = hb->odev + size_t(i) * hb->ostride;
    }
    if (hb->n > 0) {
        auto it = ctx->batches.find(batch_key(hb->n, hb->h.data(), zp.data(), op.data()));
        if (it != ctx->batches.end()) {
            free_batch(it->second);
            ctx->batches.erase(it);
        }
    }
    for (priest_loaded *h : hb->h) free_loaded(h);
    if (hb->zdev) cudaFree(hb->zdev);
    if (hb->odev) cudaFree(hb->odev);
    if (hb->stage) cudaFreeHost(hb->stage);
    if (hb->cstream) {
        cudaStreamSynchronize(hb->cstream);  // before its chunk table goes
        cudaStreamDestroy(hb->cstream);
    }
    if (hb->xin) cudaFreeHost(hb->xin);
    if (hb->xout) cudaFreeHost(hb->xout);
    if (hb->xside) cudaFreeHost(hb->xside);
    if (hb->zev) cudaEventDestroy(hb->zev);
    delete hb;
    ctx->hbatch = nullptr;
}

template <typename Real>
priest_status plan_batch_host(priest_ctx *ctx, int n, const priest_problem *probs, const double *const *z,
                              priest_result *out)
{
    cudaStream_t st = ctx->stream;
    const int L = ctx->cfg.cem_iters;
    std::vector<Shape> shapes(n);
    std::vector<std::vector<double>> oc(n), ov(n), os(n);
    std::vector<double> key;
    for (int i = 0; i < n; ++i) {
        priest_status s = resolve(ctx, &probs[i], -1, shapes[i]);
        if (s != PRIEST_OK) return s;
        if (shapes[i].dims != shapes[0].dims || shapes[i].bc_mask != shapes[0].bc_mask)
            return fail(ctx, PRIEST_ERR_INVALID, "batched problems must share dims, degree and bc_final_mask");
        order_obstacles(shapes[i], probs[i].center, probs[i].vel, probs[i].semi, oc[i], ov[i], os[i],
                        shapes[i].n_static);
        const std::vector<double> k = host_layout_key(shapes[i]);
        key.insert(key.end(), k.begin(), k.end());
    }
    const bool fp32 = ctx->cfg.precision != PRIEST_FP64_CHECK;
    const int D = shapes[0].D;
    bool reuse = ctx->hbatch && ctx->hbatch->key == key;
    if (!reuse) {
        free_host_batch(ctx);
        HostBatch *hb = new HostBatch();
        ctx->hbatch = hb;
        hb->key = key;
        hb->ostride = size_t(D) + 8;
        size_t zt = 0, sb = 0;
        for (int i = 0; i < n; ++i) {
            hb->z_off.push_back(zt);
            zt += size_t(L) * shapes[i].N * D;
            const Carve k = carve(shapes[i], fp32, 0, false);
            hb->ob_off.push_back(sb);
            hb->ob_bytes.push_back(k.semi - k.center + sizeof(double) * 2 * std::max(shapes[i].n_obs, 1));
            sb = round_up(sb + hb->ob_bytes.back());
        }
        hb->out_off = sb;
        hb->mu_off = round_up(sb + sizeof(double) * hb->ostride * n);
        const size_t stage_bytes = hb->mu_off + sizeof(double) * size_t(D) * n;
        if (cudaMalloc(&hb->zdev, sizeof(double) * std::max<size_t>(zt, 1)) != cudaSuccess ||
            cudaMalloc(&hb->odev, sizeof(double) * hb->ostride * n) != cudaSuccess ||
            cudaMallocHost(&hb->stage, stage_bytes) != cudaSuccess) {
            cudaGetLastError();
            free_host_batch(ctx);
            return fail(ctx, PRIEST_ERR_NOMEM, "batched solve buffers");
        }
        hb->stage_dev = reinterpret_cast<char *>(device_view(hb->stage));
        if (cudaStreamCreateWithFlags(&hb->cstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&hb->zev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            free_host_batch(ctx);
            return fail(ctx, PRIEST_ERR_CUDA, "batched solve stream");
        }
        for (int i = 0; i < n; ++i) {
            priest_loaded *h = nullptr;
            priest_status s = make_loaded(ctx, shapes[i], probs[i].center, probs[i].vel, probs[i].semi, 0, false, st, &h);
            if (s != PRIEST_OK) {
                free_host_batch(ctx);
                return s;
            }
            hb->h.push_back(h);
            hb->n = int(hb->h.size());
        }
    }
    HostBatch *hb = ctx->hbatch;
    std::vector<XferChunk> in, out_x, side_x;
    if (reuse) {
        // same layout: new problem data into the resident buffers
        for (int i = 0; i < n; ++i) {
            priest_loaded *h = hb->h[i];
            const bool ready = h->shape_ready;
            h->sh = shapes[i];
            h->shape_ready = ready;
            char *dst = hb->stage + hb->ob_off[i];
            const size_t vo = reinterpret_cast<char *>(h->vel) - reinterpret_cast<char *>(h->center),
                         so = reinterpret_cast<char *>(h->semi) - reinterpret_cast<char *>(h->center);
            std::memcpy(dst, oc[i].data(), sizeof(double) * oc[i].size());
            std::memcpy(dst + vo, ov[i].data(), sizeof(double) * ov[i].size());
            std::memcpy(dst + so, os[i].data(), sizeof(double) * os[i].size());
            if (hb->stage_dev)
                add_xfer(in, reinterpret_cast<const double *>(hb->stage_dev + hb->ob_off[i]), h->center,
                         hb->ob_bytes[i] / sizeof(double));
            else
                PRIEST_CUDA(ctx, cudaMemcpyAsync(h->center, dst, hb->ob_bytes[i], cudaMemcpyHostToDevice, st));
        }
    }
    // draws: from a pinned buffer, those of the first CEM iteration are read
    // in place by the transfer kernel on the solve stream and the later
    // iterations' by a narrow transfer (kSideCtas CTAs) on the side stream,
    // beside the set-up and the first projection (the recorded launches wait
    // for hb->zev before the second projection; the persistent projection
    // takes its items from a counter, so the CTAs the transfer holds for a
    // while cost it nothing but their slots); a pageable buffer is copied
    // whole by DMA on the solve stream.  Every return from here waits for
    // the side stream, since the caller may release the draws.
    struct SideCopies {
        cudaStream_t s;
        ~SideCopies() { cudaStreamSynchronize(s); }
    } side{hb->cstream};
    std::vector<const double *> zp(n);
    std::vector<double *> op(n);
    for (int i = 0; i < n; ++i) {
        double *zd = hb->zdev + hb->z_off[i];
        const size_t first = size_t(shapes[i].N) * D, cnt = size_t(L) * first;
        if (const double *zv = device_view(z[i])) {
            add_xfer(in, zv, zd, first);
            add_xfer(side_x, zv + first, zd + first, cnt - first);
        } else {
            PRIEST_CUDA(ctx, cudaMemcpyAsync(zd, z[i], sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
        }
        zp[i] = zd;
        op[i] = hb->odev + size_t(i) * hb->ostride;
    }
    PRIEST_CUDA(ctx, run_xfer(side_x, hb->xside, hb->xside_dev, hb->xside_cap, hb->cstream, kSideCtas));
    if (!side_x.empty()) ctx->launches++;
    PRIEST_CUDA(ctx, cudaEventRecord(hb->zev, hb->cstream));
    if (!in.empty()) {
        PRIEST_CUDA(ctx, run_xfer(in, hb->xin, hb->xin_dev, hb->xin_cap, st));
        ctx->launches++;
    }
    priest_status s = plan_batch<Real>(ctx, n, hb->h.data(), zp.data(), op.data(), reuse, hb->zev);
    if (s != PRIEST_OK) return s;
    double *ho = reinterpret_cast<double *>(hb->stage + hb->out_off);
    double *hm = reinterpret_cast<double *>(hb->stage + hb->mu_off);
    if (hb->stage_dev) {
        // results and means written into the pinned stage by one transfer
        add_xfer(out_x, hb->odev, reinterpret_cast<double *>(hb->stage_dev + hb->out_off), hb->ostride * n);
        for (int i = 0; i < n; ++i)
            add_xfer(out_x, hb->h[i]->mu, reinterpret_cast<double *>(hb->stage_dev + hb->mu_off) + size_t(i) * D, D);
        PRIEST_CUDA(ctx, run_xfer(out_x, hb->xout, hb->xout_dev, hb->xout_cap, st));
        ctx->launches++;
    } else {
        PRIEST_CUDA(ctx, cudaMemcpyAsync(ho, hb->odev, sizeof(double) * hb->ostride * n, cudaMemcpyDeviceToHost, st));
        for (int i = 0; i < n; ++i)
            PRIEST_CUDA(ctx, cudaMemcpyAsync(hm + size_t(i) * D, hb->h[i]->mu, sizeof(double) * D,
                                             cudaMemcpyDeviceToHost, st));
    }
    s = check_status(ctx, ctx->d_status, st);
    for (int i = 0; i < n; ++i) {
        fill_result(shapes[i], ho + size_t(i) * hb->ostride, hm + size_t(i) * D, &out[i]);
        out[i].status = s;
    }
    return s;
}

// D-PRIEST default means: the straight-line coefficients with every
// interior coefficient moved by (j - (M-1)/2) spread along the unit normal of
// the start-goal line (2-D: rotated by +90 degrees; 3-D: the horizontal
// normal; x when undefined).
void multi_default_means(const Shape &sh, int M, double spread, double *mu)
{
    const int nv = sh.nv, n = sh.degree, D = sh.D;
    double d[3] = {0.0, 0.0, 0.0}, nrm[3] = {0.0, 0.0, 0.0};
    for (int ax = 0; ax < sh.dims; ++ax) d[ax] = sh.bf[ax][0] - sh.b0[ax][0];
    const double h = std::sqrt(d[0] * d[0] + d[1] * d[1]);
    if (h > 1e-12) {
        nrm[0] = -d[1] / h;
        nrm[1] = d[0] / h;
    } else {
        nrm[0] = 1.0;
    }
    for (int j = 0; j < M; ++j) {
        const double off = (double(j) - 0.5 * double(M - 1)) * spread;
        for (int ax = 0; ax < sh.dims; ++ax)
            for (int k = 0; k < nv; ++k) {
                double v = sh.b0[ax][0] + (sh.bf[ax][0] - sh.b0[ax][0]) * double(k) / double(n);
                if (k >= 1 && k < n) v += off * nrm[ax];
                mu[size_t(j) * D + ax * nv + k] = v;
            }
    }
}

priest_status plan_multi(priest_ctx *ctx, const priest_problem *pr, int M, const double *mu0, const double *cov0,
                         const double *z_host, priest_result *best, int *best_dist, priest_result *per_dist)
{
    if (!ctx || !best || M < 1) return fail(ctx, PRIEST_ERR_INVALID, "NULL argument or M < 1");
    Shape sh;
    priest_status s = resolve(ctx, pr, -1, sh);
    if (s != PRIEST_OK) return s;
    const int N = sh.N, D = sh.D, L = ctx->cfg.cem_iters;
    if (N % M) return fail(ctx, PRIEST_ERR_INVALID, "n_samples must be a multiple of M");
    const int nj = N / M, npj = std::max(1, sh.n_proj / M), nej = std::max(1, sh.n_elite / M);
    if (npj > nj || nej > npj) return fail(ctx, PRIEST_ERR_INVALID, "need n_elite / M <= n_proj / M <= n_samples / M");
    priest_loaded *h = nullptr;
    s = scratch_for(ctx, sh, pr, L, false, &h);
    if (s != PRIEST_OK) return s;
    // per-distribution state: mu, Sigma, L, mu', elites, result rows, refit counters, CEM arguments
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = round_up(o + bytes);
        return at;
    };
    const size_t o_mu = take(sizeof(double) * M * D), o_cov = take(sizeof(double) * M * D * D),
                 o_L = take(sizeof(double) * M * D * D), o_mn = take(sizeof(double) * M * D),
                 o_el = take(sizeof(int) * M * nej), o_out = take(sizeof(double) * M * (D + 5)),
                 o_cnt = take(sizeof(unsigned) * M), o_args = take(sizeof(CemArgs) * M);
    char *blk = nullptr;
    PRIEST_CUDA(ctx, cudaMalloc(reinterpret_cast<void **>(&blk), o));
    struct Free {
        char *p;
        ~Free() { cudaFree(p); }
    } guard{blk};
    double *mu = reinterpret_cast<double *>(blk + o_mu), *cov = reinterpret_cast<double *>(blk + o_cov);
    double *Lc = reinterpret_cast<double *>(blk + o_L), *mn = reinterpret_cast<double *>(blk + o_mn);
    int *el = reinterpret_cast<int *>(blk + o_el);
    double *out = reinterpret_cast<double *>(blk + o_out);
    unsigned *cnt = reinterpret_cast<unsigned *>(blk + o_cnt);
    CemArgs *args = reinterpret_cast<CemArgs *>(blk + o_args);
    cudaStream_t st = ctx->stream;
    // inputs: draws, means, covariances, argument blocks
    const size_t nz = size_t(L) * N * D;
    std::vector<double> zbuf, hmu(size_t(M) * D), hcov;
    if (!z_host) {
        zbuf.resize(nz);
        gaussian_stream(pr->seed, int64_t(nz), zbuf.data());
        z_host = zbuf.data();
    }
    if (mu0)
        std::copy(mu0, mu0 + size_t(M) * D, hmu.begin());
    else
        multi_default_means(sh, M, 2.0 * ctx->cfg.init_std, hmu.data());
    if (!cov0) {
        hcov.assign(size_t(M) * D * D, 0.0);
        for (int j = 0; j < M; ++j)
            for (int i = 0; i < D; ++i) hcov[size_t(j) * D * D + size_t(i) * D + i] = ctx->cfg.init_std * ctx->cfg.init_std;
        cov0 = hcov.data();
    }
    std::vector<CemArgs> ha(M);
    for (int j = 0; j < M; ++j) {
        CemArgs &a = ha[j];
        std::memset(&a, 0, sizeof(a));
        a.N = nj;
        a.n_proj = npj;
        a.n_elite = nej;
        a.D = D;
        a.r = h->r + size_t(j) * nj;
        a.c1 = h->c1 + size_t(j) * nj;
        a.xb = h->xb + size_t(j) * nj * D;
        a.elite = el + size_t(j) * nej;
        a.sigma = ctx->cfg.sigma_lr;
        a.gamma = ctx->cfg.gamma;
        a.chol_eps = ctx->cfg.chol_eps;
        a.mu = mu + size_t(j) * D;
        a.cov = cov + size_t(j) * D * D;
        a.mu_new = mn + size_t(j) * D;
        a.L = Lc + size_t(j) * D * D;
        a.counter = cnt + j;
        a.status = ctx->d_status;
        a.best_out = out + size_t(j) * (D + 5);
    }
    PRIEST_CUDA(ctx, cudaMemcpyAsync(h->z, z_host, nz * sizeof(double), cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(mu, hmu.data(), sizeof(double) * M * D, cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(cov, cov0, sizeof(double) * M * D * D, cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(args, ha.data(), sizeof(CemArgs) * M, cudaMemcpyHostToDevice, st));
    PRIEST_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned) * M, st));
    // a0: tables once, then the first sampling factor of each distribution
    for (int j = 0; j < M; ++j) {
        SetupParams sp = setup_params(ctx, h, true, ctx->d_status);
        sp.mu = mu + size_t(j) * D;
        sp.cov = cov + size_t(j) * D * D;
        sp.L = Lc + size_t(j) * D * D;
        sp.default_mu = 0;
        sp.default_cov = 0;
        sp.shape_ready = (j > 0 || h->shape_ready) ? 1 : 0;
        cudaError_t e = launch_setup(sp, st);
        ctx->launches++;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "setup kernel");
    }
    h->shape_ready = true;
    // per CEM iteration: one projection of all distributions' rows, then
    // selections and refits per distribution (segmented)
    double *mu_keep = h->mu, *L_keep = h->L;
    h->mu = mu;
    h->L = Lc;
    h->seg_len = nj;
    const size_t sel_smem = select_smem_bytes(nj), ref_smem = refit_smem_bytes(D, nej);
    for (int l = 0; l < L && s == PRIEST_OK; ++l) {
        s = enqueue_project_any(ctx, h, N, 1, nullptr, h->z + size_t(l) * N * D, nullptr, nullptr, h->xb, h->r,
                                h->c1, st);
        if (s != PRIEST_OK) break;
        cudaError_t e = launch_select_batch(args, M, sel_smem, st);
        if (e == cudaSuccess) e = launch_refit_batch(args, M, D, ref_smem, st);
        ctx->launches += 2;
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "segmented selection / refit");
    }
    h->mu = mu_keep;
    h->L = L_keep;
    h->seg_len = 0;
    if (s != PRIEST_OK) return s;
    // best of M (ties: the lower j)
    std::vector<double> ho(size_t(M) * (D + 5)), hm(size_t(M) * D);
    PRIEST_CUDA(ctx, cudaMemcpyAsync(ho.data(), out, sizeof(double) * ho.size(), cudaMemcpyDeviceToHost, st));
    PRIEST_CUDA(ctx, cudaMemcpyAsync(hm.data(), mu, sizeof(double) * hm.size(), cudaMemcpyDeviceToHost, st));
    s = check_status(ctx, ctx->d_status, st);
    if (s != PRIEST_OK) return s;
    int jb = 0;
    for (int j = 1; j < M; ++j)
        if (ho[size_t(j) * (D + 5) + D + 2] < ho[size_t(jb) * (D + 5) + D + 2]) jb = j;
    for (int j = 0; j < M && per_dist; ++j) fill_result(sh, &ho[size_t(j) * (D + 5)], &hm[size_t(j) * D], &per_dist[j]);
    fill_result(sh, &ho[size_t(jb) * (D + 5)], &hm[size_t(jb) * D], best);
    if (best_dist) *best_dist = jb;
    return PRIEST_OK;
}

}  // namespace

extern "C" {

priest_status priest_plan_batch(priest_ctx *ctx, int n, priest_loaded *const *probs, const double *const *z_dev,
                                double *const *out_dev)
{
    if (!ctx) return PRIEST_ERR_INVALID;
    if (n < 1 || !probs || !z_dev || !out_dev) return fail(ctx, PRIEST_ERR_INVALID, "empty batch or NULL lists");
    for (int i = 0; i < n; ++i)
        if (!probs[i] || !z_dev[i] || !out_dev[i]) return fail(ctx, PRIEST_ERR_INVALID, "NULL entry in the batch");
    if (ctx->cfg.precision == PRIEST_FP64_CHECK) return plan_batch<double>(ctx, n, probs, z_dev, out_dev);
    return plan_batch<float>(ctx, n, probs, z_dev, out_dev);
}

priest_status priest_plan_batch_host(priest_ctx *ctx, int n, const priest_problem *probs, const double *const *z,
                                     priest_result *out)
{
    if (!ctx) return PRIEST_ERR_INVALID;
    if (n < 1 || !probs || !z || !out) return fail(ctx, PRIEST_ERR_INVALID, "empty batch or NULL lists");
    for (int i = 0; i < n; ++i)
        if (!z[i]) return fail(ctx, PRIEST_ERR_INVALID, "NULL draws in the batch");
    if (ctx->cfg.precision == PRIEST_FP64_CHECK) return plan_batch_host<double>(ctx, n, probs, z, out);
    return plan_batch_host<float>(ctx, n, probs, z, out);
}

priest_status priest_project_batch(priest_ctx *ctx, int n, priest_loaded *const *probs, const int *rows,
                                   const double *const *xi_dev, double *const *lambda_dev,
                                   double *const *xi_bar_dev, double *const *resid_dev, double *const *cost_dev)
{
    if (!ctx) return PRIEST_ERR_INVALID;
    if (n < 1 || !probs || !rows || !xi_dev || !xi_bar_dev || !resid_dev || !cost_dev)
        return fail(ctx, PRIEST_ERR_INVALID, "empty batch or NULL lists");
    int total = 0;
    for (int i = 0; i < n; ++i) {
        if (!probs[i]) return fail(ctx, PRIEST_ERR_INVALID, "NULL handle in the batch");
        if (rows[i] < 0 || rows[i] > probs[i]->sh.N)
            return fail(ctx, PRIEST_ERR_INVALID, "row count exceeds the loaded sample count");
        if (rows[i] > 0 && (!xi_dev[i] || !xi_bar_dev[i] || !resid_dev[i] || !cost_dev[i]))
            return fail(ctx, PRIEST_ERR_INVALID, "NULL pointer in the batch");
        if (probs[i]->sh.dims != probs[0]->sh.dims || probs[i]->sh.nv != probs[0]->sh.nv ||
            probs[i]->sh.bc_mask != probs[0]->sh.bc_mask)
            return fail(ctx, PRIEST_ERR_INVALID, "batched problems must share dims, degree and bc_final_mask");
        total += rows[i];
    }
    if (total == 0) return PRIEST_OK;
    if (ctx->cfg.precision == PRIEST_FP64_CHECK)
        return project_batch<double>(ctx, n, probs, rows, xi_dev, lambda_dev, xi_bar_dev, resid_dev, cost_dev);
    return project_batch<float>(ctx, n, probs, rows, xi_dev, lambda_dev, xi_bar_dev, resid_dev, cost_dev);
}

priest_status priest_read_elites(priest_ctx *ctx, const priest_loaded *h, int *elite_out, double *resid_out,
                                 double *cost_out)
{
    if (!ctx) return PRIEST_ERR_INVALID;
    const priest_loaded *src = h ? h : ctx->scratch;
    if (!src) return fail(ctx, PRIEST_ERR_INVALID, "no solve to read");
    const Shape &sh = src->sh;
    PRIEST_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (elite_out)
        PRIEST_CUDA(ctx, cudaMemcpy(elite_out, src->elite, sizeof(int) * sh.n_elite, cudaMemcpyDeviceToHost));
    if (resid_out) PRIEST_CUDA(ctx, cudaMemcpy(resid_out, src->r, sizeof(double) * sh.N, cudaMemcpyDeviceToHost));
    if (cost_out) PRIEST_CUDA(ctx, cudaMemcpy(cost_out, src->c1, sizeof(double) * sh.N, cudaMemcpyDeviceToHost));
    return PRIEST_OK;
}

int priest_last_kernel(const priest_ctx *ctx) { return ctx ? ctx->last_kind : -1; }

priest_status priest_grid_info(priest_ctx *ctx, const priest_loaded *h, int *out)
{
    if (!ctx || !out) return PRIEST_ERR_INVALID;
    const priest_loaded *src = h ? h : ctx->scratch;
    if (!src) return fail(ctx, PRIEST_ERR_INVALID, "no loaded problem to read");
    if (!src->tab32) return fail(ctx, PRIEST_ERR_INVALID, "the problem has no FP32 tables");
    const Shape &sh = src->sh;
    const TableLayout lay = table_layout(sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs);
    int hdr[8];
    PRIEST_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    PRIEST_CUDA(ctx, cudaMemcpy(hdr, src->tab32 + lay.grid, sizeof(hdr), cudaMemcpyDeviceToHost));
    out[0] = hdr[4];
    out[1] = hdr[5];
    out[2] = hdr[4] > 0 ? hdr[6] : 0;
    return PRIEST_OK;
}


priest_status priest_rng_normal(uint64_t seed, int64_t count, double *out)
{
    if (count < 0 || (count > 0 && !out)) return PRIEST_ERR_INVALID;
    gaussian_stream(seed, count, out);
    return PRIEST_OK;
}

priest_status priest_rng_normal_device(uint64_t seed, int64_t count, double *out_dev, void *cuda_stream)
{
    if (count < 0 || (count > 0 && !out_dev)) return PRIEST_ERR_INVALID;
    const cudaError_t e = launch_normal(seed, count, out_dev, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PRIEST_ERR_CUDA;
    }
    return PRIEST_OK;
}

priest_status priest_create(const priest_config *cfg, void *cuda_stream, priest_ctx **out)
{
    if (!cfg || !out) return PRIEST_ERR_INVALID;
    *out = nullptr;
    if (cfg->degree < 5 || cfg->degree > 15 || cfg->proj_iters < 0 || cfg->cem_iters < 1 || !(cfg->rho > 0) ||
        !(cfg->gamma > 0) || cfg->sigma_lr < 0 || cfg->sigma_lr > 1 || cfg->chol_eps < 0 ||
        (cfg->precision != PRIEST_FP64_CHECK && cfg->precision != PRIEST_FP32 && cfg->precision != PRIEST_MIXED_BF16) ||
        cfg->serve_slots < 0)
        return PRIEST_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return PRIEST_ERR_CUDA;
    }
    priest_ctx *ctx = new (std::nothrow) priest_ctx();
    if (!ctx) return PRIEST_ERR_NOMEM;
    ctx->cfg = *cfg;
    cudaGetDevice(&ctx->device);
    cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return PRIEST_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaMalloc(&ctx->d_status, 2 * sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, 2 * sizeof(int)) != cudaSuccess) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return PRIEST_ERR_CUDA;
    }
    *out = ctx;
    return PRIEST_OK;
}

priest_status priest_destroy(priest_ctx *ctx)
{
    if (!ctx) return PRIEST_OK;
    server_destroy(ctx);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_host_batch(ctx);
    free_loaded(ctx->scratch);
    if (ctx->pb_dev) cudaFree(ctx->pb_dev);
    if (ctx->pb_host) cudaFreeHost(ctx->pb_host);
    if (ctx->pb_done) cudaEventDestroy(ctx->pb_done);
    if (ctx->plain_work) cudaFree(ctx->plain_work);
    for (auto &kv : ctx->batches) free_batch(kv.second);
    for (auto &ev : ctx->prof_used) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    for (auto &ev : ctx->prof_free) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    cudaFree(ctx->d_status);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return PRIEST_OK;
}

const char *priest_last_error(const priest_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

int64_t priest_kernel_launches(const priest_ctx *ctx) { return ctx ? ctx->launches.load() : 0; }

priest_status priest_profile_enable(priest_ctx *ctx, int enable)
{
    if (!ctx) return PRIEST_ERR_INVALID;
    ctx->profile = enable != 0;
    return PRIEST_OK;
}

priest_status priest_profile_read(priest_ctx *ctx, int64_t *launches, double *ms)
{
    if (!ctx || !launches || !ms) return PRIEST_ERR_INVALID;
    double total = 0.0;
    for (auto &ev : ctx->prof_used) {
        PRIEST_CUDA(ctx, cudaEventSynchronize(ev.second));
        float t = 0.f;
        PRIEST_CUDA(ctx, cudaEventElapsedTime(&t, ev.first, ev.second));
        total += t;
    }
    *launches = int64_t(ctx->prof_used.size());
    *ms = total;
    ctx->prof_free.insert(ctx->prof_free.end(), ctx->prof_used.begin(), ctx->prof_used.end());
    ctx->prof_used.clear();
    return PRIEST_OK;
}

priest_status priest_sync(priest_ctx *ctx)
{
    if (!ctx) return PRIEST_ERR_INVALID;
    PRIEST_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_status(ctx, ctx->d_status, ctx->stream);
}

priest_status priest_project(priest_ctx *ctx, const priest_problem *pr, int n, const double *xi,
                             double *lambda_io, double *xi_bar_out, double *resid_out, double *cost_out)
{
    if (!ctx) return PRIEST_ERR_INVALID;
    if (n < 0 || n > PRIEST_MAX_SAMPLES) return fail(ctx, PRIEST_ERR_INVALID, "n out of range");
    if (n > 0 && (!xi || !xi_bar_out)) return fail(ctx, PRIEST_ERR_INVALID, "xi / xi_bar_out is NULL");
    Shape sh;
    priest_status s = resolve(ctx, pr, n, sh);
    if (s != PRIEST_OK) return s;
    for (size_t i = 0; i < size_t(n) * sh.D; ++i)
        if (!is_fin(xi[i]) || (lambda_io && !is_fin(lambda_io[i])))
            return fail(ctx, PRIEST_ERR_INVALID, "xi / lambda must be finite");
    if (n == 0) return PRIEST_OK;
    priest_loaded *h = nullptr;
    s = scratch_for(ctx, sh, pr, 0, true, &h);
    if (s != PRIEST_OK) return s;
    const size_t bytes = size_t(n) * sh.D * sizeof(double);
    PRIEST_CUDA(ctx, cudaMemcpyAsync(h->xi, xi, bytes, cudaMemcpyHostToDevice, ctx->stream));
    if (lambda_io) PRIEST_CUDA(ctx, cudaMemcpyAsync(h->lam, lambda_io, bytes, cudaMemcpyHostToDevice, ctx->stream));
    s = enqueue_setup(ctx, h, false, ctx->stream, ctx->d_status);
    if (s != PRIEST_OK) return s;
    s = enqueue_project_any(ctx, h, n, 0, h->xi, nullptr, lambda_io ? h->lam : nullptr,
                            lambda_io ? h->lam : nullptr, h->xb, h->r, h->c1, ctx->stream);
    if (s != PRIEST_OK) return s;
    PRIEST_CUDA(ctx, cudaMemcpyAsync(xi_bar_out, h->xb, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (lambda_io) PRIEST_CUDA(ctx, cudaMemcpyAsync(lambda_io, h->lam, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (resid_out)
        PRIEST_CUDA(ctx, cudaMemcpyAsync(resid_out, h->r, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (cost_out)
        PRIEST_CUDA(ctx, cudaMemcpyAsync(cost_out, h->c1, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return check_status(ctx, ctx->d_status, ctx->stream);
}

priest_status priest_plan(priest_ctx *ctx, const priest_problem *pr, const double *mu0, const double *cov0,
                          priest_result *out)
{
    return plan_host(ctx, pr, mu0, cov0, nullptr, out);
}

priest_status priest_plan_z(priest_ctx *ctx, const priest_problem *pr, const double *mu0, const double *cov0,
                            const double *z, priest_result *out)
{
    if (!z) return fail(ctx, PRIEST_ERR_INVALID, "z is NULL");
    return plan_host(ctx, pr, mu0, cov0, z, out);
}

priest_status priest_plan_plain(priest_ctx *ctx, const priest_problem *pr, const double *mu0, const double *cov0,
                                const double *z, priest_result *out)
{
    return plan_host(ctx, pr, mu0, cov0, z, out, true);
}

priest_status priest_plan_multi(priest_ctx *ctx, const priest_problem *pr, int M, const double *mu0,
                                const double *cov0, const double *z, priest_result *best, int *best_dist,
                                priest_result *per_dist)
{
    return plan_multi(ctx, pr, M, mu0, cov0, z, best, best_dist, per_dist);
}

priest_status priest_plan_plain_device(priest_ctx *ctx, priest_loaded *h, const double *z_dev, double *out_dev)
{
    if (!ctx || !h || !z_dev || !out_dev) return fail(ctx, PRIEST_ERR_INVALID, "NULL argument");
    h->default_mu = true;
    h->default_cov = true;
    return enqueue_plan_plain(ctx, h, z_dev, out_dev, ctx->stream, ctx->d_status);
}

priest_status priest_project_plain(priest_ctx *ctx, const priest_problem *pr, int n, const double *xi,
                                   double *lambda_io, double *xi_bar_out, double *resid_out, double *cost_out)
{
    if (!ctx) return PRIEST_ERR_INVALID;
    if (n < 0 || n > PRIEST_MAX_SAMPLES) return fail(ctx, PRIEST_ERR_INVALID, "n out of range");
    if (n > 0 && (!xi || !xi_bar_out)) return fail(ctx, PRIEST_ERR_INVALID, "xi / xi_bar_out is NULL");
    Shape sh;
    priest_status s = resolve(ctx, pr, n, sh);
    if (s != PRIEST_OK) return s;
    for (size_t i = 0; i < size_t(n) * sh.D; ++i)
        if (!is_fin(xi[i]) || (lambda_io && !is_fin(lambda_io[i])))
            return fail(ctx, PRIEST_ERR_INVALID, "xi / lambda must be finite");
    if (n == 0) return PRIEST_OK;
    float *work = nullptr;
    s = plain_workspace(ctx, sh, n, &work);
    if (s != PRIEST_OK) return s;
    priest_loaded *h = nullptr;
    s = scratch_for(ctx, sh, pr, 0, true, &h);
    if (s != PRIEST_OK) return s;
    const size_t bytes = size_t(n) * sh.D * sizeof(double);
    PRIEST_CUDA(ctx, cudaMemcpyAsync(h->xi, xi, bytes, cudaMemcpyHostToDevice, ctx->stream));
    if (lambda_io) PRIEST_CUDA(ctx, cudaMemcpyAsync(h->lam, lambda_io, bytes, cudaMemcpyHostToDevice, ctx->stream));
    s = enqueue_setup(ctx, h, false, ctx->stream, ctx->d_status);
    if (s != PRIEST_OK) return s;
    PlainParams p = plain_params(ctx, h, n, work);
    p.mode = 0;
    p.xi_in = h->xi;
    p.lam_in = lambda_io ? h->lam : nullptr;
    p.lam_out = lambda_io ? h->lam : nullptr;
    p.xi_bar = h->xb;
    p.r_out = h->r;
    p.c1_out = h->c1;
    int64_t nl = 0;
    cudaError_t e = launch_plain_project(p, ctx->stream, &nl);
    ctx->launches += nl;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "plain projection");
    PRIEST_CUDA(ctx, cudaMemcpyAsync(xi_bar_out, h->xb, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (lambda_io) PRIEST_CUDA(ctx, cudaMemcpyAsync(lambda_io, h->lam, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (resid_out)
        PRIEST_CUDA(ctx, cudaMemcpyAsync(resid_out, h->r, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (cost_out)
        PRIEST_CUDA(ctx, cudaMemcpyAsync(cost_out, h->c1, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return check_status(ctx, ctx->d_status, ctx->stream);
}

priest_status priest_load(priest_ctx *ctx, const priest_problem *pr, priest_loaded **out)
{
    if (!ctx || !out) return PRIEST_ERR_INVALID;
    Shape sh;
    priest_status s = resolve(ctx, pr, -1, sh);
    if (s != PRIEST_OK) return s;
    return make_loaded(ctx, sh, pr->center, pr->vel, pr->semi, 0, false, ctx->stream, out);
}

priest_status priest_unload(priest_ctx *ctx, priest_loaded *h)
{
    if (ctx && ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_loaded(h);
    return PRIEST_OK;
}

priest_status priest_plan_device(priest_ctx *ctx, priest_loaded *h, const double *z_dev, double *out_dev)
{
    if (!ctx || !h || !z_dev || !out_dev) return fail(ctx, PRIEST_ERR_INVALID, "NULL argument");
    h->default_mu = true;
    h->default_cov = true;
    return enqueue_plan(ctx, h, z_dev, out_dev, ctx->stream, ctx->d_status);
}

priest_status priest_project_device(priest_ctx *ctx, priest_loaded *h, int n, const double *xi_dev,
                                    double *lambda_dev, double *xi_bar_dev, double *resid_dev, double *cost_dev)
{
    if (!ctx || !h) return PRIEST_ERR_INVALID;
    if (n < 0 || n > h->sh.N) return fail(ctx, PRIEST_ERR_INVALID, "n exceeds the loaded sample count");
    if (n == 0) return PRIEST_OK;
    if (!xi_dev || !xi_bar_dev || !resid_dev || !cost_dev) return fail(ctx, PRIEST_ERR_INVALID, "NULL pointer");
    priest_status s = enqueue_setup(ctx, h, false, ctx->stream, ctx->d_status);
    if (s != PRIEST_OK) return s;
    return enqueue_project_any(ctx, h, n, 0, xi_dev, nullptr, lambda_dev, lambda_dev, xi_bar_dev, resid_dev,
                               cost_dev, ctx->stream);
}

}  // extern "C"
