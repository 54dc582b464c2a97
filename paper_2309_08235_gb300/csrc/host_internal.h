// host_internal.h -- host-side state of a context and the helpers shared by
// the C ABI (api.cu) and the serving loop (serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "priest_internal.cuh"

// Device buffers of one solve, carved out of one block of device memory.
struct priest_loaded {
    priest::Shape sh;
    void *block = nullptr;  // owned allocation (null when carved from a larger owner)
    size_t bytes = 0;
    double *center = nullptr, *vel = nullptr, *semi = nullptr;
    double *tab64 = nullptr;
    float *tab32 = nullptr;
    double *cB = nullptr;
    double *mu = nullptr, *cov = nullptr, *L = nullptr, *mu_new = nullptr;
    double *xb = nullptr, *r = nullptr, *c1 = nullptr;
    int *elite = nullptr;
    double *out = nullptr;  // D + 4 result doubles, then one double whose first int is a status word
    unsigned *counter = nullptr;
    double *z = nullptr;    // L x N x D (host-driven solves)
    double *xi = nullptr;   // N x D (host-driven projections)
    double *lam = nullptr;  // N x D
    bool default_mu = true, default_cov = true;
    bool shape_ready = false;  // basis and Gram blocks computed for this shape
    int seg_len = 0;           // D-PRIEST: samples per distribution while mu / L hold M of them
};

namespace priest {
struct BatchPlan;
struct HostBatch;
struct Server;
}  // namespace priest

struct priest_ctx {
    priest_config cfg;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, n_sm = 0;
    int *d_status = nullptr;
    std::string err;
    std::atomic<int64_t> launches{0};
    priest_loaded *scratch = nullptr;  // reused by the host-pointer entry points
    // serving loop, started by the first priest_submit
    std::mutex server_mu;
    priest::Server *server = nullptr;
    // batched solves: recorded launch sequences, keyed by the handle / buffer lists
    std::map<std::vector<uintptr_t>, priest::BatchPlan *> batches;
    // tilings chosen by the autotuner, per problem shape
    std::map<std::vector<int>, priest::Tiling> tuned;
    bool tune_cache_loaded = false;
    // workspace of the plain per-problem path (floats)
    float *plain_work = nullptr;
    size_t plain_cap = 0;
    // batched solves through host buffers: resident problems, draws and results
    priest::HostBatch *hbatch = nullptr;
    // descriptors of batched projections: device block, pinned host staging
    // and the event that marks the staging free again
    void *pb_dev = nullptr, *pb_host = nullptr;
    size_t pb_cap = 0;
    cudaEvent_t pb_done = nullptr;
    // instrumentation
    bool profile = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_used, prof_free;
    int last_kind = -1;  // projection kernel of the latest launch (Tiling::kind, 2 = tensor core)
};

namespace priest {
namespace host {

priest_status fail(priest_ctx *ctx, priest_status st, const std::string &msg);
priest_status cuda_fail(priest_ctx *ctx, cudaError_t e, const char *what);

// Resolves a problem against the context defaults and validates it;
// n_override >= 0 gives the sample count of a projection-only call.
priest_status resolve(const priest_config &c, const priest_problem *pr, int n_override, Shape &sh,
                      std::string &why);

// Static obstacles first, moving ones (|v| > 0) after them, stable.
void order_obstacles(const Shape &sh, const double *center, const double *vel, const double *semi,
                     std::vector<double> &c, std::vector<double> &v, std::vector<double> &s, int &n_static);

size_t round_up(size_t x);

// Byte offsets of the buffers of one solve inside its block.
struct Carve {
    size_t center, vel, semi, tab64, tab32, cB, mu, cov, L, mu_new, xb, r, c1, elite, out, counter, z, xi, lam,
        total;
};
Carve carve(const Shape &sh, bool fp32, int z_iters, bool proj_buffers);
// Points h's buffers into `base` laid out as k.
void carve_ptrs(priest_loaded *h, char *base, const Carve &k, bool fp32, int z_iters, bool proj_buffers);

template <typename Real>
ProjParams<Real> proj_params(const priest_ctx *ctx, const priest_loaded *h, const Tiling &t);
SetupParams setup_params(const priest_ctx *ctx, const priest_loaded *h, bool plan_mode, int *status);
CemArgs cem_args(const priest_ctx *ctx, const priest_loaded *h, int *status, double *best_out);

// Fills a result from the host copy of [xi_best, r, c_1, c_aug, index] and mu.
void fill_result(const Shape &sh, const double *host_out, const double *host_mu, priest_result *res);

// Stops the serving loop and frees what it holds (serve.cu).
void server_destroy(priest_ctx *ctx);

}  // namespace host
}  // namespace priest
