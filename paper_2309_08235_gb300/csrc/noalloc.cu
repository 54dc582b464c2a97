// noalloc.cu -- priest_project_noalloc: the projection for callers that may
// not allocate device memory at run time.
//
// Callers such as real-time control loops with a fixed memory budget, code
// that runs inside a pre-provisioned memory pool, or code that must not
// trigger the driver's allocator after start-up cannot call cudaMalloc.  This
// entry point therefore keeps the only data it needs beyond the caller's
// inputs and outputs -- the per-problem tables built by the setup kernel, a
// copy of the obstacle list and a status word -- in one file-scope device
// array of fixed size, and calls no allocating routine.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "priest_internal.cuh"

namespace priest {
namespace {

// Fixed scratch held by every device that loads the library, until exit.
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;  // 1 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device addresses of g_noalloc_scratch, one per device, looked up on the
// first call made with that device current.
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Stable static-first order of the obstacle list, formed on the device from
// the raw copy in the scratch (the kernels test static obstacles four at a
// time and moving ones by their time-dependent offsets): obstacle j goes to
// the count of earlier obstacles of its own kind (plus n_static for a moving
// one).  2-D records keep b = a.
__global__ void order_obstacles_kernel(const double *c_in, const double *v_in, const double *s_in, int n, int dims,
                                       int n_static, double *c, double *v, double *s)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        auto moving = [&](int i) {
            if (!v_in) return false;
            for (int ax = 0; ax < dims; ++ax)
                if (v_in[i * dims + ax] != 0.0) return true;
            return false;
        };
        const bool mj = moving(j);
        int k = mj ? n_static : 0;
        for (int i = 0; i < j; ++i) k += moving(i) == mj ? 1 : 0;
        for (int ax = 0; ax < dims; ++ax) {
            c[k * dims + ax] = c_in[j * dims + ax];
            v[k * dims + ax] = v_in ? v_in[j * dims + ax] : 0.0;
        }
        s[2 * k] = s_in[2 * j];
        s[2 * k + 1] = dims == 3 ? s_in[2 * j + 1] : s_in[2 * j];
    }
}

bool fin(double x) { return std::isfinite(x); }

}  // namespace
}  // namespace priest

using namespace priest;

extern "C" priest_status priest_project_noalloc(const priest_config *cfg, const priest_problem *pr, int n,
                                               const double *xi_dev, double *lambda_dev, double *xi_bar_dev,
                                               double *resid_dev, double *cost_dev, void *cuda_stream)
{
    if (!cfg || !pr) return PRIEST_ERR_INVALID;
    if (n < 0 || n > PRIEST_MAX_SAMPLES) return PRIEST_ERR_INVALID;
    if (n > 0 && (!xi_dev || !xi_bar_dev || !resid_dev || !cost_dev)) return PRIEST_ERR_INVALID;
    if (cfg->precision != PRIEST_FP64_CHECK && cfg->precision != PRIEST_FP32) return PRIEST_ERR_INVALID;
    // ---- shape and validation (host data only)
    Shape sh;
    std::memset(&sh, 0, sizeof(sh));
    sh.dims = pr->dims ? pr->dims : cfg->dims;
    sh.degree = cfg->degree;
    sh.nv = sh.degree + 1;
    sh.n_p = pr->n_p ? pr->n_p : cfg->n_p;
    sh.horizon = pr->horizon > 0 ? pr->horizon : cfg->horizon;
    sh.rho = cfg->rho;
    sh.vmax = pr->vmax > 0 ? pr->vmax : cfg->vmax;
    sh.amax = pr->amax > 0 ? pr->amax : cfg->amax;
    sh.use_bounds = cfg->use_bounds ? 1 : 0;
    sh.bc_mask = pr->bc_final_mask;
    sh.n_obs = pr->n_obs;
    if ((sh.dims != 2 && sh.dims != 3) || sh.degree < 5 || sh.degree > 15 || sh.n_p < 2 ||
        sh.n_p > PRIEST_MAX_NP || !(sh.horizon > 0) || !fin(sh.horizon) || !(sh.rho > 0) || !fin(sh.rho) ||
        !(sh.vmax > 0) || !(sh.amax > 0) || !fin(sh.vmax) || !fin(sh.amax) || cfg->proj_iters < 0 ||
        (sh.bc_mask != 0 && sh.bc_mask != 1 && sh.bc_mask != 3 && sh.bc_mask != 7) || sh.n_obs < 0 ||
        sh.n_obs > PRIEST_MAX_OBS || (sh.n_obs > 0 && (!pr->center || !pr->semi)))
        return PRIEST_ERR_INVALID;
    for (int ax = 0; ax < 3; ++ax) {
        sh.smin[ax] = cfg->smin[ax];
        sh.smax[ax] = cfg->smax[ax];
        for (int q = 0; q < 3; ++q) {
            if (ax < sh.dims && (!fin(pr->b0[ax][q]) || !fin(pr->bf[ax][q]))) return PRIEST_ERR_INVALID;
            sh.b0[ax][q] = pr->b0[ax][q];
            sh.bf[ax][q] = pr->bf[ax][q];
        }
    }
    for (int j = 0; j < sh.n_obs; ++j) {
        const double a = pr->semi[2 * j], b = pr->semi[2 * j + 1];
        if (!(a > 0) || !fin(a) || (sh.dims == 3 && (!(b > 0) || !fin(b)))) return PRIEST_ERR_INVALID;
        for (int ax = 0; ax < sh.dims; ++ax)
            if (!fin(pr->center[j * sh.dims + ax]) || (pr->vel && !fin(pr->vel[j * sh.dims + ax])))
                return PRIEST_ERR_INVALID;
    }
    sh.cost_kind = pr->cost_kind;
    sh.w_acc = pr->w_acc;
    sh.w_curv = pr->w_curv;
    sh.w_path = pr->w_path;
    sh.curv_eps = pr->curv_eps;
    sh.list_delta = list_margin(sh.dims, sh.n_obs, pr->center, pr->semi);
    if ((sh.cost_kind != 0 && sh.cost_kind != 1) ||
        (sh.cost_kind == 1 && (!(sh.w_acc >= 0) || !(sh.w_curv >= 0) || !(sh.w_path >= 0) || !fin(sh.w_acc) ||
                               !fin(sh.w_curv) || !fin(sh.w_path) || !(sh.curv_eps > 0) || !fin(sh.curv_eps))))
        return PRIEST_ERR_INVALID;
    sh.nf = sh.nv - kFree0 - final_fixed(sh.bc_mask);
    sh.D = sh.dims * sh.nv;
    sh.N = n;
    // static obstacles (zero velocity) first, as priest_project orders them
    sh.n_static = 0;
    for (int j = 0; j < sh.n_obs; ++j) {
        bool mv = false;
        for (int ax = 0; ax < sh.dims && pr->vel; ++ax) mv = mv || pr->vel[j * sh.dims + ax] != 0.0;
        sh.n_static += mv ? 0 : 1;
    }
    if (n == 0) return PRIEST_OK;

    // ---- scratch layout inside g_noalloc_scratch
    const bool fp32 = cfg->precision == PRIEST_FP32;
    const TableLayout lay = table_layout(sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs);
    const int nob = sh.n_obs > 0 ? sh.n_obs : 1;
    size_t o = 0;
    const size_t off_status = o;
    o = up256(o + sizeof(int));
    const size_t off_center = o;
    o = up256(o + sizeof(double) * nob * sh.dims);
    const size_t off_vel = o;
    o = up256(o + sizeof(double) * nob * sh.dims);
    const size_t off_semi = o;
    o = up256(o + sizeof(double) * nob * 2);
    const size_t off_raw = o;  // the caller's obstacle list as given: centres, velocities, semi-axes
    o = up256(o + sizeof(double) * nob * (2 * sh.dims + 2));
    const size_t off_cB = o;
    o = up256(o + sizeof(double) * kAuxDoubles);
    const size_t off_tab64 = o;
    o = up256(o + sizeof(double) * lay.total);
    const size_t off_tab32 = o;
    o = up256(o + (fp32 ? sizeof(float) * lay.total32 : 0));
    if (o > kNoAllocScratchBytes) return PRIEST_ERR_BUDGET;  // beyond the fixed 1 MiB scratch

    // ---- the scratch's device address for the current device (first call per device)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PRIEST_ERR_CUDA;
    char *base;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return PRIEST_ERR_CUDA;
            }
            g_scratch_addr[dev] = ptr;
        }
        base = static_cast<char *>(g_scratch_addr[dev]);
    }
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PRIEST_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int *status = reinterpret_cast<int *>(base + off_status);
    double *center = reinterpret_cast<double *>(base + off_center);
    double *vel = reinterpret_cast<double *>(base + off_vel);
    double *semi = reinterpret_cast<double *>(base + off_semi);
    double *raw_c = reinterpret_cast<double *>(base + off_raw);
    double *raw_v = raw_c + size_t(nob) * sh.dims, *raw_s = raw_v + size_t(nob) * sh.dims;

    // ---- inputs into the scratch (raw copy, then the static-first order);
    //      the status word must start at zero
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess && sh.n_obs > 0) {
        e = cudaMemcpyAsync(raw_c, pr->center, sizeof(double) * sh.n_obs * sh.dims, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && pr->vel)
            e = cudaMemcpyAsync(raw_v, pr->vel, sizeof(double) * sh.n_obs * sh.dims, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(raw_s, pr->semi, sizeof(double) * sh.n_obs * 2, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            order_obstacles_kernel<<<(sh.n_obs + 127) / 128, 128, 0, st>>>(raw_c, pr->vel ? raw_v : nullptr, raw_s,
                                                                         sh.n_obs, sh.dims, sh.n_static, center, vel,
                                                                         semi);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return PRIEST_ERR_CUDA;

    // ---- a0 setup into the scratch, then the fused projection
    SetupParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.sh = sh;
    sp.center = center;
    sp.vel = vel;
    sp.semi = semi;
    sp.tab64 = reinterpret_cast<double *>(base + off_tab64);
    sp.tab = fp32 ? static_cast<void *>(base + off_tab32) : static_cast<void *>(sp.tab64);
    sp.real_is_double = fp32 ? 0 : 1;
    sp.cB = reinterpret_cast<double *>(base + off_cB);
    sp.status = status;
    if (launch_setup(sp, st) != cudaSuccess) return PRIEST_ERR_CUDA;

    if (fp32) {
        const Tiling t = choose_tiling<float>(sh, n, n_sm);
        if (t.smem > size_t(227) * 1024) return PRIEST_ERR_INVALID;
        ProjParams<float> p;
        std::memset(&p, 0, sizeof(p));
        p.dims = sh.dims; p.nv = sh.nv; p.nf = sh.nf; p.n_p = sh.n_p; p.n_obs = sh.n_obs;
        p.n_static = sh.n_static; p.use_bounds = sh.use_bounds; p.N = n; p.K = cfg->proj_iters;
        p.S = t.S; p.C = t.C; p.WS = t.ws; p.mode = 0;
        p.rho = float(sh.rho); p.vmax = float(sh.vmax); p.amax = float(sh.amax);
        for (int ax = 0; ax < 3; ++ax) { p.smin[ax] = float(sh.smin[ax]); p.smax[ax] = float(sh.smax[ax]); }
        p.tab = reinterpret_cast<const float *>(base + off_tab32);
        p.lay = lay;
        p.cB = sp.cB;
        p.xi_in = xi_dev; p.lam_in = lambda_dev; p.lam_out = lambda_dev; p.want_lambda = lambda_dev != nullptr;
        p.xi_bar = xi_bar_dev; p.r_out = resid_dev; p.c1_out = cost_dev;
        p.cost = make_cost<float>(sh);
        p.list_delta = float(sh.list_delta);
        p.list_grid = 1;
        if (launch_project<float>(p, t, st) != cudaSuccess) return PRIEST_ERR_CUDA;
    } else {
        const Tiling t = choose_tiling<double>(sh, n, n_sm);
        if (t.smem > size_t(227) * 1024) return PRIEST_ERR_INVALID;
        ProjParams<double> p;
        std::memset(&p, 0, sizeof(p));
        p.dims = sh.dims; p.nv = sh.nv; p.nf = sh.nf; p.n_p = sh.n_p; p.n_obs = sh.n_obs;
        p.n_static = sh.n_static; p.use_bounds = sh.use_bounds; p.N = n; p.K = cfg->proj_iters;
        p.S = t.S; p.C = t.C; p.WS = t.ws; p.mode = 0;
        p.rho = sh.rho; p.vmax = sh.vmax; p.amax = sh.amax;
        for (int ax = 0; ax < 3; ++ax) { p.smin[ax] = sh.smin[ax]; p.smax[ax] = sh.smax[ax]; }
        p.tab = sp.tab64;
        p.lay = lay;
        p.cB = sp.cB;
        p.xi_in = xi_dev; p.lam_in = lambda_dev; p.lam_out = lambda_dev; p.want_lambda = lambda_dev != nullptr;
        p.xi_bar = xi_bar_dev; p.r_out = resid_dev; p.c1_out = cost_dev;
        p.cost = make_cost<double>(sh);
        if (launch_project<double>(p, t, st) != cudaSuccess) return PRIEST_ERR_CUDA;
    }
    // ---- wait, then report the setup kernel's status word
    int hs = 0;
    if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PRIEST_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PRIEST_ERR_CUDA;
    return hs ? PRIEST_ERR_NUMERIC : PRIEST_OK;
}
