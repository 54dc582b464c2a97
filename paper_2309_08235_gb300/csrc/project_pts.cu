// project_pts.cu -- launch of the FP32 point-owner projection kernel
// (project_pts.cuh): shared-memory size and dispatch over the compiled
// (dims, points per thread, fixed-column multipliers) variants.
#include <algorithm>

#include "project_pts.cuh"

namespace priest {

size_t pts_smem_bytes(const Shape &sh, int S, int R)
{
    return pts::pts_layout(sh.dims, sh.nf, sh.nv, sh.n_p, sh.n_obs, sh.n_static, S, R).total * sizeof(float);
}

int pts_threads(const Shape &sh, int S, int R) { return ((S * pts::pts_tps(sh.n_p, R) + 31) / 32) * 32; }

int pts_max_threads(int R) { return R <= 2 ? pts::pts_max_threads<2>() : pts::pts_max_threads<4>(); }

int pts_batch_threads(const Shape &sh)
{
    return (sh.dims == 2 && sh.nf == 5) ? pts::pts_batch_threads<2, 2, 5>() : pts::pts_batch_threads<3, 2, 5>();
}

// Degree 10 with the "at rest" end (5 free coefficients per axis), 2-D or
// 3-D; or 2-D with the end position only (7 free coefficients: the paper's
// four boundary rows per axis).
bool pts_supported(const Shape &sh)
{
    return sh.nv == 11 && ((sh.nf == 5 && (sh.dims == 2 || sh.dims == 3)) || (sh.nf == 7 && sh.dims == 2));
}

// Every sample a warp touches needs dims * nf state lanes in that warp.
bool pts_span_ok(const Shape &sh, int R)
{
    return pts::pts_span(pts::pts_tps(sh.n_p, R)) * sh.dims * sh.nf <= 32;
}

namespace {

template <int DIMS, int R, int NF, bool WL>
cudaError_t launch_pts_one(const ProjParams<float> &p, const Tiling &t, cudaStream_t st)
{
    static size_t granted = 0;  // per instantiation
    cudaError_t e = reserve_smem(pts::pts_kernel<DIMS, R, NF, WL>, t.smem, granted);
    if (e != cudaSuccess) return e;
    const int grid = (p.N + t.S - 1) / t.S;
    return launch_pdl(pts::pts_kernel<DIMS, R, NF, WL>, dim3(grid), dim3(t.threads), t.smem, st, p);
}

template <int DIMS, int R, int NF = 5>
cudaError_t launch_pts_wl(const ProjParams<float> &p, const Tiling &t, cudaStream_t st)
{
    return p.want_lambda ? launch_pts_one<DIMS, R, NF, true>(p, t, st) : launch_pts_one<DIMS, R, NF, false>(p, t, st);
}

template <int DIMS, int R, int NF, bool WL>
cudaError_t launch_pts_batch_one(const ProjParams<float> *params, const int2 *items, int n_items, int *counter,
                                 size_t smem, int grid, cudaStream_t st)
{
    static size_t granted = 0;
    auto kern = pts::pts_batch_kernel<DIMS, R, NF, WL>;
    cudaError_t e = reserve_smem(kern, smem, granted);
    if (e != cudaSuccess) return e;
    constexpr int threads = pts::pts_batch_threads<DIMS, R, NF>();
    if (grid <= 0) {
        int per_sm = 0, dev = 0, n_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        grid = std::max(1, per_sm) * n_sm;
    }
    kern<<<grid, threads, smem, st>>>(params, items, n_items, counter);
    return cudaGetLastError();
}

}  // namespace

// Persistent point-owner launch over (problem, first sample) items; every
// problem's p.S * TPS fits the variant's CTA (pts_batch_threads).
cudaError_t launch_project_pts_batch(const ProjParams<float> *params, const int2 *items, int n_items, int *counter,
                                     int dims, int nf, int R, int want_lambda, size_t smem, int grid, cudaStream_t st)
{
    if (n_items <= 0) return cudaSuccess;
    if (dims == 2 && R == 2 && nf == 5)
        return want_lambda ? launch_pts_batch_one<2, 2, 5, true>(params, items, n_items, counter, smem, grid, st)
                           : launch_pts_batch_one<2, 2, 5, false>(params, items, n_items, counter, smem, grid, st);
    if (dims == 2 && R == 2 && nf == 7)
        return want_lambda ? launch_pts_batch_one<2, 2, 7, true>(params, items, n_items, counter, smem, grid, st)
                           : launch_pts_batch_one<2, 2, 7, false>(params, items, n_items, counter, smem, grid, st);
    if (dims == 3 && R == 2 && nf == 5)
        return want_lambda ? launch_pts_batch_one<3, 2, 5, true>(params, items, n_items, counter, smem, grid, st)
                           : launch_pts_batch_one<3, 2, 5, false>(params, items, n_items, counter, smem, grid, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_project_pts(const ProjParams<float> &p, const Tiling &t, cudaStream_t st)
{
    if (p.N <= 0) return cudaSuccess;
    if ((p.nf != 5 && p.nf != 7) || p.nv != 11) return cudaErrorInvalidValue;
    const int tps = pts::pts_tps(p.n_p, t.R);
    if (t.S * tps > t.threads || t.threads % 32 != 0 || t.threads > pts_max_threads(t.R)) return cudaErrorInvalidValue;
    if (pts::pts_span(tps) * p.dims * p.nf > 32) return cudaErrorInvalidValue;
    if (p.dims == 2 && p.nf == 7) {
        if (t.R == 2) return launch_pts_wl<2, 2, 7>(p, t, st);
    } else if (p.dims == 2) {
        if (t.R == 2) return launch_pts_wl<2, 2>(p, t, st);
        if (t.R == 4) return launch_pts_wl<2, 4>(p, t, st);
    } else if (p.dims == 3 && p.nf == 5) {
        if (t.R == 2) return launch_pts_wl<3, 2>(p, t, st);
        if (t.R == 4) return launch_pts_wl<3, 4>(p, t, st);
    }
    return cudaErrorInvalidValue;  // not a compiled variant
}

}  // namespace priest
