// project.cu -- tile selection and dispatch of the fused projection kernel
// (project_kernel.cuh): a cost model for the default tiling and the list of
// compiled (points per item, CTA size) variants the autotuner times.
#include <algorithm>
#include <cstdlib>
#include <string>
#include <vector>

#include "project_kernel.cuh"

namespace priest {

namespace {

struct Variant {
    int dims, R, threads;
};

template <typename Real>
const std::vector<Variant> &variants()
{
    static const std::vector<Variant> f32 = {{2, 4, 512}, {2, 5, 512}, {2, 8, 512}, {2, 5, 1024},
                                             {3, 4, 512}, {3, 5, 256}, {3, 5, 512}};
    static const std::vector<Variant> f64 = {{2, 4, 256}, {3, 4, 256}};
    return sizeof(Real) == 8 ? f64 : f32;
}

constexpr size_t kSmemCap = 227 * 1024;


}  // namespace

template <typename Real>
size_t project_smem_bytes(const Shape &sh, int S, int C)
{
    size_t total = detail::smem_layout(sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs, S, C, sh.use_bounds).total;
    if (sizeof(Real) == 4) total = detail::pair_layout(sh.dims, sh.n_obs, sh.n_static, C, total).total;
    return total * sizeof(Real);
}

// Lane groups of one sample's obstacle loop: R points per item, spaced by the
// group count (FP32); blocks of 32 lanes x R points (FP64).
template <typename Real>
int lane_groups(int n_p, int R)
{
    if (sizeof(Real) == 4) return (n_p + R - 1) / R;
    return ((n_p + 32 * R - 1) / (32 * R)) * 32;
}

// Samples per CTA for a given group size: enough that the grid covers the SMs
// once, at most one group per ws warps of the CTA, and at most 15 groups when
// groups use named barriers (ids 1..15).
int samples_per_cta(int n_samples, int n_sm, int threads, int ws)
{
    int S = std::max(1, (n_samples + n_sm - 1) / n_sm);
    S = std::min(S, threads / (32 * ws));
    if (ws > 1) S = std::min(S, 15);
    return std::max(1, S);
}

bool pts_allowed();

// Point-owner tiling (FP32, project_pts.cuh): S samples per CTA with R points
// per thread; smem == 0 when the CTA does not fit.
Tiling pts_tiling(const Shape &sh, int S, int R)
{
    Tiling t;
    t.kind = 1;
    t.R = R;
    t.S = S;
    t.C = 1;
    t.ws = 0;
    t.threads = pts_threads(sh, S, R);
    t.smem = pts_smem_bytes(sh, S, R);
    if (t.threads > pts_max_threads(R) || t.smem > kSmemCap || !pts_span_ok(sh, R)) t.smem = 0;
    return t;
}

// Point-owner candidates: two or four points per thread; the samples of one
// wave over the SMs in one CTA (or the most that fit one CTA), half that, and
// one to three samples per CTA (several CTAs per SM, whose phases then
// overlap).
std::vector<Tiling> pts_candidates(const Shape &sh, int n_samples, int n_sm)
{
    std::vector<Tiling> out;
    if (!pts_supported(sh) || !pts_allowed()) return out;
    for (int R : {2, 4}) {
        if (R == 4 && sh.nf != 5) continue;  // compiled for five free coefficients only
        const int tps = (sh.n_p + R - 1) / R;
        const int s_max = std::max(1, pts_max_threads(R) / tps);
        const int s1 = std::min(s_max, std::max(1, (n_samples + n_sm - 1) / n_sm));
        std::vector<int> ss = {s1, (s1 + 1) / 2, 1, 2, 3};
        std::sort(ss.begin(), ss.end());
        ss.erase(std::unique(ss.begin(), ss.end()), ss.end());
        for (int S : ss) {
            if (S > s1) continue;
            const Tiling t = pts_tiling(sh, S, R);
            if (t.smem > 0) out.push_back(t);
        }
    }
    return out;
}

// Default tiling: the largest compiled variant, the largest warp group that
// fits the CTA, and the obstacle chunk count that gives each group's threads
// about one item each, within the shared-memory cap.
template <typename Real>
Tiling choose_tiling(const Shape &sh, int n_samples, int n_sm)
{
    if (sizeof(Real) == 4 && pts_supported(sh) && pts_span_ok(sh, 2) && pts_allowed()) {
        const int tps = (sh.n_p + 1) / 2;
        const int S = std::min(std::max(1, pts_max_threads(2) / tps), std::max(1, (n_samples + n_sm - 1) / n_sm));
        const Tiling p = pts_tiling(sh, S, 2);
        if (p.smem > 0) return p;
    }
    Tiling t;
    t.R = sizeof(Real) == 8 ? 4 : 5;
    t.threads = sizeof(Real) == 8 ? 256 : 512;
    const int S0 = std::max(1, (n_samples + n_sm - 1) / n_sm);
    t.ws = 1;
    while (t.ws < 8 && S0 * 32 * (2 * t.ws) <= t.threads && S0 <= 15) t.ws *= 2;
    int S = samples_per_cta(n_samples, n_sm, t.threads, t.ws);
    while (S > 1 && project_smem_bytes<Real>(sh, S, 1) > kSmemCap) S = std::max(1, S * 3 / 4);
    const int ng = lane_groups<Real>(sh.n_p, t.R);
    int C = std::max(1, (32 * t.ws) / ng);
    C = std::min(C, std::max(1, std::min(16, sh.n_obs)));
    while (C > 1 && project_smem_bytes<Real>(sh, S, C) > kSmemCap) --C;
    t.S = S;
    t.C = C;
    t.smem = project_smem_bytes<Real>(sh, S, C);
    return t;
}

// Candidates for the autotuner: every compiled variant for the dimension,
// every warp-group size that fits, and the chunk counts that keep each
// group's pair loop within two rounds of items, within the shared-memory cap.
template <typename Real>
std::vector<Tiling> tiling_candidates(const Shape &sh, int n_samples, int n_sm)
{
    std::vector<Tiling> out;
    if (sizeof(Real) == 4) out = pts_candidates(sh, n_samples, n_sm);
    for (const Variant &v : variants<Real>()) {
        if (v.dims != sh.dims) continue;
        for (int ws = 1; ws <= 8 && 32 * ws <= v.threads; ws *= 2) {
            int S = samples_per_cta(n_samples, n_sm, v.threads, ws);
            while (S > 1 && project_smem_bytes<Real>(sh, S, 1) > kSmemCap) S = std::max(1, S * 3 / 4);
            const int ng = lane_groups<Real>(sh.n_p, v.R);
            const int cmax = std::max(1, std::min(16, sh.n_obs));
            for (int C = 1; C <= cmax; ++C) {
                const size_t smem = project_smem_bytes<Real>(sh, S, C);
                if (smem > kSmemCap) break;
                const int rounds = (ng * C + 32 * ws - 1) / (32 * ws);
                if (rounds > 2) break;
                Tiling t;
                t.S = S;
                t.C = C;
                t.R = v.R;
                t.threads = v.threads;
                t.ws = ws;
                t.smem = smem;
                out.push_back(t);
            }
        }
    }
    return out;
}

// Point-owner tiling of one problem inside a persistent launch: two points
// per thread, the samples that fill the variant's CTA (at most N).
// Most samples of one problem that fill the persistent variant's CTA.
int pts_batch_samples(const Shape &sh)
{
    int S = std::max(1, pts_batch_threads(sh) / std::max(1, (sh.n_p + 1) / 2));
    while (S > 1 && pts_threads(sh, S, 2) > pts_batch_threads(sh)) --S;
    return S;
}

Tiling pts_batch_tiling(const Shape &sh, int S)
{
    Tiling t;
    t.kind = 1;
    t.R = 2;
    t.S = std::max(1, std::min(S, sh.N));
    t.C = 1;
    t.ws = 0;
    t.threads = pts_batch_threads(sh);
    t.smem = pts_smem_bytes(sh, t.S, 2);
    if (pts_threads(sh, t.S, 2) > t.threads || t.smem > kSmemCap || !pts_span_ok(sh, 2)) t.smem = 0;
    return t;
}

// PRIEST_PROJECT_KERNEL=chunked in the environment keeps the FP32 projection
// on the chunked kernel (comparisons; the autotuner otherwise picks).
bool pts_allowed()
{
    static const bool allowed = [] {
        const char *v = getenv("PRIEST_PROJECT_KERNEL");
        return !(v && std::string(v) == "chunked");
    }();
    return allowed;
}

bool pts_batch_ok(const Shape &sh)
{
    return pts_allowed() && pts_supported(sh) && pts_span_ok(sh, 2) && pts_batch_tiling(sh, 1).smem > 0;
}

template <typename Real>
Tiling batch_tiling(const Shape &sh)
{
    if (sizeof(Real) == 4 && pts_batch_ok(sh)) {
        const Tiling p = pts_batch_tiling(sh, pts_batch_samples(sh));
        if (p.smem > 0) return p;
    }
    Tiling t;
    t.R = sizeof(Real) == 8 ? 4 : 5;
    t.threads = sizeof(Real) == 8 ? 256 : 512;
    t.ws = (sh.dims == 2 && sizeof(Real) == 4) ? 2 : 1;
    t.S = std::max(1, std::min(sh.N, t.threads / (32 * t.ws)));
    if (t.ws > 1) t.S = std::min(t.S, 15);
    const int ng = lane_groups<Real>(sh.n_p, t.R);
    t.C = std::max(1, std::min(std::min(16, std::max(1, sh.n_obs)), (32 * t.ws) / ng));
    while (t.S > 1 && project_smem_bytes<Real>(sh, t.S, t.C) > kSmemCap) t.S = std::max(1, t.S / 2);
    t.smem = project_smem_bytes<Real>(sh, t.S, t.C);
    if (t.smem > kSmemCap) t.smem = 0;
    return t;
}

// Candidates of the batched launch's autotuner: warp-group sizes and chunk
// counts for the batched variant's CTA, within the shared-memory cap.
template <typename Real>
std::vector<Tiling> batch_candidates(const Shape &sh)
{
    std::vector<Tiling> out;
    if (sizeof(Real) == 4 && pts_batch_ok(sh)) {
        const int s_full = pts_batch_samples(sh);
        for (int S : {s_full, (s_full + 1) / 2}) {
            const Tiling t = pts_batch_tiling(sh, S);
            if (t.smem > 0 && (out.empty() || out.back().S != t.S)) out.push_back(t);
        }
    }
    const int threads = sizeof(Real) == 8 ? 256 : 512;
    for (int ws = 1; ws <= 4; ws *= 2) {
        Tiling t;
        t.R = sizeof(Real) == 8 ? 4 : 5;
        t.threads = threads;
        t.ws = ws;
        t.S = std::max(1, std::min(sh.N, threads / (32 * ws)));
        if (ws > 1) t.S = std::min(t.S, 15);
        for (int C = 1; C <= std::min(4, std::max(1, sh.n_obs)); C *= 2) {
            t.C = C;
            int S = t.S;
            while (S > 1 && project_smem_bytes<Real>(sh, S, C) > kSmemCap) S = std::max(1, S / 2);
            Tiling u = t;
            u.S = S;
            u.smem = project_smem_bytes<Real>(sh, S, C);
            if (u.smem <= kSmemCap) out.push_back(u);
        }
    }
    return out;
}

template <typename Real>
cudaError_t launch_project(const ProjParams<Real> &p, const Tiling &t, cudaStream_t st)
{
    if (p.N <= 0) return cudaSuccess;
    if constexpr (sizeof(Real) == 8) {
        if (p.dims == 2) return launch_variant<Real, 2, 4, 256>(p, t, st);
        return launch_variant<Real, 3, 4, 256>(p, t, st);
    } else {
        if (t.kind == 1) return launch_project_pts(p, t, st);
        if (t.S * 32 * t.ws > t.threads) return cudaErrorInvalidValue;
        if (p.dims == 2) {
            if (t.R == 4 && t.threads == 512) return launch_variant<Real, 2, 4, 512>(p, t, st);
            if (t.R == 5 && t.threads == 512) return launch_variant<Real, 2, 5, 512>(p, t, st);
            if (t.R == 8 && t.threads == 512) return launch_variant<Real, 2, 8, 512>(p, t, st);
            if (t.R == 5 && t.threads == 1024) return launch_variant<Real, 2, 5, 1024>(p, t, st);
            return cudaErrorInvalidValue;  // not a compiled variant
        }
        if (t.R == 4 && t.threads == 512) return launch_variant<Real, 3, 4, 512>(p, t, st);
        if (t.R == 5 && t.threads == 256) return launch_variant<Real, 3, 5, 256>(p, t, st);
        if (t.R == 5 && t.threads == 512) return launch_variant<Real, 3, 5, 512>(p, t, st);
        return cudaErrorInvalidValue;
    }
}

// Batched launches use one variant per precision and dimension: 2-D
// (R = 5, 512 threads), 3-D (R = 5, 512 threads), FP64 (R = 4, 256 threads).
template <typename Real>
cudaError_t launch_project_batch(const ProjParams<Real> *params_dev, const int2 *items_dev, int n_items,
                                 int *counter_dev, int dims, int R, int threads, int nf, int nv, int want_lambda,
                                 size_t smem, int grid, cudaStream_t st, int kind)
{
    (void)threads;
    if (n_items <= 0) return cudaSuccess;
    if constexpr (sizeof(Real) == 4) {
        if (kind == 1)
            return launch_project_pts_batch(params_dev, items_dev, n_items, counter_dev, dims, nf, R, want_lambda,
                                            smem, grid, st);
    }
    if constexpr (sizeof(Real) == 8) {
        if (dims == 2)
            return launch_variant_batch<Real, 2, 4, 256>(params_dev, items_dev, n_items, counter_dev, nf, nv,
                                                         want_lambda, smem, grid, st);
        return launch_variant_batch<Real, 3, 4, 256>(params_dev, items_dev, n_items, counter_dev, nf, nv,
                                                     want_lambda, smem, grid, st);
    } else {
        if (dims == 2)
            return launch_variant_batch<Real, 2, 5, 512>(params_dev, items_dev, n_items, counter_dev, nf, nv,
                                                         want_lambda, smem, grid, st);
        return launch_variant_batch<Real, 3, 5, 512>(params_dev, items_dev, n_items, counter_dev, nf, nv,
                                                     want_lambda, smem, grid, st);
    }
}

template cudaError_t launch_project_batch<float>(const ProjParams<float> *, const int2 *, int, int *, int, int, int,
                                                 int, int, int, size_t, int, cudaStream_t, int);
template cudaError_t launch_project_batch<double>(const ProjParams<double> *, const int2 *, int, int *, int, int,
                                                  int, int, int, int, size_t, int, cudaStream_t, int);
template size_t project_smem_bytes<float>(const Shape &, int, int);
template size_t project_smem_bytes<double>(const Shape &, int, int);
template Tiling choose_tiling<float>(const Shape &, int, int);
template Tiling choose_tiling<double>(const Shape &, int, int);
template std::vector<Tiling> tiling_candidates<float>(const Shape &, int, int);
template std::vector<Tiling> tiling_candidates<double>(const Shape &, int, int);
template Tiling batch_tiling<float>(const Shape &);
template Tiling batch_tiling<double>(const Shape &);
template std::vector<Tiling> batch_candidates<float>(const Shape &);
template std::vector<Tiling> batch_candidates<double>(const Shape &);
template cudaError_t launch_project<float>(const ProjParams<float> &, const Tiling &, cudaStream_t);
template cudaError_t launch_project<double>(const ProjParams<double> &, const Tiling &, cudaStream_t);

}  // namespace priest
