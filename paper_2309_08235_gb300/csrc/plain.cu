// plain.cu -- the plain per-problem FP32 GPU path: the same projection
// (Sec. III-A; Appendix eqs. comp_alpha .. comp_zeta) and the same readings as
// the fused kernel, written the way a direct GPU port of the method's steps
// is written -- one kernel per step, every intermediate in HBM, one problem
// at a time.  It is the comparison point of the fused / batched / serving
// forms, and it is parity-tested against the oracle like them.
//
// Per projection iteration three launches:
//   eval    thread per (sample, 4 time stamps): pos / vel / acc = base + B_F c
//           -> HBM tiles [dims][N][n_p4] (float4 stores);
//   resid   thread per (sample, 4 time stamps): every obstacle (records read
//           from global memory, no pre-filter) -> S_o; velocity /
//           acceleration / workspace residuals -> HBM tiles (float4);
//   update  warp per (sample, axis): g = P^T S_o + Pd^T R_v + Pdd^T R_a
//           (eq. lag), lambda <- lambda - rho g, c <- c + W (xi_F + lambda_F -
//           rho g_F - c) (eqs. affine_trans / comp_zeta).
// After K iterations eval + resid (final form) + reduce give r and c_1.
#include <cuda_runtime.h>

#include "priest_internal.cuh"

namespace priest {
namespace {

constexpr int kPlainThreads = 256;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 ld4f(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4f(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float el(const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ __forceinline__ void set_el(float4 &v, int i, float x)
{
    if (i == 0) v.x = x;
    else if (i == 1) v.y = x;
    else if (i == 2) v.z = x;
    else v.w = x;
}

// a1/a2: xi (given, or mu + L z in FP64), its free coefficients as the
// starting c and xi_F, lambda^0.  Thread per (sample, coefficient).
__global__ void __launch_bounds__(kPlainThreads) plain_init_kernel(const PlainParams p)
{
    const int D = p.dims * p.nv, nfp = nf_padded(p.nf);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.N * D) return;
    const int s = e / D, d = e - s * D, ax = d / p.nv, col = d - ax * p.nv;
    double x;
    if (p.mode == 0) {
        x = p.xi_in[e];
    } else {
        const double *Lrow = p.Lc + size_t(d) * D;
        const double *zi = p.z + size_t(s) * D;
        x = p.mu[d];
        for (int k = 0; k <= d; ++k) x = fma(Lrow[k], zi[k], x);
    }
    const int f = col - kFree0;
    if (f >= 0 && f < p.nf) {
        p.xiF[(s * p.dims + ax) * nfp + f] = float(x);
        p.c[(s * p.dims + ax) * nfp + f] = float(x);
    }
    p.lam[(s * p.dims + ax) * p.nv + col] = p.lam_in ? float(p.lam_in[e]) : 0.f;
}

// Trajectory of every (sample, 4 consecutive time stamps).
__global__ void __launch_bounds__(kPlainThreads) plain_eval_kernel(const PlainParams p)
{
    const int n4 = p.np4 / 4;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.N * n4) return;
    const int s = e / n4, t0 = 4 * (e - s * n4);
    const int nfp = nf_padded(p.nf);
    const float *basis = p.tab + p.lay.basis, *base = p.tab + p.lay.base;
    for (int ax = 0; ax < p.dims; ++ax) {
        const float *c = p.c + (s * p.dims + ax) * nfp;
        float4 out[3];
        for (int q = 0; q < 3; ++q) {
            for (int i = 0; i < 4; ++i) {
                const int t = min(t0 + i, p.n_p - 1);
                float v = base[(q * p.dims + ax) * p.n_p + t];
                const float *b = basis + (size_t(q) * p.n_p + t) * p.nv + kFree0;
                for (int f = 0; f < p.nf; ++f) v = fmaf(b[f], c[f], v);
                set_el(out[q], i, v);
            }
        }
        const size_t o = (size_t(ax) * p.N + s) * p.np4 + t0;
        st4f(p.pos + o, out[0]);
        st4f(p.vel + o, out[1]);
        st4f(p.acc + o, out[2]);
    }
}

// Residual tiles of every (sample, 4 consecutive time stamps).  Final pass
// (fin): per-point squared residual and squared acceleration instead.
__global__ void __launch_bounds__(kPlainThreads) plain_resid_kernel(const PlainParams p, int fin)
{
    const int n4 = p.np4 / 4;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.N * n4) return;
    const int s = e / n4, t0 = 4 * (e - s * n4);
    const int dims = p.dims, st = obs_stride(dims);
    const float *obs = p.tab + p.lay.obs, *tv = p.tab + p.lay.tval, *org = p.tab + p.lay.origin;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 P[3], V[3], A[3], So[3] = {zero4, zero4, zero4}, Rv[3] = {zero4, zero4, zero4}, Ra[3] = {zero4, zero4, zero4};
    for (int ax = 0; ax < dims; ++ax) {
        const size_t o = (size_t(ax) * p.N + s) * p.np4 + t0;
        P[ax] = ld4f(p.pos + o);
        V[ax] = ld4f(p.vel + o);
        A[ax] = ld4f(p.acc + o);
    }
    float4 rq = zero4, a2o = zero4;
    const float vmax2 = p.vmax * p.vmax, amax2 = p.amax * p.amax;
    for (int i = 0; i < 4; ++i) {
        const int t = t0 + i;
        if (t >= p.n_p) break;
        float x[3], v2 = 0.f, a2 = 0.f;
        for (int ax = 0; ax < dims; ++ax) {
            x[ax] = el(P[ax], i);
            v2 = fmaf(el(V[ax], i), el(V[ax], i), v2);
            a2 = fmaf(el(A[ax], i), el(A[ax], i), a2);
        }
        if (dims == 2) x[2] = 0.f;
        const float tt = tv[t];
        float r2 = 0.f, acc_o[3] = {0.f, 0.f, 0.f};
        // obstacles (eq. collision_avoidance_proposed): residual Delta (1 - 1/rho_s) inside
        for (int j = 0; j < p.n_obs; ++j) {
            const float *ob = obs + size_t(j) * st;
            float a, b, ia, ib, dx, dy, dz;
            if (dims == 2) {
                a = ob[3];
                b = a;
                ia = ob[4];
                ib = ia;
                dx = fmaf(x[0], ia, fmaf(ob[8], tt, ob[5]));
                dy = fmaf(x[1], ia, fmaf(ob[9], tt, ob[6]));
                dz = 0.f;
            } else {
                a = ob[5];
                b = ob[6];
                ia = ob[8];
                ib = ob[12];
                dx = fmaf(x[0], ia, fmaf(ob[13], tt, ob[9]));
                dy = fmaf(x[1], ia, fmaf(ob[14], tt, ob[10]));
                dz = fmaf(x[2], ib, fmaf(ob[15], tt, ob[11]));
            }
            const float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (!(q < 1.f)) continue;
            if (q > 0.f) {
                const float w = 1.f - rsqrtf(q);
                if (!fin) {
                    acc_o[0] = fmaf(a * w, dx, acc_o[0]);
                    acc_o[1] = fmaf(a * w, dy, acc_o[1]);
                    acc_o[2] = fmaf(b * w, dz, acc_o[2]);
                } else {
                    const float d2 = a * a * fmaf(dx, dx, dy * dy) + b * b * dz * dz;
                    r2 = fmaf(w * w, d2, r2);
                }
            } else {
                const float sc = (dims == 3) ? b : a;  // centre: target o + (a, 0) / (0, 0, b)
                if (!fin)
                    acc_o[dims == 3 ? 2 : 0] -= sc;
                else
                    r2 = fmaf(sc, sc, r2);
            }
        }
        // velocity / acceleration (eqs. fv, fa) and workspace rows (eq. bound_con)
        const float fv = (v2 > vmax2) ? 1.f - p.vmax * rsqrtf(v2) : 0.f;
        const float fa = (a2 > amax2) ? 1.f - p.amax * rsqrtf(a2) : 0.f;
        if (!fin) {
            for (int ax = 0; ax < dims; ++ax) {
                float so = acc_o[ax];
                if (p.use_bounds) {
                    const float lo = p.smin[ax] - org[ax], hi = p.smax[ax] - org[ax];
                    so += fmaxf(0.f, x[ax] - hi) - fmaxf(0.f, lo - x[ax]);
                }
                set_el(So[ax], i, so);
                set_el(Rv[ax], i, fv * el(V[ax], i));
                set_el(Ra[ax], i, fa * el(A[ax], i));
            }
        } else {
            float r = r2 + v2 * fv * fv + a2 * fa * fa;
            if (p.use_bounds)
                for (int ax = 0; ax < dims; ++ax) {
                    const float lo = p.smin[ax] - org[ax], hi = p.smax[ax] - org[ax];
                    const float h = fmaxf(0.f, x[ax] - hi), l = fmaxf(0.f, lo - x[ax]);
                    r = fmaf(h, h, fmaf(l, l, r));
                }
            set_el(rq, i, r);
            float vv[3] = {0.f, 0.f, 0.f}, aa[3] = {0.f, 0.f, 0.f};
            for (int ax = 0; ax < dims; ++ax) {
                vv[ax] = el(V[ax], i);
                aa[ax] = el(A[ax], i);
            }
            set_el(a2o, i, dims == 2 ? point_cost<float, 2>(p.cost, x, vv, aa, a2)
                                     : point_cost<float, 3>(p.cost, x, vv, aa, a2));
        }
    }
    if (!fin) {
        for (int ax = 0; ax < dims; ++ax) {
            const size_t o = (size_t(ax) * p.N + s) * p.np4 + t0;
            st4f(p.so + o, So[ax]);
            st4f(p.rv + o, Rv[ax]);
            st4f(p.ra + o, Ra[ax]);
        }
    } else {
        const size_t o = size_t(s) * p.np4 + t0;
        st4f(p.so + o, rq);  // final pass: the S_o tile holds the squared residual per point
        st4f(p.rv + o, a2o); // and the R_v tile the squared acceleration
    }
}

// Multiplier and shared-inverse steps; warp per (sample, axis), lane i owns
// column i of g.
__global__ void __launch_bounds__(kPlainThreads) plain_update_kernel(const PlainParams p)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= p.N * p.dims) return;
    const int s = warp / p.dims, ax = warp - s * p.dims;
    const int nv = p.nv, nf = p.nf, nfp = nf_padded(nf);
    const float *basis = p.tab + p.lay.basis, *W = p.tab + p.lay.W;
    const size_t row = (size_t(ax) * p.N + s) * p.np4;
    float g[kMaxNv];
    for (int i = 0; i < nv; ++i) g[i] = 0.f;
    for (int t = lane; t < p.n_p; t += 32) {
        const float so = p.so[row + t], rv = p.rv[row + t], ra = p.ra[row + t];
        const float *b0 = basis + size_t(t) * nv, *b1 = b0 + size_t(p.n_p) * nv, *b2 = b1 + size_t(p.n_p) * nv;
        for (int i = 0; i < nv; ++i) g[i] = fmaf(b0[i], so, fmaf(b1[i], rv, fmaf(b2[i], ra, g[i])));
    }
    for (int i = 0; i < nv; ++i)
        for (int off = 16; off > 0; off >>= 1) g[i] += __shfl_xor_sync(kFull, g[i], off);
    float *lam = p.lam + (s * p.dims + ax) * nv;
    float *c = p.c + (s * p.dims + ax) * nfp;
    const float *xi = p.xiF + (s * p.dims + ax) * nfp;
    float du = 0.f;
    if (lane < nf)
        for (int fi = 0; fi < nf; ++fi) {
            const float gi = g[kFree0 + fi];
            const float ui = xi[fi] + (lam[kFree0 + fi] - p.rho * gi) - p.rho * gi - c[fi];
            du = fmaf(W[lane * nf + fi], ui, du);
        }
    float gl = 0.f;
    for (int i = 0; i < nv; ++i)
        if (lane == i) gl = g[i];
    __syncwarp();
    if (lane < nv) lam[lane] -= p.rho * gl;
    if (lane < nf) c[lane] += du;
}

// r = sqrt(sum of squared residuals), c_1 = sum ||acc||^2 per sample (FP64
// accumulation), and xi_bar / lambda to the FP64 outputs.  Warp per sample.
__global__ void __launch_bounds__(kPlainThreads) plain_reduce_kernel(const PlainParams p)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= p.N) return;
    const int s = warp, D = p.dims * p.nv, nfp = nf_padded(p.nf);
    double r2 = 0.0, c1 = 0.0;
    for (int t = lane; t < p.n_p; t += 32) {
        r2 += double(p.so[size_t(s) * p.np4 + t]);
        c1 += double(p.rv[size_t(s) * p.np4 + t]);
    }
    for (int off = 16; off > 0; off >>= 1) {
        r2 += __shfl_xor_sync(kFull, r2, off);
        c1 += __shfl_xor_sync(kFull, c1, off);
    }
    if (lane == 0) {
        p.r_out[s] = sqrt(r2);
        p.c1_out[s] = c1;
    }
    for (int d = lane; d < D; d += 32) {
        const int ax = d / p.nv, cl = d - ax * p.nv, f = cl - kFree0;
        p.xi_bar[size_t(s) * D + d] = (f >= 0 && f < p.nf) ? double(p.c[(s * p.dims + ax) * nfp + f])
                                                           : p.cB[ax * kMaxNv + cl];
        if (p.lam_out) p.lam_out[size_t(s) * D + d] = double(p.lam[(s * p.dims + ax) * p.nv + cl]);
    }
}

unsigned blocks(long long threads) { return unsigned((threads + kPlainThreads - 1) / kPlainThreads); }

}  // namespace

// Workspace segments start on 256-byte boundaries (64 floats): the tiles are
// accessed as float4.
static inline size_t seg(size_t floats) { return (floats + 63) / 64 * 64; }

size_t plain_work_floats(int dims, int nv, int nf, int n_p, int N)
{
    const size_t np4 = size_t((n_p + 3) / 4) * 4, nfp = nf_padded(nf);
    return 2 * seg(size_t(N) * dims * nfp) + seg(size_t(N) * dims * nv) + 6 * seg(size_t(dims) * N * np4);
}

void plain_carve(PlainParams &p, float *work)
{
    const size_t nfp = nf_padded(p.nf), tile = seg(size_t(p.dims) * p.N * p.np4);
    float *w = work;
    p.c = w;
    w += seg(size_t(p.N) * p.dims * nfp);
    p.xiF = w;
    w += seg(size_t(p.N) * p.dims * nfp);
    p.lam = w;
    w += seg(size_t(p.N) * p.dims * p.nv);
    p.pos = w;
    w += tile;
    p.vel = w;
    w += tile;
    p.acc = w;
    w += tile;
    p.so = w;
    w += tile;
    p.rv = w;
    w += tile;
    p.ra = w;
}

cudaError_t launch_plain_project(const PlainParams &p, cudaStream_t st, int64_t *launches)
{
    if (p.N <= 0) return cudaSuccess;
    const long long pts = (long long)p.N * (p.np4 / 4);
    plain_init_kernel<<<blocks((long long)p.N * p.dims * p.nv), kPlainThreads, 0, st>>>(p);
    int64_t n = 1;
    for (int k = 0; k < p.K; ++k) {
        plain_eval_kernel<<<blocks(pts), kPlainThreads, 0, st>>>(p);
        plain_resid_kernel<<<blocks(pts), kPlainThreads, 0, st>>>(p, 0);
        plain_update_kernel<<<blocks(32LL * p.N * p.dims), kPlainThreads, 0, st>>>(p);
        n += 3;
    }
    plain_eval_kernel<<<blocks(pts), kPlainThreads, 0, st>>>(p);
    plain_resid_kernel<<<blocks(pts), kPlainThreads, 0, st>>>(p, 1);
    plain_reduce_kernel<<<blocks(32LL * p.N), kPlainThreads, 0, st>>>(p);
    n += 3;
    if (launches) *launches += n;
    return cudaGetLastError();
}

}  // namespace priest
