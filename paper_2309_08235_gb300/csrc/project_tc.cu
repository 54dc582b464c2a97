// project_tc.cu -- the fused projection with the (point, obstacle) pair
// tests on the 5th-generation tensor core (PRIEST_MIXED_BF16).
//
// The projection's hot loop decides, for every trajectory point p and
// obstacle j, whether p lies inside the obstacle (scaled distance below one,
// eq. collision_avoidance_proposed); only those pairs contribute to the
// residual.  Expanded, that test is a sign of a bilinear form:
//   Q(p, j) = |p_xy - o_xy(t)|^2 + kappa (z - o_z(t))^2 - a^2,  kappa = a^2/b^2,
//           = f(p) . g(j)
// with point features f = [x, y, z, x^2 + y^2, z^2, 1 | t x, t y, t z, t, t^2]
// and obstacle features g = [-2 o_x, -2 o_y, -2 kappa o_z, 1, kappa, |o|_k^2 - a^2 |
// -2 v_x, -2 v_y, -2 kappa v_z, 2 (o.v)_k, |v|_k^2] (the second block only for
// moving obstacles, o(t) = o + v t).  So all pair tests of a CTA are one
// matrix product F G^T: rows = the CTA's trajectory points, columns = the
// obstacles.  It runs as tcgen05.mma with BF16 operands and FP32
// accumulation in tensor memory; every feature is split into BF16 high and
// low parts and the product keeps f_h g_h + f_l g_h + f_h g_l, which leaves an
// error below 2^-16 sum_k |f_k g_k| <= 2^-16 max(1, kappa) (|p| + |o|)^2 + a^2.
// A pair is a candidate when Q < m(p), a per-point margin four times that
// bound; candidates get the exact FP32 test and residual of the FMA kernel.
// Hence the result is the FP32 path's, up to the order of the FP32 sums:
// the BF16 product only decides which pairs are tested exactly.
//
// One CTA of 512 threads (4 warpgroups) owns S samples for all K
// iterations, as the FMA kernel does.  Per iteration:
//   A  trajectory (FMA on the packed basis), velocity / acceleration /
//      workspace residuals, and the BF16 feature row of every point written
//      into the MMA's A operand in shared memory;
//   B  per wave of M-tiles (128 points) that fits tensor memory: one thread
//      issues the MMAs (static obstacles K = 16, moving ones K = 32) and
//      commits them to an mbarrier; each warpgroup then scans its (tile,
//      column segment) units -- thread = TMEM lane = point row -- 16 columns
//      per tcgen05.ld, and tests candidates exactly;
//   C/D  g = F^T (F xi_bar - e), multiplier and shared-inverse steps, warp
//      per (sample, axis), as in the FMA kernel.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "project_kernel.cuh"
#include "tc.cuh"

namespace priest {
namespace {

constexpr int kTcThreads = 512;
constexpr int kTcWarps = kTcThreads / 32;
constexpr uint64_t kTcWaitNs = 2000000000ull;  // MMA completion wait limit (2 s)
constexpr int kMaxSeg = 32;                     // column segments per tile

using detail::kFull;
using detail::ld4;
using detail::rsq;

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// Splits x into BF16 high and low parts.
__device__ __forceinline__ void split(float x, uint16_t &h, uint16_t &l)
{
    h = bf16_bits(x);
    l = bf16_bits(x - bf16_val(h));
}
__device__ __forceinline__ void split_d(double x, uint16_t &h, uint16_t &l)
{
    h = bf16_bits(float(x));
    l = bf16_bits(float(x - double(bf16_val(h))));
}

__device__ __forceinline__ void put(unsigned char *op, int row, int k, int k_total, uint16_t v)
{
    *reinterpret_cast<uint16_t *>(op + tc::offset(row, k, k_total)) = v;
}

// A-operand row of point `row`: block 0 (K 0..15, every obstacle) and, when
// moving obstacles exist, block 1 (K 16..31).  Zero rows give Q = the
// obstacle constant and are never scanned.
template <int DIMS>
__device__ void write_features(unsigned char *sA, int row, int kA, float x, float y, float z, float t)
{
    uint16_t h[5], l[5];
    const float f[5] = {x, y, DIMS == 3 ? z : fmaf(x, x, y * y), DIMS == 3 ? fmaf(x, x, y * y) : 0.f,
                        DIMS == 3 ? z * z : 0.f};
    constexpr int nf = DIMS == 3 ? 5 : 3;
#pragma unroll
    for (int i = 0; i < nf; ++i) split(f[i], h[i], l[i]);
    const uint16_t one = bf16_bits(1.f), zero = 0;
    uint16_t row_k[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) row_k[k] = zero;
    if (DIMS == 2) {
        // f_h . g_h (x, y, r2, 1), f_l . g_h (x, y, r2), f_h . g_l (x, y, 1)
        row_k[0] = h[0]; row_k[1] = h[1]; row_k[2] = h[2]; row_k[3] = one;
        row_k[4] = l[0]; row_k[5] = l[1]; row_k[6] = l[2];
        row_k[7] = h[0]; row_k[8] = h[1]; row_k[9] = one;
    } else {
        // f_h . g_h (x, y, z, r2xy, z2, 1), f_l . g_h (5), f_h . g_l (x, y, z, z2, 1)
#pragma unroll
        for (int i = 0; i < 5; ++i) row_k[i] = h[i];
        row_k[5] = one;
#pragma unroll
        for (int i = 0; i < 5; ++i) row_k[6 + i] = l[i];
        row_k[11] = h[0]; row_k[12] = h[1]; row_k[13] = h[2]; row_k[14] = h[4]; row_k[15] = one;
    }
    if (kA > 16) {
        const float g[5] = {t * x, t * y, DIMS == 3 ? t * z : t, DIMS == 3 ? t : t * t, DIMS == 3 ? t * t : 0.f};
        constexpr int ng = DIMS == 3 ? 5 : 4;
        uint16_t gh[5], gl[5];
#pragma unroll
        for (int i = 0; i < ng; ++i) split(g[i], gh[i], gl[i]);
#pragma unroll
        for (int i = 0; i < ng; ++i) {
            row_k[16 + i] = gh[i];
            row_k[16 + ng + i] = gl[i];
            row_k[16 + 2 * ng + i] = gh[i];
        }
    }
    // 16-byte stores of 8 consecutive K values (one core-matrix row each)
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
        if (kc >= 2 && kA <= 16) break;
        uint4 v;
        v.x = uint32_t(row_k[8 * kc + 0]) | (uint32_t(row_k[8 * kc + 1]) << 16);
        v.y = uint32_t(row_k[8 * kc + 2]) | (uint32_t(row_k[8 * kc + 3]) << 16);
        v.z = uint32_t(row_k[8 * kc + 4]) | (uint32_t(row_k[8 * kc + 5]) << 16);
        v.w = uint32_t(row_k[8 * kc + 6]) | (uint32_t(row_k[8 * kc + 7]) << 16);
        *reinterpret_cast<uint4 *>(sA + tc::offset(row, 8 * kc, kA)) = v;
    }
}

// B-operand rows (obstacles, FP64 features split into BF16 parts): static
// obstacle j in column j of B_s (K = 16); moving obstacle n_static + m in
// column m of B_m (K = 32).  Padding columns hold Q = +1e30-like values.
template <int DIMS>
__device__ void write_obstacles(const TcParams &q, unsigned char *sBs, unsigned char *sBm)
{
    const ProjParams<float> &p = q.p;
    const TcPlan &tp = q.tp;
    const int n_mov = p.n_obs - p.n_static;
    const int total = tp.ns_pad + tp.nm_pad;
    for (int col = threadIdx.x; col < total; col += blockDim.x) {
        const bool mov = col >= tp.ns_pad;
        const int j = mov ? p.n_static + (col - tp.ns_pad) : col;
        const bool valid = mov ? (col - tp.ns_pad) < n_mov : col < p.n_static;
        double g[6] = {0, 0, 0, 0, 0, 1e30};  // padding: Q = +1e30 (never a candidate)
        double w[5] = {0, 0, 0, 0, 0};
        if (valid) {
            const double a = q.semi[2 * j], b = DIMS == 3 ? q.semi[2 * j + 1] : a;
            const double kap = DIMS == 3 ? (a * a) / (b * b) : 1.0;
            double o[3] = {0, 0, 0}, v[3] = {0, 0, 0};
            for (int ax = 0; ax < DIMS; ++ax) {
                o[ax] = q.center[j * DIMS + ax] - q.origin64[ax];
                v[ax] = q.vel ? q.vel[j * DIMS + ax] : 0.0;
            }
            const double c = o[0] * o[0] + o[1] * o[1] + kap * o[2] * o[2] - a * a;
            if (DIMS == 2) {
                g[0] = -2.0 * o[0]; g[1] = -2.0 * o[1]; g[2] = 1.0; g[5] = c;
                w[0] = -2.0 * v[0]; w[1] = -2.0 * v[1];
                w[2] = 2.0 * (o[0] * v[0] + o[1] * v[1]);
                w[3] = v[0] * v[0] + v[1] * v[1];
            } else {
                g[0] = -2.0 * o[0]; g[1] = -2.0 * o[1]; g[2] = -2.0 * kap * o[2]; g[3] = 1.0; g[4] = kap; g[5] = c;
                w[0] = -2.0 * v[0]; w[1] = -2.0 * v[1]; w[2] = -2.0 * kap * v[2];
                w[3] = 2.0 * (o[0] * v[0] + o[1] * v[1] + kap * o[2] * v[2]);
                w[4] = v[0] * v[0] + v[1] * v[1] + kap * v[2] * v[2];
            }
        }
        uint16_t gh[6], gl[6];
        for (int i = 0; i < 6; ++i) split_d(g[i], gh[i], gl[i]);
        uint16_t bk[32];
        for (int k = 0; k < 32; ++k) bk[k] = 0;
        if (DIMS == 2) {
            // pairs with the A row: (x, y, r2, 1 | x_l, y_l, r2_l | x, y, 1)
            bk[0] = gh[0]; bk[1] = gh[1]; bk[2] = gh[2]; bk[3] = gh[5];
            bk[4] = gh[0]; bk[5] = gh[1]; bk[6] = gh[2];
            bk[7] = gl[0]; bk[8] = gl[1]; bk[9] = gl[5];
        } else {
            // (x, y, z, r2xy, z2, 1 | lows of the first five | x, y, z, z2, 1)
            for (int i = 0; i < 5; ++i) bk[i] = gh[i];
            bk[5] = gh[5];
            for (int i = 0; i < 5; ++i) bk[6 + i] = gh[i];
            bk[11] = gl[0]; bk[12] = gl[1]; bk[13] = gl[2]; bk[14] = gl[4]; bk[15] = gl[5];
        }
        if (mov) {
            const int ng = DIMS == 3 ? 5 : 4;
            uint16_t wh[5], wl[5];
            for (int i = 0; i < ng; ++i) split_d(w[i], wh[i], wl[i]);
            for (int i = 0; i < ng; ++i) {
                bk[16 + i] = wh[i];
                bk[16 + ng + i] = wh[i];
                bk[16 + 2 * ng + i] = wl[i];
            }
            for (int k = 0; k < 32; ++k) put(sBm, col - tp.ns_pad, k, 32, bk[k]);
        } else {
            for (int k = 0; k < 16; ++k) put(sBs, col, k, 16, bk[k]);
        }
    }
}

// Exact FP32 test of point (x, y, z, t) against obstacle j (record in
// shared memory) and its residual contribution (same arithmetic as the FMA
// kernel's exact test).
template <int DIMS>
__device__ __forceinline__ void exact_pair(const float *o, float x, float y, float z, float t, bool fin, float &rx,
                                           float &ry, float &rz, float &r2)
{
    float ia, nox, noy, noz = 0.f, ib = 0.f, nvx, nvy, nvz = 0.f, a, b = 0.f, d0, d1, d2, d3;
    if constexpr (DIMS == 2) {
        ld4(o, d0, d1, d2, a);
        ld4(o + 4, ia, nox, noy, d3);
        ld4(o + 8, nvx, nvy, d0, d1);
    } else {
        ld4(o + 4, d0, a, b, d1);
        ld4(o + 8, ia, nox, noy, noz);
        ld4(o + 12, ib, nvx, nvy, nvz);
    }
    const float dx = fmaf(x, ia, fmaf(nvx, t, nox));
    const float dy = fmaf(y, ia, fmaf(nvy, t, noy));
    const float dz = DIMS == 3 ? fmaf(z, ib, fmaf(nvz, t, noz)) : 0.f;
    const float qq = DIMS == 3 ? fmaf(dx, dx, fmaf(dy, dy, dz * dz)) : fmaf(dx, dx, dy * dy);
    if (!(qq < 1.f)) return;
    if (qq > 0.f) {
        const float w = 1.f - rsqrtf(qq);
        if (!fin) {
            rx = fmaf(a * w, dx, rx);
            ry = fmaf(a * w, dy, ry);
            if (DIMS == 3) rz = fmaf(b * w, dz, rz);
        } else {
            const float dd = DIMS == 3 ? a * a * fmaf(dx, dx, dy * dy) + b * b * dz * dz : a * a * qq;
            r2 = fmaf(w * w, dd, r2);
        }
    } else {
        const float s = DIMS == 3 ? b : a;
        if (!fin) {
            if (DIMS == 3)
                rz -= s;
            else
                rx -= s;
        } else {
            r2 = fmaf(s, s, r2);
        }
    }
}

// MMAs of one unit (tile, column segment) into the tensor-memory region at
// column `dcol`: the segment's static columns with K = 16, its moving ones
// with K = 32.  Issued by one thread; the caller commits.
template <int DIMS>
__device__ __forceinline__ void issue_unit(const TcPlan &tp, int tile, int lo, int hi, const unsigned char *sA,
                                           const unsigned char *sBs, const unsigned char *sBm, uint32_t dcol)
{
    const uint32_t a_addr = tc::smem_u32(sA) + uint32_t(tile) * 16u * tc::sbo(tp.kA);
    const int s_lo = lo, s_hi = min(hi, tp.ns_pad);
    if (s_hi > s_lo) {
        const uint64_t ad = tc::smem_desc(a_addr, tc::kLbo, tc::sbo(tp.kA));
        const uint64_t bd = tc::smem_desc(tc::smem_u32(sBs) + uint32_t(s_lo / 8) * tc::sbo(16), tc::kLbo, tc::sbo(16));
        tc::mma_bf16(dcol, ad, bd, tc::idesc_bf16_f32(128, s_hi - s_lo), 0u);
    }
    const int m_lo = max(lo, tp.ns_pad), m_hi = hi;
    if (m_hi > m_lo) {
        const uint32_t id = tc::idesc_bf16_f32(128, m_hi - m_lo);
        for (int ks = 0; ks < 2; ++ks) {
            const uint64_t ad = tc::smem_desc(a_addr + uint32_t(ks) * 2u * tc::kLbo, tc::kLbo, tc::sbo(tp.kA));
            const uint64_t bd = tc::smem_desc(tc::smem_u32(sBm) + uint32_t((m_lo - tp.ns_pad) / 8) * tc::sbo(32) +
                                                  uint32_t(ks) * 2u * tc::kLbo,
                                              tc::kLbo, tc::sbo(32));
            tc::mma_bf16(dcol + uint32_t(m_lo - lo), ad, bd, id, ks ? 1u : 0u);
        }
    }
}

struct CdArgs {
    const float *part, *rb, *rv, *ra;  // this (sample, axis): residual planes, offset to the sample
    const float *basis, *fb, *W;
    float *lam, *c;
    const float *xi;
    int part_stride, C, use_bounds, n_p, nv, nf, nfp, fbs;
    float rho;
};

// g = F^T (F xi_bar - e) (eq. lag) for one (sample, axis), lambda -= rho g,
// and the shared-inverse step c += W (xi_F + lambda_F - rho g_F - c) on the
// free columns.  FREE: the NGT = nf free columns from the packed basis;
// otherwise ng <= NGT columns from col_lo (all n_v when the multipliers are
// returned).  One warp; lanes over time stamps.
template <int NGT, bool FREE>
__device__ __forceinline__ void cd_unit(const CdArgs &a, int col_lo, int ng, int lane)
{
    float acc[NGT];
#pragma unroll
    for (int i = 0; i < NGT; ++i) acc[i] = 0.f;
    for (int t = lane; t < a.n_p; t += 32) {
        float rp = a.part[t];
        for (int c = 1; c < a.C; ++c) rp += a.part[c * a.part_stride + t];
        if (a.use_bounds) rp += a.rb[t];
        const float rv = a.rv[t], ra = a.ra[t];
        if constexpr (FREE) {
            constexpr int NV4 = (NGT + 3) / 4;
            const float *fbt = a.fb + size_t(t) * a.fbs;
            float b[3][4 * NV4];
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int v = 0; v < NV4; ++v)
                    ld4(fbt + q * a.nfp + 4 * v, b[q][4 * v], b[q][4 * v + 1], b[q][4 * v + 2], b[q][4 * v + 3]);
#pragma unroll
            for (int i = 0; i < NGT; ++i) acc[i] = fmaf(b[0][i], rp, fmaf(b[1][i], rv, fmaf(b[2][i], ra, acc[i])));
        } else {
            const float *b0 = a.basis + size_t(t) * a.nv + col_lo;
            const float *b1 = b0 + size_t(a.n_p) * a.nv;
            const float *b2 = b1 + size_t(a.n_p) * a.nv;
#pragma unroll
            for (int i = 0; i < NGT; ++i)
                if (i < ng) acc[i] = fmaf(b0[i], rp, fmaf(b1[i], rv, fmaf(b2[i], ra, acc[i])));
        }
    }
#pragma unroll
    for (int i = 0; i < NGT; ++i)
        if (FREE || i < ng)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[i] += __shfl_xor_sync(kFull, acc[i], off);
    float g = 0.f, du = 0.f;
    const int fl = lane - (kFree0 - col_lo);
#pragma unroll
    for (int i = 0; i < NGT; ++i) {
        if (FREE || i < ng) {
            const int ci = col_lo + i, fi = ci - kFree0;
            if (lane == i) g = acc[i];
            if (fi >= 0 && fi < a.nf) {
                const float ui = a.xi[fi] + (a.lam[ci] - a.rho * acc[i]) - a.rho * acc[i] - a.c[fi];
                if (fl >= 0 && fl < a.nf) du = fmaf(a.W[fl * a.nf + fi], ui, du);
            }
        }
    }
    __syncwarp();
    if (lane < ng) a.lam[col_lo + lane] -= a.rho * g;
    if (fl >= 0 && fl < a.nf && lane < ng) a.c[fl] += du;
    __syncwarp();
}

template <int DIMS, int NF>
__global__ void __launch_bounds__(kTcThreads, 1) project_tc_kernel(const TcParams q)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_mbar[8];  // two per warpgroup
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const ProjParams<float> &p = q.p;
    const TcPlan &tp = q.tp;
    float *sm = reinterpret_cast<float *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, wg = warp >> 2, wq = warp & 3;
    const int s0 = blockIdx.x * p.S;
    const int S_act = min(p.S, p.N - s0);
    const int nv = p.nv, nf = NF > 0 ? NF : p.nf, np_ = p.n_p, S = p.S, C = p.C;
    const int nfp = nf_padded(nf), fbs = fb_stride(nf);
    constexpr int NFV = (NF + 3) / 4;
    const int D = DIMS * nv;
    const int PS = S * np_;
    const int n_pts = S_act * np_;
    const detail::SmemLayout L = detail::smem_layout(DIMS, nv, nf, np_, p.n_obs, S, C, p.use_bounds);
    const float *sBasis = sm + L.tab.basis, *sFb = sm + L.tab.fb, *sBase = sm + L.tab.base, *sW = sm + L.tab.W;
    const float *sObs = sm + L.tab.obs, *sT = sm + L.tab.tval, *sOrg = sm + L.tab.origin;
    float *sXi = sm + L.xi, *sLam = sm + L.lam, *sC = sm + L.c, *sPos = sm + L.pos;
    float *sRV = sm + L.rv, *sRA = sm + L.ra, *sRB = sm + L.rb, *sPart = sm + L.part;
    float *sMarg = reinterpret_cast<float *>(smem_raw + tp.off_marg);
    float *sTrow = sMarg + tp.tiles * 128;  // time of each row's point
    unsigned char *sA = smem_raw + tp.off_a, *sBs = smem_raw + tp.off_bs, *sBm = smem_raw + tp.off_bm;
    const float rho = p.rho, vmax = p.vmax, amax = p.amax, vmax2 = vmax * vmax, amax2 = amax * amax;
    const int st = obs_stride(DIMS);
    const int ncol16 = (tp.ns_pad + tp.nm_pad) / 16;

    // ---- tables, samples, multipliers (as the FMA kernel)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.tab);
        uint4 *dst = reinterpret_cast<uint4 *>(sm);
        const int n16 = int(L.tab.total * sizeof(float) / 16);
        for (int i = tid; i < n16; i += kTcThreads) dst[i] = src[i];
    }
    for (int e = tid; e < S * DIMS * nfp; e += kTcThreads) {
        sXi[e] = 0.f;
        sC[e] = 0.f;
    }
    // zero A rows (padding rows stay zero)
    {
        uint4 *a4 = reinterpret_cast<uint4 *>(sA);
        const int n16 = tp.tiles * 128 * tp.kA * 2 / 16;
        for (int i = tid; i < n16; i += kTcThreads) a4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
    for (int e = tid; e < S_act * D; e += kTcThreads) {
        const int s = e / D, d = e - s * D;
        const int ax = d / nv, col = d - ax * nv;
        const size_t gi = size_t(s0 + s) * D + d;
        double x;
        if (p.mode == 0) {
            x = p.xi_in[gi];
        } else {
            const size_t seg = p.seg_len > 0 ? size_t((s0 + s) / p.seg_len) : 0;  // D-PRIEST distribution
            const double *Lrow = p.Lc + (seg * D + d) * D;
            const double *zi = p.z + size_t(s0 + s) * D;
            x = p.mu[seg * D + d];
            for (int k = 0; k <= d; ++k) x = fma(Lrow[k], zi[k], x);
        }
        const int f = col - kFree0;
        if (f >= 0 && f < nf) {
            sXi[(s * DIMS + ax) * nfp + f] = float(x);
            sC[(s * DIMS + ax) * nfp + f] = float(x);
        }
        sLam[(s * DIMS + ax) * nv + col] = p.lam_in ? float(p.lam_in[gi]) : 0.f;
    }
    // margin scale (non-negative floats, maxima through their bit patterns):
    // O = max_j |o_j| + T |v_j|, a_max, kappa_max
    __shared__ int s_oe, s_am, s_km;
    __shared__ int s_seg[kMaxSeg + 1];  // first 16-column chunk of each segment
    if (tid <= tp.nseg) s_seg[tid] = (tid * ncol16) / tp.nseg;
    for (int i = tid; i < tp.tiles * 128; i += kTcThreads) sTrow[i] = sT[i % np_];
    if (tid == 0) {
        s_oe = 0;
        s_am = 0;
        s_km = __float_as_int(1.f);
        s_abort = 0;
    }
    __syncthreads();
    write_obstacles<DIMS>(q, sBs, sBm);
    for (int j = tid; j < p.n_obs; j += kTcThreads) {
        const float a = float(q.semi[2 * j]), b = DIMS == 3 ? float(q.semi[2 * j + 1]) : a;
        float oo = 0.f, vv = 0.f;
        for (int ax = 0; ax < DIMS; ++ax) {
            const float o = float(q.center[j * DIMS + ax] - q.origin64[ax]);
            const float v = q.vel ? float(q.vel[j * DIMS + ax]) : 0.f;
            oo = fmaf(o, o, oo);
            vv = fmaf(v, v, vv);
        }
        const float oe = (sqrtf(oo) + sT[np_ - 1] * sqrtf(vv)) * 1.001f;
        atomicMax(&s_oe, __float_as_int(oe));
        atomicMax(&s_am, __float_as_int(a));
        atomicMax(&s_km, __float_as_int((a * a) / (b * b) * 1.001f));
    }
    // tensor memory, completion barrier
    if (warp == 0) tc::tmem_alloc(&s_tmem, tp.ncols);
    if (tid < 8) tc::mbar_init(&s_mbar[tid], 1);
    if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = s_tmem;
    // phase-A point walk without divisions: thread tid starts at point tid
    const int s_a0 = tid / np_, t_a0 = tid - (tid / np_) * np_;
    const int step_s = kTcThreads / np_, step_t = kTcThreads - (kTcThreads / np_) * np_;
    const float oeff = __int_as_float(s_oe) + __int_as_float(s_am) + 1.f, kmax = __int_as_float(s_km);
    uint32_t par = 0;  // phase parities of this warpgroup's two barriers
    float smin[DIMS], smax[DIMS];
#pragma unroll
    for (int ax = 0; ax < DIMS; ++ax) {
        smin[ax] = p.smin[ax] - sOrg[ax];
        smax[ax] = p.smax[ax] - sOrg[ax];
    }
    const int col_lo = p.want_lambda ? 0 : kFree0;
    const int ng = p.want_lambda ? nv : nf;

    for (int k = 0; k <= p.K; ++k) {
        const bool fin = (k == p.K);
        // ---- A: trajectory, velocity / acceleration / workspace residuals, features
        for (int i = tid, s = s_a0, t = t_a0; i < n_pts;
             i += kTcThreads, s += step_s, t += step_t, s += (t >= np_), t -= (t >= np_) ? np_ : 0) {
            const float *cc = sC + s * DIMS * nfp;
            float pos[DIMS], vel[DIMS], acc[DIMS];
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) {
                pos[ax] = sBase[(0 * DIMS + ax) * np_ + t];
                vel[ax] = sBase[(1 * DIMS + ax) * np_ + t];
                acc[ax] = sBase[(2 * DIMS + ax) * np_ + t];
            }
            if constexpr (NF > 0) {
                float b[3][4 * NFV], cf[DIMS][4 * NFV];
                const float *fbt = sFb + size_t(t) * fbs;
#pragma unroll
                for (int qq = 0; qq < 3; ++qq)
#pragma unroll
                    for (int v = 0; v < NFV; ++v)
                        ld4(fbt + qq * nfp + 4 * v, b[qq][4 * v], b[qq][4 * v + 1], b[qq][4 * v + 2],
                            b[qq][4 * v + 3]);
#pragma unroll
                for (int ax = 0; ax < DIMS; ++ax)
#pragma unroll
                    for (int v = 0; v < NFV; ++v)
                        ld4(cc + ax * nfp + 4 * v, cf[ax][4 * v], cf[ax][4 * v + 1], cf[ax][4 * v + 2],
                            cf[ax][4 * v + 3]);
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int ax = 0; ax < DIMS; ++ax) {
                        pos[ax] = fmaf(b[0][f], cf[ax][f], pos[ax]);
                        vel[ax] = fmaf(b[1][f], cf[ax][f], vel[ax]);
                        acc[ax] = fmaf(b[2][f], cf[ax][f], acc[ax]);
                    }
            } else {
                const float *b0 = sBasis + size_t(0 * np_ + t) * nv + kFree0;
                const float *b1 = sBasis + size_t(1 * np_ + t) * nv + kFree0;
                const float *b2 = sBasis + size_t(2 * np_ + t) * nv + kFree0;
                for (int f = 0; f < nf; ++f) {
#pragma unroll
                    for (int ax = 0; ax < DIMS; ++ax) {
                        const float cfv = cc[ax * nfp + f];
                        pos[ax] = fmaf(b0[f], cfv, pos[ax]);
                        vel[ax] = fmaf(b1[f], cfv, vel[ax]);
                        acc[ax] = fmaf(b2[f], cfv, acc[ax]);
                    }
                }
            }
            float v2 = 0.f, a2 = 0.f, pp = 0.f;
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) {
                sPos[ax * PS + i] = pos[ax];
                v2 = fmaf(vel[ax], vel[ax], v2);
                a2 = fmaf(acc[ax], acc[ax], a2);
                pp = fmaf(pos[ax], pos[ax], pp);
            }
            const float fv = (v2 > vmax2) ? 1.f - vmax * rsqrtf(v2) : 0.f;
            const float fa = (a2 > amax2) ? 1.f - amax * rsqrtf(a2) : 0.f;
            if (!fin) {
#pragma unroll
                for (int ax = 0; ax < DIMS; ++ax) {
                    sRV[ax * PS + i] = fv * vel[ax];
                    sRA[ax * PS + i] = fa * acc[ax];
                }
                if (p.use_bounds) {
#pragma unroll
                    for (int ax = 0; ax < DIMS; ++ax)
                        sRB[ax * PS + i] = fmaxf(0.f, pos[ax] - smax[ax]) - fmaxf(0.f, smin[ax] - pos[ax]);
                }
            } else {
                float rq = v2 * fv * fv + a2 * fa * fa;
                if (p.use_bounds) {
#pragma unroll
                    for (int ax = 0; ax < DIMS; ++ax) {
                        const float hi = fmaxf(0.f, pos[ax] - smax[ax]);
                        const float lo = fmaxf(0.f, smin[ax] - pos[ax]);
                        rq = fmaf(hi, hi, fmaf(lo, lo, rq));
                    }
                }
                sRV[i] = rq;
                sRA[i] = point_cost<float, DIMS>(p.cost, pos, vel, acc, a2);
            }
            if (ncol16 > 0) {
                write_features<DIMS>(sA, i, tp.kA, pos[0], pos[1], DIMS == 3 ? pos[DIMS - 1] : 0.f, sT[t]);
                const float r = sqrtf(pp) + oeff;
                sMarg[i] = 6.103515625e-05f * kmax * r * r;  // 2^-14 max(1, kappa) (|p| + O + a + 1)^2
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // ---- B: pair tests on the tensor core.  Units (tile, column segment)
        //      go round-robin to the warpgroups; each warpgroup owns two
        //      tensor-memory regions and runs its own pipeline: its leader
        //      issues the MMAs of the next unit into one region while the
        //      warpgroup scans the other.
        if (ncol16 > 0) {
            const int units = tp.tiles * tp.nseg;
            const bool leader = (tid & 127) == 0;
            int it = 0;
            // (tile, segment) of this warpgroup's current and next unit, advanced by 4 units a step
            int tile = wg / tp.nseg, seg = wg - (wg / tp.nseg) * tp.nseg;
            int ntile = tile, nseg_ = seg + 4;
            while (nseg_ >= tp.nseg) {
                nseg_ -= tp.nseg;
                ++ntile;
            }
            if (leader && wg < units) {
                issue_unit<DIMS>(tp, tile, 16 * s_seg[seg], 16 * s_seg[seg + 1], sA, sBs, sBm,
                                 tbase + uint32_t(2 * wg) * tp.regw);
                tc::mma_commit(&s_mbar[2 * wg]);
            }
            for (int u = wg; u < units; u += 4, ++it) {
                const int b = it & 1;
                if (leader && u + 4 < units) {
                    issue_unit<DIMS>(tp, ntile, 16 * s_seg[nseg_], 16 * s_seg[nseg_ + 1], sA, sBs, sBm,
                                     tbase + uint32_t(2 * wg + (b ^ 1)) * tp.regw);
                    tc::mma_commit(&s_mbar[2 * wg + (b ^ 1)]);
                }
                // (warp-uniform outcome: the TMEM loads below are warp-collective)
                const bool ok = __all_sync(kFull, tc::mbar_wait_bounded(&s_mbar[2 * wg + b], (par >> b) & 1u, kTcWaitNs));
                par ^= 1u << b;
                if (!ok) {
                    s_abort = 1;
                    if (q.status) atomicOr(q.status, kStatusTensor);
                }
                tc::fence_after_sync();
                const int c16a = s_seg[seg], c16b = s_seg[seg + 1];
                const int row = 32 * wq + lane, i = tile * 128 + row;
                const bool valid = i < n_pts;
                float x = 0.f, y = 0.f, z = 0.f, tt = 0.f, m = -1.f;
                if (valid) {
                    x = sPos[i];
                    y = sPos[PS + i];
                    if (DIMS == 3) z = sPos[2 * PS + i];
                    tt = sTrow[i];
                    m = sMarg[i];
                }
                float rx = 0.f, ry = 0.f, rz = 0.f, r2 = 0.f;
                const uint32_t taddr = tbase + (uint32_t(32 * wq) << 16) + uint32_t(2 * wg + b) * tp.regw;
                for (int c16 = c16a; c16 < c16b && ok; c16 += 2) {
                    // two 16-column loads in flight, then one wait
                    const bool two = c16 + 1 < c16b;
                    uint32_t v[32];
                    __syncwarp();
                    tc::tmem_ld16(taddr + uint32_t(16 * (c16 - c16a)), *reinterpret_cast<uint32_t(*)[16]>(v));
                    if (two) tc::tmem_ld16(taddr + uint32_t(16 * (c16 + 1 - c16a)), *reinterpret_cast<uint32_t(*)[16]>(v + 16));
                    tc::tmem_wait_ld();
                    if (!two) {
#pragma unroll
                        for (int e = 16; e < 32; ++e) v[e] = 0x7f800000u;  // +inf
                    }
                    float mn[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) mn[e] = fminf(__uint_as_float(v[e]), __uint_as_float(v[e + 16]));
#pragma unroll
                    for (int w2 = 8; w2 > 0; w2 >>= 1)
#pragma unroll
                        for (int e = 0; e < w2; ++e) mn[e] = fminf(mn[e], mn[e + w2]);
                    if (mn[0] < m) {  // rare: candidates (padding columns hold +1e30, invalid rows m = -1)
                        uint32_t mask = 0;
#pragma unroll
                        for (int e = 0; e < 32; ++e) mask |= (__uint_as_float(v[e]) < m ? 1u : 0u) << e;
                        while (mask) {
                            const int e = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const int col = 16 * c16 + e;
                            const int j = col < tp.ns_pad ? col : p.n_static + (col - tp.ns_pad);
                            exact_pair<DIMS>(sObs + size_t(j) * st, x, y, z, tt, fin, rx, ry, rz, r2);
                        }
                    }
                }
                if (valid) {
                    float *slot = sPart + size_t(seg) * DIMS * PS + i;
                    if (!fin) {
                        slot[0] = rx;
                        slot[PS] = ry;
                        if (DIMS == 3) slot[2 * PS] = rz;
                    } else {
                        slot[0] = r2;
                    }
                }
                // the region is free again once all 128 threads have read it
                tc::fence_before_sync();
                asm volatile("bar.sync %0, 128;" ::"r"(1 + wg) : "memory");
                tc::fence_after_sync();
                tile = ntile;
                seg = nseg_;
                nseg_ += 4;
                while (nseg_ >= tp.nseg) {
                    nseg_ -= tp.nseg;
                    ++ntile;
                }
            }
            __syncthreads();
        }
        if (s_abort) break;
        if (ncol16 == 0) {  // no obstacles: empty residual slots
            for (int i = tid; i < n_pts; i += kTcThreads)
                for (int ax = 0; ax < (fin ? 1 : DIMS); ++ax) sPart[ax * PS + i] = 0.f;
            __syncthreads();
        }
        if (s_abort || fin) break;
        // ---- C/D: g = F^T (F xi_bar - e), multiplier and shared-inverse steps;
        //      warp per (sample, axis)
        for (int u = warp; u < S_act * DIMS; u += kTcWarps) {
            const int s = u / DIMS, ax = u - s * DIMS;
            CdArgs ca{sPart + ax * PS + s * np_, sRB + ax * PS + s * np_, sRV + ax * PS + s * np_,
                      sRA + ax * PS + s * np_, sBasis, sFb, sW, sLam + (s * DIMS + ax) * nv,
                      sC + (s * DIMS + ax) * nfp, sXi + (s * DIMS + ax) * nfp, DIMS * PS, C, p.use_bounds, np_, nv,
                      nf, nfp, fbs, rho};
            if constexpr (NF > 0) {
                if (!p.want_lambda) {
                    cd_unit<NF, true>(ca, kFree0, NF, lane);
                    continue;
                }
            }
            cd_unit<kMaxNv, false>(ca, col_lo, ng, lane);
        }
        __syncthreads();
    }

    if (!s_abort) {
        // ---- a9: r and c_1 per sample, warp per sample
        for (int s = warp; s < S_act; s += kTcWarps) {
            const int ps0 = s * np_;
            double r2 = 0.0, c1 = 0.0;
            for (int t = lane; t < np_; t += 32) {
                const int pp = ps0 + t;
                double v = double(sRV[pp]);
                for (int c = 0; c < C; ++c) v += double(sPart[c * DIMS * PS + pp]);
                r2 += v;
                c1 += double(sRA[pp]);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                r2 += __shfl_xor_sync(kFull, r2, off);
                c1 += __shfl_xor_sync(kFull, c1, off);
            }
            if (lane == 0) {
                p.r_out[s0 + s] = sqrt(r2);
                p.c1_out[s0 + s] = c1;
            }
        }
        for (int e = tid; e < S_act * D; e += kTcThreads) {
            const int s = e / D, d = e - s * D;
            const int ax = d / nv, cl = d - ax * nv, f = cl - kFree0;
            const size_t gi = size_t(s0 + s) * D + d;
            p.xi_bar[gi] = (f >= 0 && f < nf) ? double(sC[(s * DIMS + ax) * nfp + f]) : p.cB[ax * kMaxNv + cl];
            if (p.lam_out) p.lam_out[gi] = double(sLam[(s * DIMS + ax) * nv + cl]);
        }
    }
    if (s_abort && (tid & 127) == 0)  // work still in flight
        for (int b = 0; b < 2; ++b) tc::mbar_wait_bounded(&s_mbar[2 * wg + b], (par >> b) & 1u, kTcWaitNs);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, tp.ncols);
}

// dynamic shared memory cap: 227 KB per CTA less the kernel's static part
constexpr size_t kSmemCap = 226 * 1024;

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

// Plan of one tensor-core launch for S samples per CTA; smem == 0 when the
// shape does not fit (too many obstacles for tensor memory, or shared memory).
TcPlan tc_plan(const Shape &sh, int S)
{
    TcPlan tp;
    std::memset(&tp, 0, sizeof(tp));
    const int n_mov = sh.n_obs - sh.n_static;
    tp.ns_pad = (sh.n_static + 15) / 16 * 16;
    tp.nm_pad = (n_mov + 15) / 16 * 16;
    const int ntot = tp.ns_pad + tp.nm_pad;
    tp.kA = tp.nm_pad ? 32 : 16;
    tp.rows = S * sh.n_p;
    tp.tiles = (tp.rows + 127) / 128;
    if (ntot > 1024) return tp;
    // column segments of at most 64 columns; each warpgroup double-buffers
    // one segment in tensor memory (8 regions of regw columns)
    const int ncol16 = ntot / 16;
    tp.nseg = std::max(1, (ncol16 + 3) / 4);
    if (tp.nseg > kMaxSeg) return tp;
    tp.regw = 16 * ((std::max(ncol16, 1) + tp.nseg - 1) / tp.nseg);
    tp.ncols = 32;
    while (tp.ncols < uint32_t(8 * tp.regw)) tp.ncols <<= 1;
    const size_t fl = detail::smem_layout(sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs, S, tp.nseg, sh.use_bounds).total *
                      sizeof(float);
    size_t o = up(fl, 16);
    tp.off_marg = o;  // margins, then row times
    o = up(o + 2 * sizeof(float) * tp.tiles * 128, 1024);
    tp.off_a = o;
    o = up(o + size_t(tp.tiles) * 128 * tp.kA * 2, 1024);
    tp.off_bs = o;
    o = up(o + size_t(tp.ns_pad) * 16 * 2, 1024);
    tp.off_bm = o;
    o = up(o + size_t(tp.nm_pad) * 32 * 2, 16);
    tp.smem = o <= kSmemCap ? o : 0;
    return tp;
}

// Samples per CTA: fill the SMs in as few waves as the shared memory allows.
TcPlan tc_choose(const Shape &sh, int N, int n_sm, int *S_out)
{
    TcPlan best;
    std::memset(&best, 0, sizeof(best));
    double best_cost = 1e300;
    int bestS = 0;
    for (int S = 1; S <= 16; ++S) {
        const TcPlan tp = tc_plan(sh, S);
        if (!tp.smem) continue;
        const int ctas = (N + S - 1) / S;
        const int waves = (ctas + n_sm - 1) / n_sm;
        // per-CTA time ~ the longest warpgroup pipeline (units of regw
        // columns x 128 rows) plus the per-point phases
        const int units = tp.tiles * tp.nseg;
        const double cost = double(waves) * (double((units + 3) / 4) * tp.regw + 0.5 * S * sh.n_p);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = tp;
            bestS = S;
        }
    }
    *S_out = bestS;
    return best;
}

cudaError_t launch_project_tc(const TcParams &q, cudaStream_t st)
{
    if (q.p.N <= 0) return cudaSuccess;
    const int grid = (q.p.N + q.p.S - 1) / q.p.S;
    const bool nf5 = q.p.nf == 5;
    static size_t g2a = 0, g2b = 0, g3a = 0, g3b = 0;
    cudaError_t e;
    if (q.p.dims == 2) {
        if (nf5) {
            e = reserve_smem(project_tc_kernel<2, 5>, q.tp.smem, g2a);
            if (e == cudaSuccess) project_tc_kernel<2, 5><<<grid, kTcThreads, q.tp.smem, st>>>(q);
        } else {
            e = reserve_smem(project_tc_kernel<2, 0>, q.tp.smem, g2b);
            if (e == cudaSuccess) project_tc_kernel<2, 0><<<grid, kTcThreads, q.tp.smem, st>>>(q);
        }
    } else {
        if (nf5) {
            e = reserve_smem(project_tc_kernel<3, 5>, q.tp.smem, g3a);
            if (e == cudaSuccess) project_tc_kernel<3, 5><<<grid, kTcThreads, q.tp.smem, st>>>(q);
        } else {
            e = reserve_smem(project_tc_kernel<3, 0>, q.tp.smem, g3b);
            if (e == cudaSuccess) project_tc_kernel<3, 0><<<grid, kTcThreads, q.tp.smem, st>>>(q);
        }
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace priest
