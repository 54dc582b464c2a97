// project_kernel.cuh -- fused batched projection (Sec. III-A; Appendix eqs. lagrange,
// comp_alpha .. comp_zeta), the hot path.
//
// One CTA owns S samples of one problem for all K alternating-minimisation
// iterations; the per-sample state (xi_F, lambda, c_F) and the per-point
// residual planes stay in shared memory, next to the problem's basis, KKT
// block inverse and obstacle records.  Per iteration, with c = the free
// coefficients of xi_bar^k:
//   A  trajectory:  pos / vel / acc = base + B_F c                  (eq. parametrized)
//      vel / acc blocks: d = min(1, ||v|| / v_max), residual v (1 - v_max/||v||)_+ (eqs. fv, fa)
//      workspace rows:   residual (x - s_max)_+ - (s_min - x)_+      (eq. bound_con, slack step)
//   B  obstacle blocks, every (point, obstacle) pair: with the scaled offset
//      delta = (x - x_o) / (a, a, b) and rho_s = ||delta||, the closed-form
//      alpha, beta, d (d = max(1, rho_s)) give the target on the ray from the
//      centre, so the residual x - e is Delta (1 - 1/rho_s) when rho_s < 1 and
//      exactly zero otherwise (eq. collision_avoidance_proposed).  Summed over
//      obstacles per point: S_o = sum_j (x - e_j), i.e. F_o^T (F_o xi - e_o) = P^T S_o
//      because F_o stacks the same P once per obstacle.
//   C  g = P^T S_o + Pd^T R_v + Pdd^T R_a  (= F^T (F xi_bar^k - e^{k+1}))
//      lambda^{k+1} = lambda^k - rho g                                 (eq. lag)
//   D  shared-inverse step (eqs. affine_trans / matrix_vec / comp_zeta) on the
//      free coefficients: c <- c + W (xi_F + lambda_F - rho g_F - c),
//      W = (I + rho Q_FF)^-1 (identical to the KKT solution because the
//      boundary coefficients are fixed exactly and rho W Q_FF = I - W).
// After K iterations one more A/B pass evaluates r = ||F xi_bar - e(xi_bar)||
// and c_1 = sum ||acc||^2 (Alg. 1 residual and cost).
#pragma once

#include <algorithm>

#include "priest_internal.cuh"

namespace priest {
namespace detail {

constexpr unsigned kFull = 0xffffffffu;

// Shared-memory layout in Real units: the problem tables first (same layout
// as in global memory, so they are copied as one block), then the state.
// Coefficient rows (xi_F, c) use the padded stride nf_padded(nf).
struct SmemLayout {
    TableLayout tab;
    size_t xi, lam, c, pos, rv, ra, rb, part, total;
};

__host__ __device__ inline SmemLayout smem_layout(int dims, int nv, int nf, int n_p, int n_obs, int S,
                                                  int C, int use_bounds)
{
    SmemLayout L;
    L.tab = table_layout(dims, nv, nf, n_p, n_obs);
    const int nfp = nf_padded(nf);
    size_t o = L.tab.total;
    const size_t PS = size_t(S) * n_p;
    L.xi = o;
    o = align8(o + size_t(S) * dims * nfp);
    L.lam = o;
    o = align8(o + size_t(S) * dims * nv);
    L.c = o;
    o = align8(o + size_t(S) * dims * nfp);
    L.pos = o;
    o = align8(o + dims * PS);
    L.rv = o;
    o = align8(o + dims * PS);
    L.ra = o;
    o = align8(o + dims * PS);
    L.rb = o;
    o = align8(o + (use_bounds ? dims * PS : 0));
    L.part = o;
    o = align8(o + size_t(C) * dims * PS);
    L.total = o;
    return L;
}

// FP32 pair records of the packed obstacle loop, placed after the main layout
// (FP32 kernels only).  Obstacles are taken two at a time so one f32x2 FMA
// evaluates a point against both; every obstacle chunk holds the same number
// of pairs (short chunks are padded with records that never test positive),
// so all lanes of a warp run the same trip counts.
//   static pair (2-D, 8 floats):  {m2x_j, m2x_j', m2y_j, m2y_j'} {nthr_j, nthr_j', 0, 0}
//   static pair (3-D, 12 floats): {m2x, m2x', m2y, m2y'} {m2z, m2z', kap, kap'} {nthr, nthr', 0, 0}
//   moving pair (2-D, 12 floats): {ia, ia', nox, nox'} {noy, noy', nvx, nvx'} {nvy, nvy', 0, 0}
//   moving pair (3-D, 16 floats): {ia, ia', ib, ib'} {nox, nox', noy, noy'} {noz, noz', nvx, nvx'}
//                                 {nvy, nvy', nvz, nvz'}
// with m2 = -2 o, nthr = -thr of the pre-filter, (ia, ib) = 1 / (a, b), no = -o / (a, b),
// nv = -v / (a, b) (the obstacle records' fields).
struct PairLayout {
    int pcs, pcm;      // static / moving pairs per chunk
    size_t st, mv;     // offsets (Real units) of the static / moving pair records
    size_t total;
};

__host__ __device__ inline int pair_rec_static(int dims) { return dims == 2 ? 8 : 12; }
__host__ __device__ inline int pair_rec_moving(int dims) { return dims == 2 ? 12 : 16; }

__host__ __device__ inline PairLayout pair_layout(int dims, int n_obs, int n_static, int C, size_t base)
{
    PairLayout P;
    const int n_mov = n_obs - n_static;
    P.pcs = (n_static + 2 * C - 1) / (2 * C);
    P.pcm = (n_mov + 2 * C - 1) / (2 * C);
    P.st = base;
    size_t o = align8(base + size_t(C) * P.pcs * pair_rec_static(dims));
    P.mv = o;
    o = align8(o + size_t(C) * P.pcm * pair_rec_moving(dims));
    P.total = o;
    return P;
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Three-input minimum (one instruction on sm_100 and later).
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

__device__ __forceinline__ void ld4(const float *p, float &a, float &b, float &c, float &d)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = v.x;
    b = v.y;
    c = v.z;
    d = v.w;
}
__device__ __forceinline__ void ld4(const double *p, double &a, double &b, double &c, double &d)
{
    const double2 v0 = reinterpret_cast<const double2 *>(p)[0];
    const double2 v1 = reinterpret_cast<const double2 *>(p)[1];
    a = v0.x;
    b = v0.y;
    c = v1.x;
    d = v1.y;
}

// Barrier of one sample's warp group: a named barrier for groups of two or
// more warps (ids 1..15; id 0 is __syncthreads), a warp barrier otherwise.
__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    if (nthreads == 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Exact contribution of one (point, obstacle) pair given its scaled offset
// (dx, dy, dz) = (x - x_o) / (a, a, b) and q = |offset|^2 < 1: the residual
// x - e = Delta (1 - 1/rho_s) is added to the point's P-row slot, or in the
// final pass its squared norm (Delta = (a dx, a dy, b dz)).  At the centre
// (q = 0) alpha = beta = 0 puts the target at o + (a, 0) (2-D) / o + (0, 0, b).
template <typename Real, int DIMS>
__device__ __forceinline__ void active_pair(Real dx, Real dy, Real dz, Real q, Real a, Real b, bool fin,
                                            Real *slot, int PS)
{
    if (q > Real(0)) {
        const Real rs = rsq(q);
        const Real w = Real(1) - rs;
        if (!fin) {
            slot[0] = fma(a * w, dx, slot[0]);
            slot[PS] = fma(a * w, dy, slot[PS]);
            if (DIMS == 3) slot[2 * PS] = fma(b * w, dz, slot[2 * PS]);
        } else {
            const Real d2 = (DIMS == 3) ? a * a * fma(dx, dx, dy * dy) + b * b * dz * dz : a * a * q;
            slot[0] = fma(w * w, d2, slot[0]);
        }
    } else {
        const Real s = (DIMS == 3) ? b : a;
        if (!fin)
            slot[(DIMS == 3) ? 2 * PS : 0] -= s;
        else
            slot[0] = fma(s, s, slot[0]);
    }
}

// Exact scaled test of the candidates of one static obstacle (pre-filter
// value q < thr) and their residual contributions.
template <typename Real, int DIMS, int R>
__device__ __forceinline__ void static_exact(const Real *o, const Real (&q)[R], Real thr, const Real (&px)[R],
                                             const Real (&py)[R], const Real (&pz)[R], bool fin, Real *slot0,
                                             int PS, unsigned vmask)
{
    Real ia, nox, noy, noz = Real(0), ib = Real(0), a, b = Real(0), d0, d1, d2;
    if constexpr (DIMS == 2) {
        ld4(o, d0, d1, d2, a);
        ld4(o + 4, ia, nox, noy, d0);
    } else {
        ld4(o + 4, d0, a, b, d1);
        ld4(o + 8, ia, nox, noy, noz);
        ld4(o + 12, ib, d0, d1, d2);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (q[r] < thr && ((vmask >> r) & 1u)) {
            const Real dx = fma(px[r], ia, nox), dy = fma(py[r], ia, noy);
            const Real dz = (DIMS == 3) ? fma(pz[r], ib, noz) : Real(0);
            const Real qq = (DIMS == 3) ? fma(dx, dx, fma(dy, dy, dz * dz)) : fma(dx, dx, dy * dy);
            if (qq < Real(1)) active_pair<Real, DIMS>(dx, dy, dz, qq, a, b, fin, slot0 + 32 * r, PS);
        }
    }
}

// OB consecutive static obstacles against the R points of an item: the
// expanded pre-filter |p|^2 - 2 p.o < thr (two FMAs per pair in 2-D, four in
// 3-D) for all of them, one warp vote for the batch, and the exact test only
// for candidates.
template <typename Real, int DIMS, int R, int OB>
__device__ __forceinline__ void static_batch(const Real *o, const Real (&px)[R], const Real (&py)[R],
                                             const Real (&pz)[R], const Real (&pq)[R], const Real (&pzz)[R],
                                             bool fin, Real *slot0, int PS, unsigned vmask)
{
    constexpr int ST = DIMS == 2 ? 12 : 16;
    Real q[OB][R], thr[OB], dmin[OB];
#pragma unroll
    for (int b = 0; b < OB; ++b) {
        const Real *ob = o + b * ST;
        if constexpr (DIMS == 2) {
            Real m2x, m2y, a;
            ld4(ob, m2x, m2y, thr[b], a);
#pragma unroll
            for (int r = 0; r < R; ++r) q[b][r] = fma(px[r], m2x, fma(py[r], m2y, pq[r]));
        } else {
            Real m2x, m2y, m2z, kap, a, bb, pad;
            ld4(ob, m2x, m2y, m2z, thr[b]);
            ld4(ob + 4, kap, a, bb, pad);
#pragma unroll
            for (int r = 0; r < R; ++r)
                q[b][r] = fma(px[r], m2x, fma(py[r], m2y, fma(pz[r], m2z, fma(pzz[r], kap, pq[r]))));
        }
        Real qmin = q[b][0];
#pragma unroll
        for (int r = 1; r < R; ++r) qmin = min(qmin, q[b][r]);
        dmin[b] = qmin - thr[b];
    }
    Real mm = dmin[0];
#pragma unroll
    for (int b = 1; b < OB; ++b) mm = min(mm, dmin[b]);
    if (__any_sync(kFull, mm < Real(0))) {
#pragma unroll
        for (int b = 0; b < OB; ++b)
            if (dmin[b] < Real(0))
                static_exact<Real, DIMS, R>(o + b * ST, q[b], thr[b], px, py, pz, fin, slot0, PS, vmask);
    }
}

// Moving obstacle j: exact scaled test at each point's own time stamp.
template <typename Real, int DIMS, int R>
__device__ __forceinline__ void moving_obstacle(const Real *o, const Real (&px)[R], const Real (&py)[R],
                                                const Real (&pz)[R], const Real (&tt)[R], bool fin, Real *slot0,
                                                int PS, unsigned vmask)
{
    Real ia, nox, noy, noz = Real(0), ib = Real(0), nvx, nvy, nvz = Real(0), a, b = Real(0), d0, d1, d2, d3;
    if constexpr (DIMS == 2) {
        ld4(o, d0, d1, d2, a);
        ld4(o + 4, ia, nox, noy, d3);
        ld4(o + 8, nvx, nvy, d0, d1);
    } else {
        ld4(o + 4, d0, a, b, d1);
        ld4(o + 8, ia, nox, noy, noz);
        ld4(o + 12, ib, nvx, nvy, nvz);
    }
    Real dx[R], dy[R], dz[R], q[R];
    Real qmin = Real(1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        dx[r] = fma(px[r], ia, fma(nvx, tt[r], nox));
        dy[r] = fma(py[r], ia, fma(nvy, tt[r], noy));
        if constexpr (DIMS == 3) {
            dz[r] = fma(pz[r], ib, fma(nvz, tt[r], noz));
            q[r] = fma(dx[r], dx[r], fma(dy[r], dy[r], dz[r] * dz[r]));
        } else {
            dz[r] = Real(0);
            q[r] = fma(dx[r], dx[r], dy[r] * dy[r]);
        }
        qmin = min(qmin, q[r]);
    }
    if (__any_sync(kFull, qmin < Real(1))) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (q[r] < Real(1) && ((vmask >> r) & 1u))
                active_pair<Real, DIMS>(dx[r], dy[r], dz[r], q[r], a, b, fin, slot0 + 32 * r, PS);
    }
}

// ---- packed FP32 obstacle loop ---------------------------------------------
// One item = R points of one sample (time stamps g, g + G, ..., G = ceil(n_p / R))
// against one obstacle chunk.  Each point is held twice in a float2 so one
// f32x2 FMA evaluates it against an obstacle pair; a running three-input
// minimum per point over a batch of pairs and one warp vote per batch find
// the (rare) candidates, which are then recomputed with the same operations
// and tested exactly.

// Exact test of static obstacle j against one point (scalar coordinates),
// from the obstacle record, and its residual contribution.
template <int DIMS>
__device__ __forceinline__ void exact_static_f32(const float *sObs, int j, float x, float y, float z, bool fin,
                                                 float *slot, int PS)
{
    constexpr int ST = DIMS == 2 ? 12 : 16;
    const float *o = sObs + size_t(j) * ST;
    float ia, nox, noy, noz = 0.f, ib = 0.f, a, b = 0.f, d0, d1;
    if constexpr (DIMS == 2) {
        a = o[3];
        ld4(o + 4, ia, nox, noy, d0);
    } else {
        ld4(o + 4, d0, a, b, d1);
        ld4(o + 8, ia, nox, noy, noz);
        ib = o[12];
    }
    const float dx = fmaf(x, ia, nox), dy = fmaf(y, ia, noy);
    const float dz = (DIMS == 3) ? fmaf(z, ib, noz) : 0.f;
    const float q = (DIMS == 3) ? fmaf(dx, dx, fmaf(dy, dy, dz * dz)) : fmaf(dx, dx, dy * dy);
    if (q < 1.f) active_pair<float, DIMS>(dx, dy, dz, q, a, b, fin, slot, PS);
}

// Pre-filter values of one static pair record against one point: the
// expanded test without |p|^2, to be compared with -|p|^2.
template <int DIMS>
__device__ __forceinline__ float2 static_value(const float *q, float2 xd, float2 yd, float2 zd, float2 zzd)
{
    const float4 A = *reinterpret_cast<const float4 *>(q);
    const float4 B = *reinterpret_cast<const float4 *>(q + 4);
    if constexpr (DIMS == 2) {
        return ffma2(xd, make_float2(A.x, A.y), ffma2(yd, make_float2(A.z, A.w), make_float2(B.x, B.y)));
    } else {
        const float4 Cc = *reinterpret_cast<const float4 *>(q + 8);
        return ffma2(xd, make_float2(A.x, A.y),
                     ffma2(yd, make_float2(A.z, A.w),
                           ffma2(zd, make_float2(B.x, B.y), ffma2(zzd, make_float2(B.z, B.w), make_float2(Cc.x, Cc.y)))));
    }
}

// Scaled offsets and squared scaled distance of one moving pair record
// against one point at its time stamp.
template <int DIMS>
__device__ __forceinline__ float2 moving_value(const float *q, float2 xd, float2 yd, float2 zd, float2 td, float2 &dx,
                                               float2 &dy, float2 &dz)
{
    const float4 A = *reinterpret_cast<const float4 *>(q);
    const float4 B = *reinterpret_cast<const float4 *>(q + 4);
    const float4 Cc = *reinterpret_cast<const float4 *>(q + 8);
    if constexpr (DIMS == 2) {
        const float2 ia = make_float2(A.x, A.y);
        dx = ffma2(xd, ia, ffma2(td, make_float2(B.z, B.w), make_float2(A.z, A.w)));
        dy = ffma2(yd, ia, ffma2(td, make_float2(Cc.x, Cc.y), make_float2(B.x, B.y)));
        dz = make_float2(0.f, 0.f);
        return ffma2(dx, dx, fmul2(dy, dy));
    } else {
        const float4 Dd = *reinterpret_cast<const float4 *>(q + 12);
        const float2 ia = make_float2(A.x, A.y), ib = make_float2(A.z, A.w);
        dx = ffma2(xd, ia, ffma2(td, make_float2(Cc.z, Cc.w), make_float2(B.x, B.y)));
        dy = ffma2(yd, ia, ffma2(td, make_float2(Dd.x, Dd.y), make_float2(B.z, B.w)));
        dz = ffma2(zd, ib, ffma2(td, make_float2(Dd.z, Dd.w), make_float2(Cc.x, Cc.y)));
        return ffma2(dx, dx, ffma2(dy, dy, fmul2(dz, dz)));
    }
}

template <int DIMS, int R>
struct PackedPoints {
    float2 x[R], y[R], z[R], zz[R], t[R];
    float npq[R];  // -(x^2 + y^2)
};

// Static pairs [k0, k0 + nb) of a chunk whose first obstacle is j0: the
// candidates of the flagged points, tested exactly in obstacle order.
template <int DIMS, int R>
__device__ __forceinline__ void static_rescan(const float *rec, const float *sObs, int k0, int nb, int j0,
                                              const PackedPoints<DIMS, R> &P, const float (&m)[R], bool fin,
                                              float *slot0, int G, int PS)
{
    constexpr int RS = DIMS == 2 ? 8 : 12;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (m[r] < P.npq[r]) {
            for (int b = k0; b < k0 + nb; ++b) {
                const float2 v = static_value<DIMS>(rec + size_t(b) * RS, P.x[r], P.y[r], P.z[r], P.zz[r]);
                if (v.x < P.npq[r])
                    exact_static_f32<DIMS>(sObs, j0 + 2 * b, P.x[r].x, P.y[r].x, P.z[r].x, fin, slot0 + G * r, PS);
                if (v.y < P.npq[r])
                    exact_static_f32<DIMS>(sObs, j0 + 2 * b + 1, P.x[r].x, P.y[r].x, P.z[r].x, fin, slot0 + G * r,
                                           PS);
            }
        }
    }
}

template <int DIMS, int R>
__device__ __forceinline__ void moving_rescan(const float *rec, const float *sObs, int k0, int nb, int j0,
                                              const PackedPoints<DIMS, R> &P, const float (&m)[R], bool fin,
                                              float *slot0, int G, int PS)
{
    constexpr int RM = DIMS == 2 ? 12 : 16;
    constexpr int ST = DIMS == 2 ? 12 : 16;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (m[r] < 1.f) {
            for (int b = k0; b < k0 + nb; ++b) {
                float2 dx, dy, dz;
                const float2 q = moving_value<DIMS>(rec + size_t(b) * RM, P.x[r], P.y[r], P.z[r], P.t[r], dx, dy, dz);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float qh = h ? q.y : q.x;
                    if (qh < 1.f) {
                        const float *o = sObs + size_t(j0 + 2 * b + h) * ST;
                        const float a = (DIMS == 2) ? o[3] : o[5], bb = (DIMS == 2) ? o[3] : o[6];
                        active_pair<float, DIMS>(h ? dx.y : dx.x, h ? dy.y : dy.x, h ? dz.y : dz.x, qh, a, bb, fin,
                                                 slot0 + G * r, PS);
                    }
                }
            }
        }
    }
}

// All static and moving pairs of one chunk against the item's points.  `am`
// is the mask of the warp's lanes that hold an item (all run the same trip
// counts).
template <int DIMS, int R, int NPB>
__device__ __forceinline__ void packed_pairs(const float *srec, const float *mrec, const float *sObs, int pcs,
                                             int pcm, int js0, int jm0, const PackedPoints<DIMS, R> &P, bool fin,
                                             float *slot0, int G, int PS, unsigned am)
{
    constexpr int RS = DIMS == 2 ? 8 : 12;
    constexpr int RM = DIMS == 2 ? 12 : 16;
    int k = 0;
    for (; k + NPB <= pcs; k += NPB) {
        float m[R];
#pragma unroll
        for (int b = 0; b < NPB; ++b) {
            const float *q = srec + size_t(k + b) * RS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 v = static_value<DIMS>(q, P.x[r], P.y[r], P.z[r], P.zz[r]);
                m[r] = (b == 0) ? fminf(v.x, v.y) : fmin3(m[r], v.x, v.y);
            }
        }
        bool f = false;
#pragma unroll
        for (int r = 0; r < R; ++r) f |= m[r] < P.npq[r];
        if (__any_sync(am, f)) static_rescan<DIMS, R>(srec, sObs, k, NPB, js0, P, m, fin, slot0, G, PS);
    }
    if (k < pcs) {
        float m[R];
#pragma unroll
        for (int r = 0; r < R; ++r) m[r] = INFINITY;
        for (int b = k; b < pcs; ++b) {
            const float *q = srec + size_t(b) * RS;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 v = static_value<DIMS>(q, P.x[r], P.y[r], P.z[r], P.zz[r]);
                m[r] = fmin3(m[r], v.x, v.y);
            }
        }
        bool f = false;
#pragma unroll
        for (int r = 0; r < R; ++r) f |= m[r] < P.npq[r];
        if (__any_sync(am, f)) static_rescan<DIMS, R>(srec, sObs, k, pcs - k, js0, P, m, fin, slot0, G, PS);
    }
    // moving obstacles: the batch minimum is the exact squared scaled distance
    constexpr int NPM = 2;
    for (k = 0; k < pcm; k += NPM) {
        const int nb = min(NPM, pcm - k);
        float m[R];
#pragma unroll
        for (int r = 0; r < R; ++r) m[r] = INFINITY;
#pragma unroll
        for (int b = 0; b < NPM; ++b) {
            if (b < nb) {
                const float *q = mrec + size_t(k + b) * RM;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float2 dx, dy, dz;
                    const float2 v = moving_value<DIMS>(q, P.x[r], P.y[r], P.z[r], P.t[r], dx, dy, dz);
                    m[r] = fmin3(m[r], v.x, v.y);
                }
            }
        }
        bool f = false;
#pragma unroll
        for (int r = 0; r < R; ++r) f |= m[r] < 1.f;
        if (__any_sync(am, f)) moving_rescan<DIMS, R>(mrec, sObs, k, nb, jm0, P, m, fin, slot0, G, PS);
    }
}

// NF: free coefficients (0 = runtime); NG: columns of the transposed basis
// product (0 = runtime, <= 16).  Each sample of the CTA is owned by its own
// group of p.WS warps, which runs all K iterations with group barriers only.
// The projection of samples [s0, s0 + S) of one problem by the calling CTA
// (all threads call it; it returns with the CTA converged).
template <typename Real, int DIMS, int R, int THREADS, int NF, int NG>
__device__ void project_body(const ProjParams<Real> &p, int s0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *sm = reinterpret_cast<Real *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int T = THREADS;
    constexpr int NGM = NG > 0 ? NG : kMaxNv;
    constexpr int NFV = (NF + 3) / 4;  // float4 rows of the packed basis (NF > 0)
    const int nv = p.nv, nf = NF > 0 ? NF : p.nf, np_ = p.n_p, S = p.S, C = p.C;
    const int nfp = nf_padded(nf), fbs = fb_stride(nf);
    const int D = DIMS * nv;
    const int S_act = min(S, p.N - s0);
    if (S_act <= 0) return;
    const int PS = S * np_;
    const SmemLayout L = smem_layout(DIMS, nv, nf, np_, p.n_obs, S, C, p.use_bounds);
    const Real *sBasis = sm + L.tab.basis;
    const Real *sFb = sm + L.tab.fb;
    const Real *sBase = sm + L.tab.base;
    const Real *sW = sm + L.tab.W;
    const Real *sObs = sm + L.tab.obs;
    const Real *sT = sm + L.tab.tval;
    const Real *sOrg = sm + L.tab.origin;
    Real *sXi = sm + L.xi;
    Real *sLam = sm + L.lam;
    Real *sC = sm + L.c;
    Real *sPos = sm + L.pos;
    Real *sRV = sm + L.rv;
    Real *sRA = sm + L.ra;
    Real *sRB = sm + L.rb;
    Real *sPart = sm + L.part;
    const Real rho = p.rho, vmax = p.vmax, amax = p.amax;
    const Real vmax2 = vmax * vmax, amax2 = amax * amax;

    // problem tables -> shared memory (16-byte copies; the table size is a
    // multiple of 8 Real)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(p.tab);
        uint4 *dst = reinterpret_cast<uint4 *>(sm);
        const int n16 = int(L.tab.total * sizeof(Real) / 16);
        for (int i = tid; i < n16; i += T) dst[i] = src[i];
    }
    // a1/a2: samples (given, or xi = mu + L z in FP64), xi_bar^0 = Pi_A(xi)
    // (free coefficients copied, boundary ones implied), lambda^0
    for (int e = tid; e < S * DIMS * nfp; e += T) {
        sXi[e] = Real(0);
        sC[e] = Real(0);
    }
    __syncthreads();
    // FP32: obstacle pair records of the packed loop, from the obstacle records
    constexpr bool kPacked = sizeof(Real) == 4;
    const PairLayout PL = pair_layout(DIMS, p.n_obs, p.n_static, C, L.total);
    if constexpr (kPacked) {
        constexpr int ST = DIMS == 2 ? 12 : 16;
        constexpr int RS = DIMS == 2 ? 8 : 12, RM = DIMS == 2 ? 12 : 16;
        const int ns = p.n_static;
        for (int q = tid; q < C * PL.pcs; q += T) {
            const int c = q / PL.pcs, k = q - c * PL.pcs;
            Real *d = sm + PL.st + size_t(q) * RS;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = c * 2 * PL.pcs + 2 * k + h;
                const bool ok = j < ns;
                const Real *o = sObs + size_t(ok ? j : 0) * ST;
                d[h] = ok ? o[0] : Real(0);
                d[2 + h] = ok ? o[1] : Real(0);
                if constexpr (DIMS == 2) {
                    d[4 + h] = ok ? -o[2] : Real(3e38);  // padding: never below -|p|^2
                    d[6 + h] = Real(0);
                } else {
                    d[4 + h] = ok ? o[2] : Real(0);
                    d[6 + h] = ok ? o[4] : Real(0);
                    d[8 + h] = ok ? -o[3] : Real(3e38);
                    d[10 + h] = Real(0);
                }
            }
        }
        for (int q = tid; q < C * PL.pcm; q += T) {
            const int c = q / PL.pcm, k = q - c * PL.pcm;
            Real *d = sm + PL.mv + size_t(q) * RM;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = ns + c * 2 * PL.pcm + 2 * k + h;
                const bool ok = j < p.n_obs;
                const Real *o = sObs + size_t(ok ? j : 0) * ST;
                // padding: scaled offset (4, 4[, 4]) at every time, never active
                if constexpr (DIMS == 2) {
                    d[h] = ok ? o[4] : Real(0);       // ia
                    d[2 + h] = ok ? o[5] : Real(4);   // nox
                    d[4 + h] = ok ? o[6] : Real(4);   // noy
                    d[6 + h] = ok ? o[8] : Real(0);   // nvx
                    d[8 + h] = ok ? o[9] : Real(0);   // nvy
                    d[10 + h] = Real(0);
                } else {
                    d[h] = ok ? o[8] : Real(0);        // ia
                    d[2 + h] = ok ? o[12] : Real(0);   // ib
                    d[4 + h] = ok ? o[9] : Real(4);    // nox
                    d[6 + h] = ok ? o[10] : Real(4);   // noy
                    d[8 + h] = ok ? o[11] : Real(4);   // noz
                    d[10 + h] = ok ? o[13] : Real(0);  // nvx
                    d[12 + h] = ok ? o[14] : Real(0);  // nvy
                    d[14 + h] = ok ? o[15] : Real(0);  // nvz
                }
            }
        }
    }
    for (int e = tid; e < S_act * D; e += T) {
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
            sXi[(s * DIMS + ax) * nfp + f] = Real(x);
            sC[(s * DIMS + ax) * nfp + f] = Real(x);
        }
        sLam[(s * DIMS + ax) * nv + col] = p.lam_in ? Real(p.lam_in[gi]) : Real(0);
    }
    __syncthreads();

    // ---- from here on each sample's warp group works on its own
    const int WS = p.WS, GT = 32 * WS;
    const int s = warp / WS;
    if (s < S_act) {
    const int lt = tid - s * GT, wl = warp - s * WS, bar = 1 + s;
    const int ps0 = s * np_;
    Real smin[DIMS], smax[DIMS];
#pragma unroll
    for (int ax = 0; ax < DIMS; ++ax) {
        smin[ax] = p.smin[ax] - sOrg[ax];
        smax[ax] = p.smax[ax] - sOrg[ax];
    }
    // obstacle-loop items of the sample: (lane group of R points, obstacle
    // chunk); a warp covers a block of 32 R points, lane l taking points
    // l, l + 32, ... (conflict-free shared memory); static / moving obstacles
    // are split evenly over the chunks
    const int nblk32 = ((np_ + 32 * R - 1) / (32 * R)) * 32;
    const int n_mov = p.n_obs - p.n_static;
    const int Cs_s = (p.n_static + C - 1) / C, Cs_m = (n_mov + C - 1) / C;
    const int items = nblk32 * C;
    // g columns: the free ones only, or all n_v when the multipliers are
    // returned (NG = NF fixes the former at compile time; otherwise the
    // choice is per problem, so one launch may mix both)
    constexpr bool kFreeOnly = NF > 0 && NG == NF;
    const int col_lo = (!kFreeOnly && p.want_lambda) ? 0 : kFree0;
    const int ng = kFreeOnly ? NF : (p.want_lambda ? nv : nf);
    constexpr int ST = DIMS == 2 ? 12 : 16;
    constexpr int OB = 4;
    const Real *cc_s = sC + s * DIMS * nfp;

    for (int k = 0; k <= p.K; ++k) {
        const bool fin = (k == p.K);
        // ---- A: trajectory, velocity / acceleration / workspace residuals
        for (int t = lt; t < np_; t += GT) {
            const int pt = ps0 + t;
            Real pos[DIMS], vel[DIMS], acc[DIMS];
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) {
                pos[ax] = sBase[(0 * DIMS + ax) * np_ + t];
                vel[ax] = sBase[(1 * DIMS + ax) * np_ + t];
                acc[ax] = sBase[(2 * DIMS + ax) * np_ + t];
            }
            if constexpr (NF > 0) {
                Real b[3][4 * NFV], cf[DIMS][4 * NFV];
                const Real *fbt = sFb + size_t(t) * fbs;
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int v = 0; v < NFV; ++v)
                        ld4(fbt + q * nfp + 4 * v, b[q][4 * v], b[q][4 * v + 1], b[q][4 * v + 2], b[q][4 * v + 3]);
#pragma unroll
                for (int ax = 0; ax < DIMS; ++ax)
#pragma unroll
                    for (int v = 0; v < NFV; ++v)
                        ld4(cc_s + ax * nfp + 4 * v, cf[ax][4 * v], cf[ax][4 * v + 1], cf[ax][4 * v + 2],
                            cf[ax][4 * v + 3]);
#pragma unroll
                for (int f = 0; f < NF; ++f)
#pragma unroll
                    for (int ax = 0; ax < DIMS; ++ax) {
                        pos[ax] = fma(b[0][f], cf[ax][f], pos[ax]);
                        vel[ax] = fma(b[1][f], cf[ax][f], vel[ax]);
                        acc[ax] = fma(b[2][f], cf[ax][f], acc[ax]);
                    }
            } else {
                const Real *b0 = sBasis + size_t(0 * np_ + t) * nv + kFree0;
                const Real *b1 = sBasis + size_t(1 * np_ + t) * nv + kFree0;
                const Real *b2 = sBasis + size_t(2 * np_ + t) * nv + kFree0;
                for (int f = 0; f < nf; ++f) {
                    const Real p0 = b0[f], p1 = b1[f], p2 = b2[f];
#pragma unroll
                    for (int ax = 0; ax < DIMS; ++ax) {
                        const Real cfv = cc_s[ax * nfp + f];
                        pos[ax] = fma(p0, cfv, pos[ax]);
                        vel[ax] = fma(p1, cfv, vel[ax]);
                        acc[ax] = fma(p2, cfv, acc[ax]);
                    }
                }
            }
            Real v2 = Real(0), a2 = Real(0);
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) {
                sPos[ax * PS + pt] = pos[ax];
                v2 = fma(vel[ax], vel[ax], v2);
                a2 = fma(acc[ax], acc[ax], a2);
            }
            const Real fv = (v2 > vmax2) ? Real(1) - vmax * rsq(v2) : Real(0);
            const Real fa = (a2 > amax2) ? Real(1) - amax * rsq(a2) : Real(0);
            if (!fin) {
#pragma unroll
                for (int ax = 0; ax < DIMS; ++ax) {
                    sRV[ax * PS + pt] = fv * vel[ax];
                    sRA[ax * PS + pt] = fa * acc[ax];
                }
                if (p.use_bounds) {
#pragma unroll
                    for (int ax = 0; ax < DIMS; ++ax)
                        sRB[ax * PS + pt] = max(Real(0), pos[ax] - smax[ax]) - max(Real(0), smin[ax] - pos[ax]);
                }
            } else {
                Real rq = v2 * fv * fv + a2 * fa * fa;
                if (p.use_bounds) {
#pragma unroll
                    for (int ax = 0; ax < DIMS; ++ax) {
                        const Real hi = max(Real(0), pos[ax] - smax[ax]);
                        const Real lo = max(Real(0), smin[ax] - pos[ax]);
                        rq = fma(hi, hi, fma(lo, lo, rq));
                    }
                }
                sRV[pt] = rq;
                sRA[pt] = point_cost<Real, DIMS>(p.cost, pos, vel, acc, a2);
            }
        }
        group_sync(bar, GT);
        // ---- B: obstacle pairs, per (lane group of R points, obstacle chunk);
        //      each item owns its points' slots of its chunk in sPart
        if constexpr (kPacked) {
            const int G = (np_ + R - 1) / R, itemsP = G * C;
            for (int base = 0; base < itemsP; base += GT) {
                const int it = base + lt;
                const unsigned am = __ballot_sync(kFull, it < itemsP);
                if (it < itemsP) {
                    const int c = it / G, g = it - c * G;
                    Real *slot0 = sPart + size_t(c) * DIMS * PS + ps0 + g;
                    PackedPoints<DIMS, R> P;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int tl = g + G * r;
                        const bool ok = tl < np_;
                        // padding points sit far outside every obstacle
                        const float x = ok ? sPos[ps0 + tl] : 1e15f;
                        const float y = ok ? sPos[PS + ps0 + tl] : 1e15f;
                        const float z = (DIMS == 3 && ok) ? sPos[2 * PS + ps0 + tl] : 0.f;
                        const float tv = ok ? sT[tl] : 0.f;
                        P.x[r] = make_float2(x, x);
                        P.y[r] = make_float2(y, y);
                        P.z[r] = make_float2(z, z);
                        P.zz[r] = make_float2(z * z, z * z);
                        P.t[r] = make_float2(tv, tv);
                        P.npq[r] = -fmaf(x, x, y * y);
                        if (ok) {
                            slot0[G * r] = Real(0);
                            if (!fin) {
                                slot0[PS + G * r] = Real(0);
                                if (DIMS == 3) slot0[2 * PS + G * r] = Real(0);
                            }
                        }
                    }
                    packed_pairs<DIMS, R, 4>(reinterpret_cast<const float *>(sm + PL.st) +
                                                 size_t(c) * PL.pcs * pair_rec_static(DIMS),
                                             reinterpret_cast<const float *>(sm + PL.mv) +
                                                 size_t(c) * PL.pcm * pair_rec_moving(DIMS),
                                             reinterpret_cast<const float *>(sObs), PL.pcs, PL.pcm,
                                             c * 2 * PL.pcs, p.n_static + c * 2 * PL.pcm, P, fin,
                                             reinterpret_cast<float *>(slot0), G, PS, am);
                }
            }
        } else
        for (int it = lt; it < items; it += GT) {
            const int c = it / nblk32, g = it - c * nblk32;
            const int pl = (g >> 5) * (32 * R) + (g & 31);  // first local point of the lane
            Real *slot0 = sPart + size_t(c) * DIMS * PS + ps0 + pl;
            Real px[R], py[R], pz[R], pq[R], pzz[R];
            unsigned vmask = 0u;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int tl = pl + 32 * r;
                const bool ok = tl < np_;
                vmask |= ok ? (1u << r) : 0u;
                // padding points sit far outside every obstacle
                px[r] = ok ? sPos[ps0 + tl] : Real(1e15);
                py[r] = ok ? sPos[PS + ps0 + tl] : Real(1e15);
                pz[r] = (DIMS == 3 && ok) ? sPos[2 * PS + ps0 + tl] : Real(0);
                pzz[r] = pz[r] * pz[r];
                pq[r] = fma(px[r], px[r], py[r] * py[r]);
                if (ok) {
                    slot0[32 * r] = Real(0);
                    if (!fin) {
                        slot0[PS + 32 * r] = Real(0);
                        if (DIMS == 3) slot0[2 * PS + 32 * r] = Real(0);
                    }
                }
            }
            const int js0 = c * Cs_s, js1 = min(js0 + Cs_s, p.n_static);
            int j = js0;
            for (; j + OB <= js1; j += OB)
                static_batch<Real, DIMS, R, OB>(sObs + size_t(j) * ST, px, py, pz, pq, pzz, fin, slot0, PS, vmask);
            for (; j < js1; ++j)
                static_batch<Real, DIMS, R, 1>(sObs + size_t(j) * ST, px, py, pz, pq, pzz, fin, slot0, PS, vmask);
            const int jm0 = p.n_static + c * Cs_m, jm1 = min(jm0 + Cs_m, p.n_obs);
            if (jm0 < jm1) {
                Real tt[R];
#pragma unroll
                for (int r = 0; r < R; ++r) tt[r] = ((vmask >> r) & 1u) ? sT[pl + 32 * r] : Real(0);
                for (int jj = jm0; jj < jm1; ++jj)
                    moving_obstacle<Real, DIMS, R>(sObs + size_t(jj) * ST, px, py, pz, tt, fin, slot0, PS, vmask);
            }
        }
        group_sync(bar, GT);
        if (fin) break;
        // ---- C/D: g = F^T(F xi_bar - e) (eq. lag) with the obstacle chunks and
        //      workspace rows summed on the fly, the multiplier step and the
        //      shared-inverse step (eqs. affine_trans / comp_zeta); one warp per axis
        for (int ax = wl; ax < DIMS; ax += WS) {
            Real acc[NGM];
#pragma unroll
            for (int i = 0; i < NGM; ++i) acc[i] = Real(0);
            for (int t = lane; t < np_; t += 32) {
                const int pp = ps0 + t;
                Real rp = sPart[ax * PS + pp];
                for (int c = 1; c < C; ++c) rp += sPart[(c * DIMS + ax) * PS + pp];
                if (p.use_bounds) rp += sRB[ax * PS + pp];
                const Real rv = sRV[ax * PS + pp], ra = sRA[ax * PS + pp];
                if constexpr (kFreeOnly) {
                    const Real *fbt = sFb + size_t(t) * fbs;
                    Real b[3][4 * NFV];
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int v = 0; v < NFV; ++v)
                            ld4(fbt + q * nfp + 4 * v, b[q][4 * v], b[q][4 * v + 1], b[q][4 * v + 2],
                                b[q][4 * v + 3]);
#pragma unroll
                    for (int i = 0; i < NG; ++i) acc[i] = fma(b[0][i], rp, fma(b[1][i], rv, fma(b[2][i], ra, acc[i])));
                } else {
                    const Real *b0 = sBasis + size_t(t) * nv + col_lo;
                    const Real *b1 = b0 + size_t(np_) * nv;
                    const Real *b2 = b1 + size_t(np_) * nv;
#pragma unroll
                    for (int i = 0; i < NGM; ++i)
                        if (i < ng) acc[i] = fma(b0[i], rp, fma(b1[i], rv, fma(b2[i], ra, acc[i])));
                }
            }
#pragma unroll
            for (int i = 0; i < NGM; ++i) {
                if (kFreeOnly || i < ng) {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) acc[i] += __shfl_xor_sync(kFull, acc[i], off);
                }
            }
            // every lane now holds g for all columns; lane f owns column col_lo + f
            Real *lam = sLam + (s * DIMS + ax) * nv;
            Real *cc = sC + (s * DIMS + ax) * nfp;
            const Real *xi = sXi + (s * DIMS + ax) * nfp;
            Real g = Real(0), du = Real(0);
            const int fl = lane - (kFree0 - col_lo);
#pragma unroll
            for (int i = 0; i < NGM; ++i) {
                if (kFreeOnly || i < ng) {
                    const int ci = col_lo + i, fi = ci - kFree0;
                    if (lane == i) g = acc[i];
                    if (fi >= 0 && fi < nf) {
                        // u_i = xi + lambda^{k+1} - rho g - c on the free column fi
                        const Real ui = xi[fi] + (lam[ci] - rho * acc[i]) - rho * acc[i] - cc[fi];
                        if (fl >= 0 && fl < nf) du = fma(sW[fl * nf + fi], ui, du);
                    }
                }
            }
            __syncwarp();
            if (lane < ng) lam[col_lo + lane] -= rho * g;
            if (fl >= 0 && fl < nf && lane < ng) cc[fl] += du;
            __syncwarp();
        }
        group_sync(bar, GT);
    }

    // ---- a9: r = sqrt(sum of squared residual rows), c_1 = sum ||acc||^2
    if (wl == 0) {
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
    // ---- outputs: xi_bar (boundary coefficients from the closed form), lambda
    for (int d = lt; d < D; d += GT) {
        const int ax = d / nv, cl = d - ax * nv, f = cl - kFree0;
        const size_t gi = size_t(s0 + s) * D + d;
        p.xi_bar[gi] = (f >= 0 && f < nf) ? double(sC[(s * DIMS + ax) * nfp + f]) : p.cB[ax * kMaxNv + cl];
        if (p.lam_out) p.lam_out[gi] = double(sLam[(s * DIMS + ax) * nv + cl]);
    }
    }  // this sample's warp group
    __syncthreads();
}

template <typename Real, int DIMS, int R, int THREADS, int NF, int NG>
__global__ void __launch_bounds__(THREADS, 1) project_kernel(const ProjParams<Real> p)
{
    project_body<Real, DIMS, R, THREADS, NF, NG>(p, blockIdx.x * p.S);
}

// Persistent projection over many problems: CTAs take (problem, first sample)
// items from `items` through an atomic counter until none is left.  Items are
// listed most expensive first.  *next must be zero at launch.
template <typename Real, int DIMS, int R, int THREADS, int NF, int NG>
__global__ void __launch_bounds__(THREADS, 1)
    project_batch_kernel(const ProjParams<Real> *params, const int2 *items, int n_items, int *next)
{
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 w = items[it];
        const ProjParams<Real> p = params[w.x];
        project_body<Real, DIMS, R, THREADS, NF, NG>(p, w.y);
        __syncthreads();
    }
}

}  // namespace detail

template <typename Real, int DIMS, int R, int THREADS, int NF, int NG>
cudaError_t launch_one(const ProjParams<Real> &p, const Tiling &t, cudaStream_t st)
{
    static size_t granted = 0;  // per instantiation
    cudaError_t e = reserve_smem(detail::project_kernel<Real, DIMS, R, THREADS, NF, NG>, t.smem, granted);
    if (e != cudaSuccess) return e;
    const int grid = (p.N + t.S - 1) / t.S;
    detail::project_kernel<Real, DIMS, R, THREADS, NF, NG><<<grid, THREADS, t.smem, st>>>(p);
    return cudaGetLastError();
}

// Free-coefficient and column counts: specialised for degree 10 with the "at
// rest" end (5 free coefficients; 5 columns, or all 11 when the multipliers
// are returned), generic otherwise.
template <typename Real, int DIMS, int R, int THREADS>
cudaError_t launch_variant(const ProjParams<Real> &p, const Tiling &t, cudaStream_t st)
{
    if (p.nf == 5 && !p.want_lambda) return launch_one<Real, DIMS, R, THREADS, 5, 5>(p, t, st);
    if (p.nf == 5 && p.nv == 11) return launch_one<Real, DIMS, R, THREADS, 5, 11>(p, t, st);
    return launch_one<Real, DIMS, R, THREADS, 0, 0>(p, t, st);
}

template <typename Real, int DIMS, int R, int THREADS, int NF, int NG>
cudaError_t launch_batch_one(const ProjParams<Real> *params, const int2 *items, int n_items, int *counter,
                             size_t smem, int grid, cudaStream_t st)
{
    static size_t granted = 0;
    cudaError_t e = reserve_smem(detail::project_batch_kernel<Real, DIMS, R, THREADS, NF, NG>, smem, granted);
    if (e != cudaSuccess) return e;
    if (grid <= 0) {
        int per_sm = 0, dev = 0, n_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, detail::project_batch_kernel<Real, DIMS, R, THREADS, NF, NG>, THREADS, smem);
        grid = std::max(1, per_sm) * n_sm;
    }
    detail::project_batch_kernel<Real, DIMS, R, THREADS, NF, NG><<<grid, THREADS, smem, st>>>(params, items, n_items,
                                                                                             counter);
    return cudaGetLastError();
}

template <typename Real, int DIMS, int R, int THREADS>
cudaError_t launch_variant_batch(const ProjParams<Real> *params, const int2 *items, int n_items, int *counter,
                                 int nf, int nv, int want_lambda, size_t smem, int grid, cudaStream_t st)
{
    if (nf == 5 && !want_lambda)
        return launch_batch_one<Real, DIMS, R, THREADS, 5, 5>(params, items, n_items, counter, smem, grid, st);
    if (nf == 5 && nv == 11)
        return launch_batch_one<Real, DIMS, R, THREADS, 5, 11>(params, items, n_items, counter, smem, grid, st);
    return launch_batch_one<Real, DIMS, R, THREADS, 0, 0>(params, items, n_items, counter, smem, grid, st);
}

}  // namespace priest
