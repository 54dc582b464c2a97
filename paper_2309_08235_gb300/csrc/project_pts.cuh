// project_pts.cuh -- FP32 fused projection with point-owning threads (Sec. III-A;
// Appendix eqs. lagrange, comp_alpha .. comp_zeta, lag, affine_trans /
// matrix_vec / comp_zeta), the hot path of the FP32 solver.
//
// Same iteration as project_kernel.cuh (phases A: trajectory and velocity /
// acceleration / workspace residuals, B: obstacle pairs, C: g = F^T (F xi_bar
// - e) and the multiplier step, D: the shared-inverse step), organised so the
// per-point work never leaves registers:
//   * a CTA holds S samples of one problem; thread (s, j) owns the R time
//     stamps j, j + TPS, ..., TPS = ceil(n_p / R), of sample s for all K
//     iterations, with its rows of the free-column basis (P, Pd, Pdd) and of
//     the fixed-coefficient part in registers (loaded once per launch);
//   * phase B tests the thread's points against the obstacles through
//     neighbour lists: each thread keeps, per point, the obstacles within
//     a_j + delta of the point's position at the last rebuild (at most
//     list_cap(dims), in obstacle order, each with the obstacle's offset terms
//     at the point's time) and tests only those exactly.  The CTA
//     rebuilds its lists when one of its points has moved farther than
//     7/8 delta since the last rebuild (always in the first iteration; one
//     vote of the whole CTA, so rebuilds do not hold warps at the barrier
//     of phase C one warp at a time): a point then screens the static
//     obstacles of its cell of the tables' uniform grid (or, without a grid,
//     every static obstacle four at a time from "quad" records, one f32x2 FMA
//     evaluating a point against two obstacles), with thresholds inflated by
//     delta, and every moving obstacle, two at a time by their scaled
//     offsets; the flagged ones are appended to the lists.  An
//     obstacle left out lies at least a_j + delta from the point's rebuild
//     position, so while the point stays within 7/8 delta of it the pair is
//     inactive (its residual row is zero) and skipping it changes nothing; the
//     eighth of delta held back covers the FP32 rounding of the screening.
//     The exact tests run in obstacle order with one FMA per accumulated
//     term on every path, so the sums are bitwise those of testing every
//     obstacle.  A warp whose lists overflowed screens every obstacle
//     and tests its candidates exactly in every iteration until its next
//     rebuild; residuals S_o accumulate in registers;
//   * phase C forms each thread's share of g on the free columns and reduces
//     it over the sample's threads with a segmented warp reduction (a warp may
//     hold the end of one sample and the start of the next; lanes 2i, 2i + 1
//     always share a sample), one partial per (sample, warp) in shared memory,
//     summed in a fixed order;
//   * phase D: every warp holds, for each sample it touches, the free
//     coefficients c, multipliers lambda_F and sample xi_F in registers of
//     dims * nf "state lanes" (one per axis and free column); after the single
//     CTA barrier of the iteration those lanes read their sample's partial
//     sums, apply the multiplier and shared-inverse steps (the W products by
//     warp shuffles), and the warp's threads take the new c by shuffles.
//     Warps sharing a sample repeat the same arithmetic, so they agree.
// One CTA barrier per iteration.  The multipliers of the fixed columns
// (returned only on request) follow from the linearity of eq. lag:
// lambda_B^K = lambda_B^0 - rho P_B^T sum_k r^k, so the per-point residual rows
// are summed over the iterations and reduced once at the end.
#pragma once

#include "project_kernel.cuh"

namespace priest {
namespace pts {

using detail::ffma2;
using detail::fmin3;
using detail::fmul2;
using detail::kFull;

// Shared-memory layout (float units; every block 32-byte aligned).
//   obs   [n_obs][12 | 16]  obstacle records (copied from the tables)
//   srec  [nq][12 | 20]     static quads: {m2x x4} {m2y x4} [{m2z x4} {kap x4}] {nthr x4}
//   mrec  [nm2][12 | 16]    moving pairs (layout of project_kernel.cuh)
//   W     [nf][nf]
//   cd    [S][dims][cds]    free coefficients, each stored twice (c_f, c_f)
//   lam, xi, u [S][dims][8] multipliers, sample (free columns; set-up and output only)
//   part  [2][S][maxw][dims*nv] per-(sample, warp) partial sums, double-buffered by
//                           iteration parity
//   part2 [S][maxw][2]      (doubles) residual / cost partials of the final pass
//   ref   [R][dims][tl]     each thread's point positions at the last list rebuild
//   list  [R][cap][tl]      (float4) each thread's neighbour lists, tl = threads rounded
//                           to 32: per entry the obstacle's scaled offset terms at the
//                           point's time, 2-D (1/a, -o_x(t)/a, -o_y(t)/a, a), 3-D
//                           (1/a, 1/b, -o_x(t)/a, -o_y(t)/a)
//   listz [R][cap][tl]      3-D: -o_z(t)/b
//   listi [R][cap][tl]      3-D (uint16): the obstacle's index (its a, b for active pairs)
//   grid  [gl.smem]         the static-obstacle grid of the tables (header, cell starts,
//                           entries; none below kGridMinStatic static obstacles)
struct PtsLayout {
    int tps, nq, nm2, maxw, cds, tl, cap;
    size_t obs, srec, mrec, W, cd, lam, xi, part, part2, ref, list, listz, listi, grid, gsz, total;
};

// Neighbour-list entries per point.
__host__ __device__ constexpr int list_cap(int dims) { return dims == 2 ? 8 : 6; }

// Threads per sample, rounded up to an even count so the lanes 2i, 2i + 1 of
// a warp always hold the same sample (the paired reduction of phase C).
__host__ __device__ inline int pts_tps(int n_p, int R) { return (((n_p + R - 1) / R) + 1) & ~1; }

// Most samples one warp can touch (its 32 consecutive threads cover TPS-thread
// blocks); every warp keeps the multiplier and coefficient state of each of
// its samples in dims * nf lanes, so dims * nf * span must fit in 32 lanes.
__host__ __device__ inline int pts_span(int tps) { return (31 + tps - 1) / tps + 1; }

__host__ __device__ inline PtsLayout pts_layout(int dims, int nf, int nv, int n_p, int n_obs, int n_static, int S,
                                                int R)
{
    PtsLayout L;
    L.tps = pts_tps(n_p, R);
    L.nq = (n_static + 3) / 4;
    L.nm2 = (n_obs - n_static + 1) / 2;
    L.maxw = (L.tps + 31) / 32 + 1;
    L.cds = ((2 * nf + 3) / 4) * 4;
    size_t o = 0;
    L.obs = o;
    o = align8(o + size_t(n_obs) * (dims == 2 ? 12 : 16));
    L.srec = o;
    o = align8(o + size_t(L.nq) * (dims == 2 ? 12 : 20));
    L.mrec = o;
    o = align8(o + size_t(L.nm2) * (dims == 2 ? 12 : 16));
    L.W = o;
    o = align8(o + size_t(nf) * nf);
    L.cd = o;
    o = align8(o + size_t(S) * dims * L.cds);
    L.lam = o;
    o = align8(o + size_t(S) * dims * 8);
    L.xi = o;
    o = align8(o + size_t(S) * dims * 8);
    L.part = o;
    o = align8(o + size_t(2) * S * L.maxw * dims * nv);
    L.part2 = o;
    o = align8(o + size_t(S) * L.maxw * 4);
    L.tl = ((S * L.tps + 31) / 32) * 32;
    L.ref = o;
    o = align8(o + size_t(R) * dims * L.tl);
    L.cap = list_cap(dims);
    L.list = o;
    o = align8(o + size_t(R) * L.cap * L.tl * 4);
    L.listz = o;
    o = align8(o + (dims == 3 ? size_t(R) * L.cap * L.tl : 0));
    L.listi = o;
    o = align8(o + (dims == 3 ? (size_t(R) * L.cap * L.tl + 1) / 2 : 0));
    L.grid = o;
    L.gsz = n_static >= kGridMinStatic ? grid_layout(n_static).smem : 0;
    o = align8(o + L.gsz);
    L.total = o;
    return L;
}

// Segmented warp sum: lanes [lane, send] of one segment (send = the last lane
// of the calling lane's segment in this warp); afterwards the first lane of
// each segment holds its segment's in-warp sum.
template <typename T>
__device__ __forceinline__ T seg_sum(T v, int lane, int send)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T o = __shfl_down_sync(kFull, v, d);
        if (lane + d <= send) v += o;
    }
    return v;
}

// Residual contribution of an active pair into registers (the arithmetic of
// project_kernel.cuh's active_pair): so[] += Delta (1 - 1/rho_s), or in the
// final pass so[0] += |Delta (1 - 1/rho_s)|^2.
template <int DIMS>
__device__ __forceinline__ void active_add(float dx, float dy, float dz, float q, float a, float b, bool fin,
                                           float (&so)[DIMS])
{
    if (q > 0.f) {
        const float rs = rsqrtf(q);
        const float w = 1.f - rs;
        if (!fin) {
            so[0] = fmaf(a * w, dx, so[0]);
            so[1] = fmaf(a * w, dy, so[1]);
            if constexpr (DIMS == 3) so[DIMS - 1] = fmaf(b * w, dz, so[DIMS - 1]);
        } else {
            // one explicit FMA: every inlined copy rounds the same way
            const float d2 = (DIMS == 3) ? fmaf(b * b * dz, dz, a * a * fmaf(dx, dx, dy * dy)) : a * a * q;
            so[0] = fmaf(w * w, d2, so[0]);
        }
    } else {
        // at the centre the target is o + (a, 0) (2-D) / o + (0, 0, b) (3-D)
        const float s = (DIMS == 3) ? b : a;
        if (!fin)
            so[DIMS == 3 ? DIMS - 1 : 0] -= s;
        else
            so[0] = fmaf(s, s, so[0]);
    }
}

template <int DIMS>
__device__ __forceinline__ void exact_static(const float *sObs, int j, float x, float y, float z, bool fin,
                                             float (&so)[DIMS])
{
    constexpr int ST = DIMS == 2 ? 12 : 16;
    const float *o = sObs + size_t(j) * ST;
    float ia, nox, noy, noz = 0.f, ib = 0.f, a, b = 0.f, d0, d1;
    if constexpr (DIMS == 2) {
        a = o[3];
        detail::ld4(o + 4, ia, nox, noy, d0);
    } else {
        detail::ld4(o + 4, d0, a, b, d1);
        detail::ld4(o + 8, ia, nox, noy, noz);
        ib = o[12];
    }
    const float dx = fmaf(x, ia, nox), dy = fmaf(y, ia, noy);
    const float dz = (DIMS == 3) ? fmaf(z, ib, noz) : 0.f;
    const float q = (DIMS == 3) ? fmaf(dx, dx, fmaf(dy, dy, dz * dz)) : fmaf(dx, dx, dy * dy);
    if (q < 1.f) active_add<DIMS>(dx, dy, dz, q, a, b, fin, so);
}

// Pre-filter values of one static quad against one point (obstacles 0-1 and
// 2-3): the expanded test without |p|^2, compared with -|p|^2.
template <int DIMS>
__device__ __forceinline__ void quad_values(const float *q, float2 xd, float2 yd, float2 zd, float2 zzd, float2 &v01,
                                            float2 &v23)
{
    const float4 A = *reinterpret_cast<const float4 *>(q);
    const float4 B = *reinterpret_cast<const float4 *>(q + 4);
    const float4 Cc = *reinterpret_cast<const float4 *>(q + 8);
    if constexpr (DIMS == 2) {
        v01 = ffma2(xd, make_float2(A.x, A.y), ffma2(yd, make_float2(B.x, B.y), make_float2(Cc.x, Cc.y)));
        v23 = ffma2(xd, make_float2(A.z, A.w), ffma2(yd, make_float2(B.z, B.w), make_float2(Cc.z, Cc.w)));
    } else {
        const float4 Dd = *reinterpret_cast<const float4 *>(q + 12);
        const float4 E = *reinterpret_cast<const float4 *>(q + 16);
        v01 = ffma2(xd, make_float2(A.x, A.y),
                    ffma2(yd, make_float2(B.x, B.y),
                          ffma2(zd, make_float2(Cc.x, Cc.y), ffma2(zzd, make_float2(Dd.x, Dd.y), make_float2(E.x, E.y)))));
        v23 = ffma2(xd, make_float2(A.z, A.w),
                    ffma2(yd, make_float2(B.z, B.w),
                          ffma2(zd, make_float2(Cc.z, Cc.w), ffma2(zzd, make_float2(Dd.z, Dd.w), make_float2(E.z, E.w)))));
    }
}

template <typename T, int R>
__device__ __forceinline__ T pick(const T (&a)[R], int r)
{
    T v = a[0];
#pragma unroll
    for (int i = 1; i < R; ++i)
        if (r == i) v = a[i];
    return v;
}

// Exact tests of the candidates of a batch of quads [k, k + NB): bit r * NB + i
// of `cand` flags point r against quad k + i.  Candidates are visited point by
// point in obstacle order; the four obstacles of a flagged quad are
// re-evaluated with the same operations and the ones below the threshold
// tested exactly, accumulated into the point's sums as the list path does
// (one FMA per term), so both paths give the same sums.
template <int DIMS, int R, int NB>
__device__ __forceinline__ void quad_candidates(unsigned cand, const float *srec, const float *sObs, int k,
                                                const detail::PackedPoints<DIMS, R> &P, bool fin,
                                                float (&so)[R][DIMS])
{
    constexpr int QS = DIMS == 2 ? 12 : 20;
    while (cand) {
        const int bit = __ffs(cand) - 1;
        cand &= cand - 1;
        const int r = bit / NB, i = bit - r * NB;
        const float2 xd = pick(P.x, r), yd = pick(P.y, r), zd = pick(P.z, r), zzd = pick(P.zz, r);
        const float npq = pick(P.npq, r);
        float2 v01, v23;
        quad_values<DIMS>(srec + size_t(k + i) * QS, xd, yd, zd, zzd, v01, v23);
        unsigned hb = (v01.x < npq ? 1u : 0u) | (v01.y < npq ? 2u : 0u) | (v23.x < npq ? 4u : 0u) |
                      (v23.y < npq ? 8u : 0u);
        while (hb) {
            const int h = __ffs(hb) - 1;
            hb &= hb - 1;
#pragma unroll
            for (int rr = 0; rr < R; ++rr)
                if (rr == r) exact_static<DIMS>(sObs, 4 * (k + i) + h, xd.x, yd.x, zd.x, fin, so[rr]);
        }
    }
}

// Per-point minimum of the pre-filter values over one quad.
template <int DIMS>
__device__ __forceinline__ float quad_min(const float *q, float2 xd, float2 yd, float2 zd, float2 zzd)
{
    float2 v01, v23;
    quad_values<DIMS>(q, xd, yd, zd, zzd, v01, v23);
    return fmin3(v01.x, v01.y, fminf(v23.x, v23.y));
}

template <int DIMS, int R>
__device__ __forceinline__ void moving_rescan(const float *rec, const float *sObs, int k0, int nb, int j0,
                                              const detail::PackedPoints<DIMS, R> &P, const float (&m)[R], bool fin,
                                              float (&so)[R][DIMS])
{
    constexpr int RM = DIMS == 2 ? 12 : 16;
    constexpr int ST = DIMS == 2 ? 12 : 16;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (m[r] < 1.f) {
            for (int b = k0; b < k0 + nb; ++b) {
                float2 dx, dy, dz;
                const float2 q =
                    detail::moving_value<DIMS>(rec + size_t(b) * RM, P.x[r], P.y[r], P.z[r], P.t[r], dx, dy, dz);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float qh = h ? q.y : q.x;
                    if (qh < 1.f) {
                        const float *o = sObs + size_t(j0 + 2 * b + h) * ST;
                        const float a = (DIMS == 2) ? o[3] : o[5], bb = (DIMS == 2) ? o[3] : o[6];
                        active_add<DIMS>(h ? dx.y : dx.x, h ? dy.y : dy.x, h ? dz.y : dz.x, qh, a, bb, fin, so[r]);
                    }
                }
            }
        }
    }
}

// Every obstacle against the thread's R points; all lanes of the CTA run the
// same trip counts, so the votes use the full warp.  Static quads go in
// batches of NQB: one minimum per (point, quad) kept in registers and their
// minimum per point; a thread with a candidate records the batch's (point,
// quad) bits, and after the loop each thread tests its recorded candidates
// exactly, oldest first (all lanes with candidates in one pass instead of one
// warp-wide detour per batch).
template <int DIMS, int R, int NQB>
__device__ __forceinline__ void all_pairs(const float *srec, const float *mrec, const float *sObs, int nq, int nm2,
                                          int ns, const detail::PackedPoints<DIMS, R> &P, bool fin,
                                          float (&so)[R][DIMS])
{
    static_assert(R * NQB <= 32, "candidate bits");
    constexpr int QS = DIMS == 2 ? 12 : 20;
    constexpr int RM = DIMS == 2 ? 12 : 16;
    // candidate batches of this thread, processed after the screening loop
    // (oldest first, so each point still sees its obstacles in order)
    constexpr int MAXE = 3;
    int ek0 = 0, ek1 = 0, ek2 = 0, ne = 0;
    unsigned ec0 = 0u, ec1 = 0u, ec2 = 0u;
    auto flush = [&]() {
        for (int e = 0; e < ne; ++e) {
            const int ke = e == 0 ? ek0 : (e == 1 ? ek1 : ek2);
            const unsigned ce = e == 0 ? ec0 : (e == 1 ? ec1 : ec2);
            quad_candidates<DIMS, R, NQB>(ce, srec, sObs, ke, P, fin, so);
        }
        ne = 0;
    };
    int k = 0;
    for (; k + NQB <= nq; k += NQB) {
        // screening: one minimum per (point, quad), their minimum per point
        float mq[R][NQB];
#pragma unroll
        for (int i = 0; i < NQB; ++i) {
            const float *q = srec + size_t(k + i) * QS;
#pragma unroll
            for (int r = 0; r < R; ++r) mq[r][i] = quad_min<DIMS>(q, P.x[r], P.y[r], P.z[r], P.zz[r]);
        }
        bool f = false;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float m = mq[r][0];
#pragma unroll
            for (int i = 1; i < NQB; i += 2) m = (i + 1 < NQB) ? fmin3(m, mq[r][i], mq[r][i + 1]) : fminf(m, mq[r][i]);
            f |= m < P.npq[r];
        }
        if (f) {
            // record the (point, quad) candidate bits of the batch
            unsigned cand = 0u;
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int i = 0; i < NQB; ++i) cand |= (mq[r][i] < P.npq[r] ? 1u : 0u) << (r * NQB + i);
            if (ne == MAXE) flush();
            if (ne == 0) {
                ek0 = k;
                ec0 = cand;
            } else if (ne == 1) {
                ek1 = k;
                ec1 = cand;
            } else {
                ek2 = k;
                ec2 = cand;
            }
            ++ne;
        }
    }
    flush();
    for (; k < nq; ++k) {
        unsigned cand = 0u;
#pragma unroll
        for (int r = 0; r < R; ++r)
            cand |= (quad_min<DIMS>(srec + size_t(k) * QS, P.x[r], P.y[r], P.z[r], P.zz[r]) < P.npq[r] ? 1u : 0u) << r;
        if (__any_sync(kFull, cand != 0u)) quad_candidates<DIMS, R, 1>(cand, srec, sObs, k, P, fin, so);
    }
    // moving obstacles: the batch minimum is the exact squared scaled distance
    constexpr int NPM = 2;
    for (k = 0; k < nm2; k += NPM) {
        const int nb = min(NPM, nm2 - k);
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
                    const float2 v = detail::moving_value<DIMS>(q, P.x[r], P.y[r], P.z[r], P.t[r], dx, dy, dz);
                    m[r] = fmin3(m[r], v.x, v.y);
                }
            }
        }
        bool f = false;
#pragma unroll
        for (int r = 0; r < R; ++r) f |= m[r] < 1.f;
        if (__any_sync(kFull, f)) moving_rescan<DIMS, R>(mrec, sObs, k, nb, ns, P, m, fin, so);
    }
}

constexpr unsigned kListOverflow = 0x80000000u;

// Shared-memory neighbour lists of one CTA (see PtsLayout).
struct PtsLists {
    float4 *w;             // [R][cap][tl]
    float *z;              // [R][cap][tl] (3-D)
    unsigned short *idx;   // [R][cap][tl] (3-D)
    int tl;
};

// Neighbour lists of the thread's R points (4 bits of count per point in the
// returned word, kListOverflow set when a point had more than list_cap
// obstacles): the static obstacles screened with the quads' inflated
// thresholds and every moving pair by its scaled offsets against
// (1 + delta max(1/a, 1/b))^2, the flagged obstacles appended in obstacle
// order with their offset terms at the point's time.  With a grid (gsm: its
// region, nx > 0) a point screens only the static obstacles of its cell, each
// with the arithmetic of its lane of the quad test, in increasing order; the
// cell holds every obstacle that test can pass for a point in it, so the lists
// are the same as with every quad screened.  Padding entries of the quad and
// pair records are never flagged.
template <int DIMS, int R>
__device__ __forceinline__ unsigned build_lists(const float *srec, const float *mrec, const float *sObs,
                                                const float *gsm, int nq, int nm2, int ns,
                                                const detail::PackedPoints<DIMS, R> &P, float delta,
                                                const PtsLists &Ls, int tid)
{
    constexpr int QS = DIMS == 2 ? 12 : 20;
    constexpr int RM = DIMS == 2 ? 12 : 16;
    constexpr int ST = DIMS == 2 ? 12 : 16;
    constexpr int CAP = list_cap(DIMS);
    unsigned cnt = 0u;
    auto append = [&](int r, int j, float t) {
        const unsigned c = (cnt >> (4 * r)) & 15u;
        if (c < unsigned(CAP)) {
            const int e = (r * CAP + int(c)) * Ls.tl + tid;
            const float *o = sObs + size_t(j) * ST;
            if constexpr (DIMS == 2) {
                Ls.w[e] = make_float4(o[4], fmaf(t, o[8], o[5]), fmaf(t, o[9], o[6]), o[3]);
            } else {
                Ls.w[e] = make_float4(o[8], o[12], fmaf(t, o[13], o[9]), fmaf(t, o[14], o[10]));
                Ls.z[e] = fmaf(t, o[15], o[11]);
                Ls.idx[e] = static_cast<unsigned short>(j);
            }
            cnt += 1u << (4 * r);
        } else {
            cnt |= kListOverflow;
        }
    };
    const int gnx = gsm ? __float_as_int(gsm[4]) : 0;
    if (gnx > 0) {
        const int gny = __float_as_int(gsm[5]);
        const float gx0 = gsm[0], gy0 = gsm[1], gih = gsm[2];
        const unsigned short *gstart = reinterpret_cast<const unsigned short *>(gsm + 8);
        const unsigned short *gent = reinterpret_cast<const unsigned short *>(gsm + grid_layout(ns).ent);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float x = P.x[r].x, y = P.y[r].x;
            const float fx = (x - gx0) * gih, fy = (y - gy0) * gih;
            if (fx >= 0.f && fx < float(gnx) && fy >= 0.f && fy < float(gny)) {
                const int c = min(int(fy), gny - 1) * gnx + min(int(fx), gnx - 1);
                const int e1 = gstart[c + 1];
                const float npq = P.npq[r], t = P.t[r].x;
                for (int e = gstart[c]; e < e1; ++e) {
                    const int jo = gent[e];
                    const float *q = srec + size_t(jo >> 2) * QS + (jo & 3);
                    float v;
                    if constexpr (DIMS == 2)
                        v = fmaf(x, q[0], fmaf(y, q[4], q[8]));
                    else
                        v = fmaf(x, q[0], fmaf(y, q[4], fmaf(P.z[r].x, q[8], fmaf(P.zz[r].x, q[12], q[16]))));
                    if (v < npq) append(r, jo, t);
                }
            }
        }
    } else
    for (int k = 0; k < nq; ++k) {
        const float *q = srec + size_t(k) * QS;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 v01, v23;
            quad_values<DIMS>(q, P.x[r], P.y[r], P.z[r], P.zz[r], v01, v23);
            const float npq = P.npq[r];
            if (fmin3(v01.x, v01.y, fminf(v23.x, v23.y)) < npq) {
                const float t = P.t[r].x;
                if (v01.x < npq) append(r, 4 * k, t);
                if (v01.y < npq) append(r, 4 * k + 1, t);
                if (v23.x < npq) append(r, 4 * k + 2, t);
                if (v23.y < npq) append(r, 4 * k + 3, t);
            }
        }
    }
    for (int k = 0; k < nm2; ++k) {
        const float *q = mrec + size_t(k) * RM;
        const float4 A = *reinterpret_cast<const float4 *>(q);
        const float i0 = DIMS == 2 ? A.x : fmaxf(A.x, A.z), i1 = DIMS == 2 ? A.y : fmaxf(A.y, A.w);
        const float b0 = fmaf(delta, i0, 1.f), b1 = fmaf(delta, i1, 1.f);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 dx, dy, dz;
            const float2 v = detail::moving_value<DIMS>(q, P.x[r], P.y[r], P.z[r], P.t[r], dx, dy, dz);
            if (v.x < b0 * b0) append(r, ns + 2 * k, P.t[r].x);
            if (v.y < b1 * b1) append(r, ns + 2 * k + 1, P.t[r].x);
        }
    }
    return cnt;
}

// Exact tests of the listed obstacles of the thread's points, in list order:
// the arithmetic of exact_static / moving_rescan with the obstacle's offset
// terms at the point's time taken from the list entry.
template <int DIMS, int R>
__device__ __forceinline__ void list_pairs(const float *sObs, const PtsLists &Ls, unsigned cnt, int tid,
                                           const detail::PackedPoints<DIMS, R> &P, bool fin, float (&so)[R][DIMS])
{
    constexpr int CAP = list_cap(DIMS);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int n = int((cnt >> (4 * r)) & 15u);
        const float x = P.x[r].x, y = P.y[r].x, z = P.z[r].x;
        for (int e = 0; e < n; ++e) {
            const int ei = (r * CAP + e) * Ls.tl + tid;
            const float4 w = Ls.w[ei];
            if constexpr (DIMS == 2) {
                const float dx = fmaf(x, w.x, w.y), dy = fmaf(y, w.x, w.z);
                const float q = fmaf(dx, dx, dy * dy);
                if (q < 1.f) active_add<DIMS>(dx, dy, 0.f, q, w.w, w.w, fin, so[r]);
            } else {
                const float dx = fmaf(x, w.x, w.z), dy = fmaf(y, w.x, w.w), dz = fmaf(z, w.y, Ls.z[ei]);
                const float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (q < 1.f) {
                    const float *o = sObs + size_t(Ls.idx[ei]) * 16;
                    active_add<DIMS>(dx, dy, dz, q, o[5], o[6], fin, so[r]);
                }
            }
        }
    }
}

// The projection of samples [s0, s0 + S) of one problem by the calling CTA
// (blockDim.x >= S * TPS, a multiple of 32; all threads call it).
// WL: also return the multipliers of the fixed columns.
template <int DIMS, int R, int NF, bool WL>
__device__ void pts_body(const ProjParams<float> &p, int s0)
{
    static_assert(R % 2 == 0, "points are paired for the f32x2 basis products");
    constexpr int H = R / 2;
    constexpr int ST = DIMS == 2 ? 12 : 16;
    constexpr int QS = DIMS == 2 ? 12 : 20;
    constexpr int RM = DIMS == 2 ? 12 : 16;
    constexpr int NB = 11 - NF;  // fixed columns (degree 10: 11 coefficients per axis)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, T = blockDim.x;
    const int np_ = p.n_p, nv = p.nv, D = DIMS * nv, nobs = p.n_obs, ns = p.n_static;
    const int S = p.S;
    const int S_act = min(S, p.N - s0);
    if (S_act <= 0) return;
    const PtsLayout L = pts_layout(DIMS, NF, nv, np_, nobs, ns, S, R);
    const int TPS = L.tps, CDS = L.cds, PD = DIMS * nv;
    const int s = tid / TPS, j = tid - s * TPS;
    const bool act = s < S_act;
    const int sc = act ? s : 0;  // a valid sample index for idle threads' reads
    const int fw = (sc * TPS) >> 5;
    // last lane of this thread's segment in the warp (idle threads form one segment)
    const int send = act ? min(31, (sc + 1) * TPS - 1 - 32 * warp) : 31;
    const bool head = act && (lane == 0 || j == 0);
    float *sObs = sm + L.obs, *sW = sm + L.W, *sCd = sm + L.cd, *sLam = sm + L.lam, *sXi = sm + L.xi,
          *sPart = sm + L.part;
    double *sPart2 = reinterpret_cast<double *>(sm + L.part2);
    float *sRef = sm + L.ref;
    PtsLists Ls;
    Ls.w = reinterpret_cast<float4 *>(sm + L.list);
    Ls.z = sm + L.listz;
    Ls.idx = reinterpret_cast<unsigned short *>(sm + L.listi);
    Ls.tl = L.tl;
    const float rho = p.rho, vmax = p.vmax, amax = p.amax, vmax2 = vmax * vmax, amax2 = amax * amax;

    // ---- obstacle records and W -> shared memory; a1/a2 sample set-up
    {
        const float4 *src = reinterpret_cast<const float4 *>(p.tab + p.lay.obs);
        float4 *dst = reinterpret_cast<float4 *>(sObs);
        for (int i = tid; i < nobs * ST / 4; i += T) dst[i] = src[i];
        for (int i = tid; i < NF * NF; i += T) sW[i] = p.tab[p.lay.W + i];
        const float4 *gsrc = reinterpret_cast<const float4 *>(p.tab + p.lay.grid);
        float4 *gdst = reinterpret_cast<float4 *>(sm + L.grid);
        for (int i = tid; i < int(L.gsz / 4); i += T) gdst[i] = gsrc[i];
    }
    for (int e = tid; e < S_act * D; e += T) {
        const int ss = e / D, d = e - ss * D;
        const int ax = d / nv, col = d - ax * nv;
        const size_t gi = size_t(s0 + ss) * D + d;
        const int f = col - kFree0;
        if (f < 0 || f >= NF) continue;
        double x;
        if (p.mode == 0) {
            x = p.xi_in[gi];
        } else {
            const size_t seg = p.seg_len > 0 ? size_t((s0 + ss) / p.seg_len) : 0;  // D-PRIEST distribution
            const double *Lrow = p.Lc + (seg * D + d) * D;
            const double *zi = p.z + size_t(s0 + ss) * D;
            x = p.mu[seg * D + d];
            for (int q = 0; q <= d; ++q) x = fma(Lrow[q], zi[q], x);
        }
        const int ro = ss * DIMS + ax;
        sXi[ro * 8 + f] = float(x);
        sCd[ro * CDS + 2 * f] = float(x);
        sCd[ro * CDS + 2 * f + 1] = float(x);
        sLam[ro * 8 + f] = p.lam_in ? float(p.lam_in[gi]) : 0.f;
    }
    // per-thread constants: basis rows (pairs of points), fixed part, time stamps
    float2 bf[3][NF][H], bs[3][DIMS][H];
    float tt[R];
    bool ok[R];
    {
        const int fbs = fb_stride(NF), nfp = nf_padded(NF);
        const float *fb = p.tab + p.lay.fb, *bas = p.tab + p.lay.base, *tv = p.tab + p.lay.tval;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int t = j + TPS * r;
            ok[r] = act && t < np_;
            tt[r] = ok[r] ? tv[t] : 0.f;
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int t0 = j + TPS * (2 * h), t1 = t0 + TPS;
            const bool o0 = ok[2 * h], o1 = ok[2 * h + 1];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    bf[q][f][h] = make_float2(o0 ? fb[size_t(t0) * fbs + q * nfp + f] : 0.f,
                                              o1 ? fb[size_t(t1) * fbs + q * nfp + f] : 0.f);
#pragma unroll
                for (int ax = 0; ax < DIMS; ++ax) {
                    // padding points: far from every obstacle, at rest
                    const float pad = q == 0 ? 1e15f : 0.f;
                    bs[q][ax][h] = make_float2(o0 ? bas[(q * DIMS + ax) * np_ + t0] : pad,
                                               o1 ? bas[(q * DIMS + ax) * np_ + t1] : pad);
                }
            }
        }
    }
    __syncthreads();
    // ---- pair records of the obstacle loop (static thresholds inflated by the
    //      neighbour-list margin: (a + delta)^2 in 2-D, a^2 (1 + delta / min(a, b))^2 in 3-D)
    const float dl = p.list_delta;
    for (int q = tid; q < L.nq; q += T) {
        float *d = sm + L.srec + size_t(q) * QS;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int jo = 4 * q + i;
            const bool okj = jo < ns;
            const float *o = sObs + size_t(okj ? jo : 0) * ST;
            d[i] = okj ? o[0] : 0.f;
            d[4 + i] = okj ? o[1] : 0.f;
            if constexpr (DIMS == 2) {
                d[8 + i] = okj ? -(o[2] + (2.f * o[3] + dl) * dl) : 3e38f;  // padding: never below -|p|^2
            } else {
                const float dm = dl * fmaxf(o[8], o[12]);
                d[8 + i] = okj ? o[2] : 0.f;
                d[12 + i] = okj ? o[4] : 0.f;
                d[16 + i] = okj ? -(o[3] + o[5] * o[5] * dm * (2.f + dm)) : 3e38f;
            }
        }
    }
    for (int q = tid; q < L.nm2; q += T) {
        float *d = sm + L.mrec + size_t(q) * RM;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jo = ns + 2 * q + h;
            const bool okj = jo < nobs;
            const float *o = sObs + size_t(okj ? jo : 0) * ST;
            // padding: scaled offset (4, 4[, 4]) at every time, never active
            if constexpr (DIMS == 2) {
                d[h] = okj ? o[4] : 0.f;
                d[2 + h] = okj ? o[5] : 4.f;
                d[4 + h] = okj ? o[6] : 4.f;
                d[6 + h] = okj ? o[8] : 0.f;
                d[8 + h] = okj ? o[9] : 0.f;
                d[10 + h] = 0.f;
            } else {
                d[h] = okj ? o[8] : 0.f;
                d[2 + h] = okj ? o[12] : 0.f;
                d[4 + h] = okj ? o[9] : 4.f;
                d[6 + h] = okj ? o[10] : 4.f;
                d[8 + h] = okj ? o[11] : 4.f;
                d[10 + h] = okj ? o[13] : 0.f;
                d[12 + h] = okj ? o[14] : 0.f;
                d[14 + h] = okj ? o[15] : 0.f;
            }
        }
    }
    __syncthreads();

    float smin[DIMS], smax[DIMS];
#pragma unroll
    for (int ax = 0; ax < DIMS; ++ax) {
        smin[ax] = p.smin[ax] - p.tab[p.lay.origin + ax];
        smax[ax] = p.smax[ax] - p.tab[p.lay.origin + ax];
    }
    // state lanes: lane = q * DIMS * NF + ax * NF + f serves the warp's q-th
    // sample (sw0 + q), axis ax, free column f
    constexpr int SL = DIMS * NF;
    const int sw0 = (32 * warp) / TPS;               // first sample the warp touches
    const int dq = lane / SL, dax = (lane % SL) / NF, df = lane % NF;
    const int ds = sw0 + dq;
    const bool dact = lane < (32 / SL) * SL && ds < S_act && ds * TPS < 32 * (warp + 1);
    float stC = 0.f, stLam = 0.f, stXi = 0.f, wrow[NF];
    {
        const int ro = (dact ? ds : 0) * DIMS + dax;
        if (dact) {
            stC = sCd[ro * CDS + 2 * df];
            stLam = sLam[ro * 8 + df];
            stXi = sXi[ro * 8 + df];
        }
#pragma unroll
        for (int fi = 0; fi < NF; ++fi) wrow[fi] = sW[df * NF + fi];
    }
    // the state lane holding (my sample, axis, column 0)
    const int cbase = act ? (sc - sw0) * SL : 0;
    float rsum[WL ? R : 1][3][DIMS];  // WL: per-point residual rows summed over the iterations
#pragma unroll
    for (int r = 0; r < (WL ? R : 1); ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) rsum[r][q][ax] = 0.f;

    unsigned lcnt = 0u;  // neighbour-list counts of the thread's points
    for (int k = 0; k <= p.K; ++k) {
        const bool fin = (k == p.K);
        // ---- A: trajectory (pairs of points share one f32x2 FMA per term)
        float pos[R][DIMS], vel[R][DIMS], acc[R][DIMS];
        {
            float cfs[DIMS][NF];
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax)
#pragma unroll
                for (int f = 0; f < NF; ++f) cfs[ax][f] = __shfl_sync(kFull, stC, (cbase + ax * NF + f) & 31);
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) {
                float2 cf[NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) cf[f] = make_float2(cfs[ax][f], cfs[ax][f]);
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    float2 P2 = bs[0][ax][h], V2 = bs[1][ax][h], A2 = bs[2][ax][h];
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        P2 = ffma2(bf[0][f][h], cf[f], P2);
                        V2 = ffma2(bf[1][f][h], cf[f], V2);
                        A2 = ffma2(bf[2][f][h], cf[f], A2);
                    }
                    pos[2 * h][ax] = P2.x;
                    pos[2 * h + 1][ax] = P2.y;
                    vel[2 * h][ax] = V2.x;
                    vel[2 * h + 1][ax] = V2.y;
                    acc[2 * h][ax] = A2.x;
                    acc[2 * h + 1][ax] = A2.y;
                }
            }
        }
        float rv[R][DIMS], ra[R][DIMS], rb[R][DIMS], fvv[R], faa[R], v2v[R], a2v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float v2 = 0.f, a2 = 0.f;
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) {
                v2 = fmaf(vel[r][ax], vel[r][ax], v2);
                a2 = fmaf(acc[r][ax], acc[r][ax], a2);
            }
            const float fv = (v2 > vmax2) ? 1.f - vmax * rsqrtf(v2) : 0.f;
            const float fa = (a2 > amax2) ? 1.f - amax * rsqrtf(a2) : 0.f;
            fvv[r] = fv;
            faa[r] = fa;
            v2v[r] = v2;
            a2v[r] = a2;
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) {
                rv[r][ax] = fv * vel[r][ax];
                ra[r][ax] = fa * acc[r][ax];
                rb[r][ax] = (p.use_bounds && ok[r])
                                ? fmaxf(0.f, pos[r][ax] - smax[ax]) - fmaxf(0.f, smin[ax] - pos[r][ax])
                                : 0.f;
            }
        }
        // ---- B: the thread's points against their listed obstacles (lists rebuilt when needed)
        float so[R][DIMS];
        {
            detail::PackedPoints<DIMS, R> P;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float x = pos[r][0], y = pos[r][1], z = DIMS == 3 ? pos[r][DIMS - 1] : 0.f;
                P.x[r] = make_float2(x, x);
                P.y[r] = make_float2(y, y);
                P.z[r] = make_float2(z, z);
                P.zz[r] = make_float2(z * z, z * z);
                P.t[r] = make_float2(tt[r], tt[r]);
                P.npq[r] = -fmaf(x, x, y * y);
#pragma unroll
                for (int ax = 0; ax < DIMS; ++ax) so[r][ax] = 0.f;
            }
            constexpr int NQB = DIMS == 3 ? 2 : (R >= 4 ? 4 : 2);
            if (dl > 0.f) {
                // rebuild when a point of the CTA moved farther than 7/8 delta:
                // one vote of the whole CTA, so that all warps rebuild in the same
                // iteration instead of each one holding the others at the barrier
                bool moved = k == 0;
                if (act && !moved) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        float d2 = 0.f;
#pragma unroll
                        for (int ax = 0; ax < DIMS; ++ax) {
                            const float e = pos[r][ax] - sRef[(r * DIMS + ax) * L.tl + tid];
                            d2 = fmaf(e, e, d2);
                        }
                        moved = moved || (ok[r] && d2 > 0.765625f * dl * dl);
                    }
                }
                if (__syncthreads_or(moved)) {
                    lcnt = build_lists<DIMS, R>(sm + L.srec, sm + L.mrec, sObs, L.gsz && p.list_grid ? sm + L.grid : nullptr, L.nq,
                                                L.nm2, ns, P, dl, Ls, tid);
                    if (act) {
#pragma unroll
                        for (int r = 0; r < R; ++r)
#pragma unroll
                            for (int ax = 0; ax < DIMS; ++ax) sRef[(r * DIMS + ax) * L.tl + tid] = pos[r][ax];
                    }
                }
                if (__any_sync(kFull, (lcnt & kListOverflow) != 0u))
                    all_pairs<DIMS, R, NQB>(sm + L.srec, sm + L.mrec, sObs, L.nq, L.nm2, ns, P, fin, so);
                else
                    list_pairs<DIMS, R>(sObs, Ls, lcnt, tid, P, fin, so);
            } else {
                all_pairs<DIMS, R, NQB>(sm + L.srec, sm + L.mrec, sObs, L.nq, L.nm2, ns, P, fin, so);
            }
        }
        if (fin) {
            // ---- a9: r = sqrt(sum of squared residual rows), c_1
            double r2 = 0.0, c1 = 0.0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (ok[r]) {
                    float rq = v2v[r] * fvv[r] * fvv[r] + a2v[r] * faa[r] * faa[r];
                    if (p.use_bounds) {
#pragma unroll
                        for (int ax = 0; ax < DIMS; ++ax) {
                            const float hi = fmaxf(0.f, pos[r][ax] - smax[ax]);
                            const float lo = fmaxf(0.f, smin[ax] - pos[r][ax]);
                            rq = fmaf(hi, hi, fmaf(lo, lo, rq));
                        }
                    }
                    r2 += double(rq) + double(so[r][0]);
                    c1 += double(point_cost<float, DIMS>(p.cost, pos[r], vel[r], acc[r], a2v[r]));
                }
            }
            r2 = seg_sum(r2, lane, send);
            c1 = seg_sum(c1, lane, send);
            if (head) {
                double *dst = sPart2 + (size_t(sc) * L.maxw + (warp - fw)) * 2;
                dst[0] = r2;
                dst[1] = c1;
            }
            break;
        }
        // ---- C: this thread's share of g on the free columns, reduced per sample
        float g[DIMS * NF];
#pragma unroll
        for (int ax = 0; ax < DIMS; ++ax) {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const float2 rp = make_float2(so[2 * h][ax] + rb[2 * h][ax], so[2 * h + 1][ax] + rb[2 * h + 1][ax]);
                    const float2 r1 = make_float2(rv[2 * h][ax], rv[2 * h + 1][ax]);
                    const float2 r2v = make_float2(ra[2 * h][ax], ra[2 * h + 1][ax]);
                    acc2 = ffma2(bf[0][f][h], rp, ffma2(bf[1][f][h], r1, ffma2(bf[2][f][h], r2v, acc2)));
                }
                g[ax * NF + f] = acc2.x + acc2.y;
            }
        }
        // reduce g over the sample's threads: the lanes 2i, 2i + 1 always share
        // a sample (TPS is even), so one exchange leaves the first half of the
        // values on even lanes and the second half on odd lanes, and the
        // segmented sum runs over stride-2 lanes on half the values
        constexpr int V = DIMS * NF, VH = (V + 1) / 2;
        float *part = sPart + size_t(k & 1) * S * L.maxw * PD;
        {
            const bool odd = (lane & 1) != 0;
            float h[VH];
#pragma unroll
            for (int i = 0; i < VH; ++i) {
                const float hi = VH + i < V ? g[VH + i] : 0.f;
                const float other = __shfl_xor_sync(kFull, odd ? g[i] : hi, 1);
                h[i] = (odd ? hi : g[i]) + other;
            }
#pragma unroll
            for (int d = 2; d < 32; d <<= 1) {
                float o[VH];
#pragma unroll
                for (int i = 0; i < VH; ++i) o[i] = __shfl_down_sync(kFull, h[i], d);
                if (lane + d <= send) {
#pragma unroll
                    for (int i = 0; i < VH; ++i) h[i] += o[i];
                }
            }
            // the segment's first two lanes hold the sums of the two halves
            const bool h0 = act && !odd && (lane == 0 || j == 0);
            const bool h1 = act && odd && (lane == 1 || j == 1);
            if (h0 || h1) {
                float *dst = part + (size_t(sc) * L.maxw + (warp - fw)) * PD + kFree0;
#pragma unroll
                for (int i = 0; i < VH; ++i) {
                    const int v = (h1 ? VH : 0) + i;
                    if (v < V) dst[(v / NF) * nv + (v % NF)] = h[i];
                }
            }
        }
        if constexpr (WL) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int ax = 0; ax < DIMS; ++ax) {
                    rsum[r][0][ax] += so[r][ax] + rb[r][ax];
                    rsum[r][1][ax] += rv[r][ax];
                    rsum[r][2][ax] += ra[r][ax];
                }
        }
        __syncthreads();
        // ---- D: multiplier step (eq. lag) and shared-inverse step in the state
        //      lanes: lambda^{k+1} = lambda^k - rho g, u = xi + lambda^{k+1} - rho g - c,
        //      c += W u (the u of the lane's sample and axis gathered by shuffles)
        {
            float gs = 0.f;
            if (dact) {
                const int nw = (((ds + 1) * TPS - 1) >> 5) - ((ds * TPS) >> 5) + 1;
                for (int w = 0; w < nw; ++w) gs += part[(size_t(ds) * L.maxw + w) * PD + dax * nv + kFree0 + df];
            }
            const float lnew = stLam - rho * gs;
            const float u = stXi + lnew - rho * gs - stC;
            const int ub = lane - df;  // lane of (sample, axis, column 0)
            float du = 0.f;
#pragma unroll
            for (int fi = 0; fi < NF; ++fi) du = fmaf(wrow[fi], __shfl_sync(kFull, u, (ub + fi) & 31), du);
            if (dact) {
                stLam = lnew;
                stC = stC + du;
            }
        }
    }

    // ---- fixed-column multipliers: P_B^T of the summed residual rows
    if constexpr (WL) {
        const float *bas = p.tab + p.lay.basis;
        for (int cb = 0; cb < NB; ++cb) {
            const int col = cb < kFree0 ? cb : cb + NF;
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) {
                float v = 0.f;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (ok[r]) {
                        const int t = j + TPS * r;
                        v = fmaf(bas[(size_t(0) * np_ + t) * nv + col], rsum[r][0][ax],
                                 fmaf(bas[(size_t(1) * np_ + t) * nv + col], rsum[r][1][ax],
                                      fmaf(bas[(size_t(2) * np_ + t) * nv + col], rsum[r][2][ax], v)));
                    }
                }
                v = seg_sum(v, lane, send);
                if (head) sPart[(size_t(p.K & 1) * S * L.maxw + size_t(sc) * L.maxw + (warp - fw)) * PD + ax * nv + col] = v;
            }
        }
    }
    // free coefficients and multipliers of each sample from its first warp's state lanes
    if (dact && (ds * TPS) >> 5 == warp) {
        const int ro = ds * DIMS + dax;
        sCd[ro * CDS + 2 * df] = stC;
        sLam[ro * 8 + df] = stLam;
    }
    __syncthreads();
    // ---- outputs: r, c_1; xi_bar (boundary coefficients from the closed form), lambda
    for (int ss = tid; ss < S_act; ss += T) {
        const int nw = (((ss + 1) * TPS - 1) >> 5) - ((ss * TPS) >> 5) + 1;
        double r2 = 0.0, c1 = 0.0;
        for (int w = 0; w < nw; ++w) {
            r2 += sPart2[(size_t(ss) * L.maxw + w) * 2];
            c1 += sPart2[(size_t(ss) * L.maxw + w) * 2 + 1];
        }
        p.r_out[s0 + ss] = sqrt(r2);
        p.c1_out[s0 + ss] = c1;
    }
    for (int e = tid; e < S_act * D; e += T) {
        const int ss = e / D, d = e - ss * D;
        const int ax = d / nv, cl = d - ax * nv, f = cl - kFree0;
        const size_t gi = size_t(s0 + ss) * D + d;
        const int ro = ss * DIMS + ax;
        const bool free_col = f >= 0 && f < NF;
        p.xi_bar[gi] = free_col ? double(sCd[ro * CDS + 2 * f]) : p.cB[ax * kMaxNv + cl];
        if (p.lam_out) {
            float lv;
            if (free_col) {
                lv = sLam[ro * 8 + f];
            } else {
                float gsum = 0.f;
                if constexpr (WL) {
                    const int nw = (((ss + 1) * TPS - 1) >> 5) - ((ss * TPS) >> 5) + 1;
                    for (int w = 0; w < nw; ++w)
                        gsum += sPart[(size_t(p.K & 1) * S * L.maxw + size_t(ss) * L.maxw + w) * PD + ax * nv + cl];
                }
                lv = (p.lam_in ? float(p.lam_in[gi]) : 0.f) - rho * gsum;
            }
            p.lam_out[gi] = double(lv);
        }
    }
}

// Largest CTA of each variant: more points per thread need more registers.
template <int R>
constexpr int pts_max_threads() { return R <= 2 ? 384 : 256; }

// The persistent form's CTA: the 2-D five-column variant with two points per
// thread fits 128 registers, so two CTAs of 256 threads share an SM (16
// warps; half the warps per barrier than one CTA of 512, and finer items);
// the other variants keep one CTA of 384 per SM.  The single-problem launch
// keeps the larger register budget, since its grid has one CTA per SM anyway.
template <int DIMS, int R, int NF>
constexpr int pts_batch_threads() { return (DIMS == 2 && R == 2 && NF == 5) ? 256 : pts_max_threads<R>(); }
template <int DIMS, int R, int NF>
constexpr int pts_batch_ctas_per_sm() { return (DIMS == 2 && R == 2 && NF == 5) ? 2 : 1; }

template <int DIMS, int R, int NF, bool WL>
__global__ void __launch_bounds__(pts_max_threads<R>(), 1) pts_kernel(const ProjParams<float> p)
{
    pdl_trigger();
    pdl_wait();
    pts_body<DIMS, R, NF, WL>(p, blockIdx.x * p.S);
}

// Persistent form over many problems: CTAs take (problem, first sample)
// items (each problem's p.S samples per item, p.S * TPS <= blockDim.x) through
// an atomic counter until none is left; the item's parameters are staged in
// shared memory (held in registers they would cost the CTA its size).  *next
// must be zero at launch.
template <int DIMS, int R, int NF, bool WL>
__global__ void __launch_bounds__(pts_batch_threads<DIMS, R, NF>(), pts_batch_ctas_per_sm<DIMS, R, NF>())
    pts_batch_kernel(const ProjParams<float> *params, const int2 *items, int n_items, int *next)
{
    __shared__ int s_item;
    __shared__ ProjParams<float> s_p;  // the item's parameters, read from shared memory where used
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 w = items[it];
        if (threadIdx.x == 0) s_p = params[w.x];
        __syncthreads();
        pts_body<DIMS, R, NF, WL>(s_p, w.y);
        __syncthreads();
    }
}

}  // namespace pts
}  // namespace priest
