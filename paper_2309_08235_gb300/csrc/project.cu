// project.cu -- fused batched projection (Sec. III-A; Appendix eqs. lagrange,
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
#include <algorithm>

#include "priest_internal.cuh"

namespace priest {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Shared-memory layout in Real units: the problem tables first (same layout
// as in global memory, so they are copied as one block), then the state.
struct SmemLayout {
    TableLayout tab;
    size_t xi, lam, c, tp, pos, rv, ra, rb, part, total;
};

__host__ __device__ inline SmemLayout smem_layout(int dims, int nv, int nf, int n_p, int n_obs, int S,
                                                  int C, int use_bounds)
{
    SmemLayout L;
    L.tab = table_layout(dims, nv, nf, n_p, n_obs);
    size_t o = L.tab.total;
    const size_t PS = size_t(S) * n_p;
    L.xi = o;
    o = align8(o + size_t(S) * dims * nf);
    L.lam = o;
    o = align8(o + size_t(S) * dims * nv);
    L.c = o;
    o = align8(o + size_t(S) * dims * nf);
    L.tp = o;
    o = align8(o + PS);
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

// One obstacle against the R points of an item.  Inactive pairs (rho_s >= 1)
// contribute exactly zero; the active branch is taken only when some pair of
// the item is inside.
template <typename Real, int DIMS, int R, bool DYN>
__device__ __forceinline__ void obstacle_pairs(const Real *o, const Real (&px)[R], const Real (&py)[R],
                                               const Real (&pz)[R], const Real (&tt)[R],
                                               Real (&sx)[R], Real (&sy)[R], Real (&sz)[R],
                                               Real (&rq)[R])
{
    if constexpr (DIMS == 2) {
        Real ia, nox, noy, a;
        ld4(o, ia, nox, noy, a);
        Real nvx = Real(0), nvy = Real(0), dum0, dum1;
        if constexpr (DYN) ld4(o + 4, nvx, nvy, dum0, dum1);
        Real dx[R], dy[R], q[R];
        Real qmin = Real(1);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            Real ox = nox, oy = noy;
            if constexpr (DYN) {
                ox = fma(nvx, tt[r], nox);
                oy = fma(nvy, tt[r], noy);
            }
            dx[r] = fma(px[r], ia, ox);
            dy[r] = fma(py[r], ia, oy);
            q[r] = fma(dx[r], dx[r], dy[r] * dy[r]);
            qmin = min(qmin, q[r]);
        }
        if (__any_sync(kFull, qmin < Real(1))) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (q[r] < Real(1)) {
                    if (q[r] > Real(0)) {
                        const Real rs = rsq(q[r]);
                        const Real f = a - a * rs;  // a (1 - 1/rho_s)
                        sx[r] = fma(f, dx[r], sx[r]);
                        sy[r] = fma(f, dy[r], sy[r]);
                        const Real g = rs - Real(1);
                        rq[r] = fma(g * g, a * a * q[r], rq[r]);
                    } else {  // at the centre: alpha = 0, target o + (a, 0)
                        sx[r] -= a;
                        rq[r] = fma(a, a, rq[r]);
                    }
                }
            }
        }
    } else {
        Real ia, nox, noy, noz, ib, a, b, pad;
        ld4(o, ia, nox, noy, noz);
        ld4(o + 4, ib, a, b, pad);
        Real nvx = Real(0), nvy = Real(0), nvz = Real(0), dum;
        if constexpr (DYN) ld4(o + 8, nvx, nvy, nvz, dum);
        Real dx[R], dy[R], dz[R], q[R];
        Real qmin = Real(1);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            Real ox = nox, oy = noy, oz = noz;
            if constexpr (DYN) {
                ox = fma(nvx, tt[r], nox);
                oy = fma(nvy, tt[r], noy);
                oz = fma(nvz, tt[r], noz);
            }
            dx[r] = fma(px[r], ia, ox);
            dy[r] = fma(py[r], ia, oy);
            dz[r] = fma(pz[r], ib, oz);
            q[r] = fma(dx[r], dx[r], fma(dy[r], dy[r], dz[r] * dz[r]));
            qmin = min(qmin, q[r]);
        }
        if (__any_sync(kFull, qmin < Real(1))) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (q[r] < Real(1)) {
                    if (q[r] > Real(0)) {
                        const Real rs = rsq(q[r]);
                        const Real w = Real(1) - rs;
                        const Real fa = a * w, fb = b * w;
                        sx[r] = fma(fa, dx[r], sx[r]);
                        sy[r] = fma(fa, dy[r], sy[r]);
                        sz[r] = fma(fb, dz[r], sz[r]);
                        const Real d2 = a * a * fma(dx[r], dx[r], dy[r] * dy[r]) + b * b * dz[r] * dz[r];
                        rq[r] = fma(w * w, d2, rq[r]);
                    } else {  // at the centre: alpha = beta = 0, target o + (0, 0, b)
                        sz[r] -= b;
                        rq[r] = fma(b, b, rq[r]);
                    }
                }
            }
        }
    }
}

template <typename Real, int DIMS, int R, int THREADS>
__global__ void __launch_bounds__(THREADS) project_kernel(const ProjParams<Real> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *sm = reinterpret_cast<Real *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int T = THREADS, NW = THREADS / 32;
    const int nv = p.nv, nf = p.nf, np_ = p.n_p, S = p.S, C = p.C;
    const int D = DIMS * nv;
    const int s0 = blockIdx.x * S;
    const int S_act = min(S, p.N - s0);
    if (S_act <= 0) return;
    const int PS = S * np_;
    const int P_act = S_act * np_;
    const SmemLayout L = smem_layout(DIMS, nv, nf, np_, p.n_obs, S, C, p.use_bounds);
    const Real *sBasis = sm + L.tab.basis;
    const Real *sBase = sm + L.tab.base;
    const Real *sW = sm + L.tab.W;
    const Real *sObs = sm + L.tab.obs;
    const Real *sT = sm + L.tab.tval;
    Real *sXi = sm + L.xi;
    Real *sLam = sm + L.lam;
    Real *sC = sm + L.c;
    Real *sTp = sm + L.tp;
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
    for (int e = tid; e < S_act * D; e += T) {
        const int s = e / D, d = e - s * D;
        const int ax = d / nv, col = d - ax * nv;
        const size_t gi = size_t(s0 + s) * D + d;
        double x;
        if (p.mode == 0) {
            x = p.xi_in[gi];
        } else {
            const double *Lrow = p.Lc + size_t(d) * D;
            const double *zi = p.z + size_t(s0 + s) * D;
            x = p.mu[d];
            for (int k = 0; k <= d; ++k) x = fma(Lrow[k], zi[k], x);
        }
        const int f = col - kFree0;
        if (f >= 0 && f < nf) {
            sXi[(s * DIMS + ax) * nf + f] = Real(x);
            sC[(s * DIMS + ax) * nf + f] = Real(x);
        }
        sLam[(s * DIMS + ax) * nv + col] = p.lam_in ? Real(p.lam_in[gi]) : Real(0);
    }
    __syncthreads();
    // time stamp of every point (for moving obstacles)
    for (int pt = tid; pt < P_act; pt += T) sTp[pt] = sT[pt % np_];

    // obstacle-loop items: (group of R points, obstacle chunk); the group
    // count is padded to a warp multiple so each warp works on one chunk
    const int n_groups = (((P_act + R - 1) / R) + 31) & ~31;
    const int Cs = (p.n_obs + C - 1) / C;
    const int items = n_groups * C;
    // transposed-basis step: one warp per (sample, axis); lane = (column, segment)
    const int col_lo = p.want_lambda ? 0 : kFree0;
    const int ng = p.want_lambda ? nv : nf;
    int ngp = 1;
    while (ngp < ng) ngp <<= 1;
    const int nseg = 32 / ngp;
    const int f_lane = lane / nseg, seg = lane - f_lane * nseg;
    const int col = col_lo + f_lane;
    const bool col_ok = f_lane < ng;
    const int fcol = col - kFree0;
    const bool is_free = col_ok && fcol >= 0 && fcol < nf;
    constexpr int ST = DIMS == 2 ? 8 : 12;

    for (int k = 0; k <= p.K; ++k) {
        const bool fin = (k == p.K);
        // ---- A: trajectory, velocity / acceleration / workspace residuals
        for (int pt = tid; pt < P_act; pt += T) {
            const int s = pt / np_, t = pt - s * np_;
            const Real *b0 = sBasis + size_t(0 * np_ + t) * nv + kFree0;
            const Real *b1 = sBasis + size_t(1 * np_ + t) * nv + kFree0;
            const Real *b2 = sBasis + size_t(2 * np_ + t) * nv + kFree0;
            const Real *cc = sC + s * DIMS * nf;
            Real pos[DIMS], vel[DIMS], acc[DIMS];
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax) {
                pos[ax] = sBase[(0 * np_ + t) * DIMS + ax];
                vel[ax] = sBase[(1 * np_ + t) * DIMS + ax];
                acc[ax] = sBase[(2 * np_ + t) * DIMS + ax];
            }
            for (int f = 0; f < nf; ++f) {
                const Real p0 = b0[f], p1 = b1[f], p2 = b2[f];
#pragma unroll
                for (int ax = 0; ax < DIMS; ++ax) {
                    const Real cf = cc[ax * nf + f];
                    pos[ax] = fma(p0, cf, pos[ax]);
                    vel[ax] = fma(p1, cf, vel[ax]);
                    acc[ax] = fma(p2, cf, acc[ax]);
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
                        sRB[ax * PS + pt] = max(Real(0), pos[ax] - p.smax[ax]) - max(Real(0), p.smin[ax] - pos[ax]);
                }
            } else {
                Real rq = v2 * fv * fv + a2 * fa * fa;
                if (p.use_bounds) {
#pragma unroll
                    for (int ax = 0; ax < DIMS; ++ax) {
                        const Real hi = max(Real(0), pos[ax] - p.smax[ax]);
                        const Real lo = max(Real(0), p.smin[ax] - pos[ax]);
                        rq = fma(hi, hi, fma(lo, lo, rq));
                    }
                }
                sRV[pt] = rq;
                sRA[pt] = a2;
            }
        }
        __syncthreads();
        // ---- B: obstacle pairs, per (group of R points, obstacle chunk)
        for (int it = tid; it < items; it += T) {
            const int c = it / n_groups, g = it - c * n_groups;
            const int p0 = g * R;
            Real px[R], py[R], pz[R], tt[R], sx[R], sy[R], sz[R], rq[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int pp = p0 + r;
                const bool ok = pp < P_act;
                // padding points sit far outside every obstacle
                px[r] = ok ? sPos[pp] : Real(1e15);
                py[r] = ok ? sPos[PS + pp] : Real(1e15);
                pz[r] = (DIMS == 3 && ok) ? sPos[2 * PS + pp] : Real(1e15);
                tt[r] = Real(0);
                sx[r] = sy[r] = sz[r] = rq[r] = Real(0);
            }
            const int j0 = c * Cs, j1 = min(j0 + Cs, p.n_obs);
            const int js = min(j1, p.n_static);
            for (int j = j0; j < js; ++j)
                obstacle_pairs<Real, DIMS, R, false>(sObs + size_t(j) * ST, px, py, pz, tt, sx, sy, sz, rq);
            const int jd = max(j0, p.n_static);
            if (jd < j1) {
#pragma unroll
                for (int r = 0; r < R; ++r) tt[r] = (p0 + r < P_act) ? sTp[p0 + r] : Real(0);
                for (int j = jd; j < j1; ++j)
                    obstacle_pairs<Real, DIMS, R, true>(sObs + size_t(j) * ST, px, py, pz, tt, sx, sy, sz, rq);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int pp = p0 + r;
                if (pp < P_act) {
                    if (!fin) {
                        sPart[(c * DIMS + 0) * PS + pp] = sx[r];
                        sPart[(c * DIMS + 1) * PS + pp] = sy[r];
                        if (DIMS == 3) sPart[(c * DIMS + 2) * PS + pp] = sz[r];
                    } else {
                        sPart[c * DIMS * PS + pp] = rq[r];
                    }
                }
            }
        }
        __syncthreads();
        if (fin) break;
        // ---- chunk partials -> one P-row residual per point (+ workspace rows)
        if (C > 1 || p.use_bounds) {
#pragma unroll
            for (int ax = 0; ax < DIMS; ++ax)
                for (int pt = tid; pt < P_act; pt += T) {
                    Real v = sPart[ax * PS + pt];
                    for (int c = 1; c < C; ++c) v += sPart[(c * DIMS + ax) * PS + pt];
                    if (p.use_bounds) v += sRB[ax * PS + pt];
                    sPart[ax * PS + pt] = v;
                }
            __syncthreads();
        }
        // ---- C/D: g = F^T(F xi_bar - e) (eq. lag), multiplier step, shared-inverse
        //      step (eqs. affine_trans / comp_zeta); one warp per (sample, axis)
        for (int task = warp; task < S_act * DIMS; task += NW) {
            const int s = task / DIMS, ax = task - s * DIMS;
            Real acc = Real(0);
            if (col_ok) {
                for (int t = seg; t < np_; t += nseg) {
                    const int pp = s * np_ + t;
                    const Real rp = sPart[ax * PS + pp], rv = sRV[ax * PS + pp], ra = sRA[ax * PS + pp];
                    const Real *b = sBasis + size_t(t) * nv + col;
                    acc = fma(b[0], rp, fma(b[size_t(np_) * nv], rv, fma(b[size_t(2 * np_) * nv], ra, acc)));
                }
            }
            for (int off = nseg >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
            const Real g = acc;
            Real *lam = sLam + (s * DIMS + ax) * nv;
            Real *cc = sC + (s * DIMS + ax) * nf;
            const Real *xi = sXi + (s * DIMS + ax) * nf;
            const Real lam_new = col_ok ? lam[col] - rho * g : Real(0);
            const Real u = is_free ? xi[fcol] + lam_new - rho * g - cc[fcol] : Real(0);
            Real du = Real(0);
            for (int j = 0; j < nf; ++j) {
                const Real uj = __shfl_sync(kFull, u, (j + kFree0 - col_lo) * nseg);
                if (is_free) du = fma(sW[fcol * nf + j], uj, du);
            }
            __syncwarp();
            if (seg == 0) {
                if (col_ok) lam[col] = lam_new;
                if (is_free) cc[fcol] += du;
            }
        }
        __syncthreads();
    }

    // ---- a9: r = sqrt(sum of squared residual rows), c_1 = sum ||acc||^2
    for (int s = warp; s < S_act; s += NW) {
        double r2 = 0.0, c1 = 0.0;
        for (int t = lane; t < np_; t += 32) {
            const int pp = s * np_ + t;
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
    for (int e = tid; e < S_act * D; e += T) {
        const int s = e / D, d = e - s * D;
        const int ax = d / nv, cl = d - ax * nv, f = cl - kFree0;
        const size_t gi = size_t(s0 + s) * D + d;
        p.xi_bar[gi] = (f >= 0 && f < nf) ? double(sC[(s * DIMS + ax) * nf + f]) : p.cB[ax * kMaxNv + cl];
        if (p.lam_out) p.lam_out[gi] = double(sLam[(s * DIMS + ax) * nv + cl]);
    }
}

template <typename Real, int DIMS, int R, int THREADS>
cudaError_t launch_one(const ProjParams<Real> &p, const Tiling &t, cudaStream_t st)
{
    static size_t granted = 0;  // per instantiation
    cudaError_t e = reserve_smem(project_kernel<Real, DIMS, R, THREADS>, t.smem, granted);
    if (e != cudaSuccess) return e;
    const int grid = (p.N + t.S - 1) / t.S;
    project_kernel<Real, DIMS, R, THREADS><<<grid, THREADS, t.smem, st>>>(p);
    return cudaGetLastError();
}

// CTA size per (precision, dims): bounded by the registers the kernel needs.
template <typename Real>
int threads_for(int dims)
{
    if (sizeof(Real) == 8) return 256;
    return dims == 2 ? 1024 : 512;
}

}  // namespace

template <typename Real>
size_t project_smem_bytes(const Shape &sh, int S, int C)
{
    return smem_layout(sh.dims, sh.nv, sh.nf, sh.n_p, sh.n_obs, S, C, sh.use_bounds).total * sizeof(Real);
}

// Tile choice: S samples per CTA so the grid covers the SMs once, then the
// obstacle chunk count C that minimises the modelled critical path of the
// pair loop (rounds of items x per-item work) within the shared-memory cap.
template <typename Real>
Tiling choose_tiling(const Shape &sh, int n_samples, int n_sm)
{
    Tiling t;
    t.R = 4;
    t.threads = threads_for<Real>(sh.dims);
    const size_t cap = 227 * 1024;
    int S = std::max(1, (n_samples + n_sm - 1) / n_sm);
    while (S > 1 && project_smem_bytes<Real>(sh, S, 1) > cap) S = std::max(1, S * 3 / 4);
    const double pair_cost = sh.dims == 2 ? 5.5 : 7.5, item_cost = 48.0;
    const int groups = (((S * sh.n_p + t.R - 1) / t.R) + 31) & ~31;
    int bestC = 1;
    double best = 1e300;
    const int cmax = std::max(1, std::min(16, sh.n_obs));
    for (int C = 1; C <= cmax; ++C) {
        if (project_smem_bytes<Real>(sh, S, C) > cap) break;
        const int items = groups * C;
        const int rounds = (items + t.threads - 1) / t.threads;
        const int Cs = (sh.n_obs + C - 1) / C;
        const double cost = rounds * (Cs * t.R * pair_cost + item_cost) + (C - 1) * 4.0;
        if (cost < best - 1e-9) {
            best = cost;
            bestC = C;
        }
    }
    t.S = S;
    t.C = bestC;
    t.smem = project_smem_bytes<Real>(sh, S, bestC);
    return t;
}

template <typename Real>
cudaError_t launch_project(const ProjParams<Real> &p, const Tiling &t, cudaStream_t st)
{
    if (p.N <= 0) return cudaSuccess;
    if constexpr (sizeof(Real) == 8) {
        if (p.dims == 2) return launch_one<Real, 2, 4, 256>(p, t, st);
        return launch_one<Real, 3, 4, 256>(p, t, st);
    } else {
        if (p.dims == 2) return launch_one<Real, 2, 4, 1024>(p, t, st);
        return launch_one<Real, 3, 4, 512>(p, t, st);
    }
}

template size_t project_smem_bytes<float>(const Shape &, int, int);
template size_t project_smem_bytes<double>(const Shape &, int, int);
template Tiling choose_tiling<float>(const Shape &, int, int);
template Tiling choose_tiling<double>(const Shape &, int, int);
template cudaError_t launch_project<float>(const ProjParams<float> &, const Tiling &, cudaStream_t);
template cudaError_t launch_project<double>(const ProjParams<double> &, const Tiling &, cudaStream_t);

}  // namespace priest
