// setup.cu -- step a0 of the hot path, once per problem: the Bernstein basis
// and its derivatives (Sec. II-A.2, eq. parametrized), the coefficients fixed
// by the boundary conditions (A xi = b_eq), the inverse of the shared KKT block
// (Sec. III-A, eqs. affine_trans / matrix_vec, reduced to the free
// coefficients), pre-scaled obstacle records, and for a full solve the first
// sampling factor chol(Sigma_0 + eps I) (Alg. 1).  All arithmetic in FP64; the
// FP32 working tables are rounded copies.
//
// Design note: with the Bernstein basis every boundary row of A touches only
// the end coefficients (c_0..c_2 at t_0, c_{n-2}..c_n at t_f), so {A c = b}
// fixes those coefficients in closed form and leaves the interior ones free.
// The KKT system of eq. matrix_vec then reduces to
//   c_F = (I + rho Q_FF)^-1 (rhs_F - rho Q_FB c_B),  Q = F^T F per axis,
// and the projection only ever needs W = (I + rho Q_FF)^-1.
#include "block_linalg.cuh"
#include "priest_internal.cuh"

namespace priest {
namespace {

constexpr int kSetupThreads = 512;
// The FP64 basis is staged in shared memory when it fits.
constexpr size_t kSetupBasisSmem = 160 * 1024;

// Bernstein values of degree n, n-1 and n-2 at tau by the triangular
// recurrence B_{j,m} = (1 - tau) B_{j,m-1} + tau B_{j-1,m-1}.
__device__ void bernstein_levels(int n, double tau, double *bn, double *bn1, double *bn2)
{
    double b[kMaxNv];
    for (int j = 0; j <= n; ++j) b[j] = 0.0;
    b[0] = 1.0;
    for (int m = 1; m <= n; ++m) {
        for (int j = m; j >= 1; --j) b[j] = (1.0 - tau) * b[j] + tau * b[j - 1];
        b[0] = (1.0 - tau) * b[0];
        if (m == n - 2)
            for (int j = 0; j <= n; ++j) bn2[j] = (j <= m) ? b[j] : 0.0;
        if (m == n - 1)
            for (int j = 0; j <= n; ++j) bn1[j] = (j <= m) ? b[j] : 0.0;
    }
    for (int j = 0; j <= n; ++j) bn[j] = b[j];
}

// Rounding margin of the expanded pre-filter of one obstacle record
// (|o|^2-scaled, so it also bounds the rounding for points near the obstacle).
__device__ inline double screen_margin(double oo, double a, double kap, int dims, double eps)
{
    const double on = double(sqrtf(float(oo)) * 1.001f) + a + 1.0;  // bound only
    return 64.0 * eps * (4.0 * on * on) * (dims == 3 ? 1.0 + kap : 1.0);
}

// Step (9), FP32 tables: the uniform grid over the static obstacles (layout in
// priest_internal.cuh) for the point-owner kernel's neighbour-list builds.
// The pre-filter of the list build (thresholds inflated by the list margin
// delta) accepts a point only within the x-y radius
//   rho^2 = R^2 (1 + 1e-5) + 2 margin,  R = a + delta (2-D),
//   R = a (1 + delta max(1/a, 1/b)) (3-D),
// (the factor covers the FP32 evaluation of the expanded test and of the
// inflation; rho itself is evaluated in FP32 and enlarged by another factor
// 1 + 1e-5, far above that evaluation's rounding); every obstacle is entered
// in each cell its square of half-width rho + h/1000 meets, so a cell's list
// holds every static obstacle that any point the kernel maps to the cell can
// pass, in increasing order.  Counting and filling use shared-memory atomics,
// then each cell is sorted; a cell of more than kGridCellMax obstacles (or no
// margin) leaves nx = 0 (no grid).
__device__ void build_grid(const SetupParams &p, const double *org, float *reg, float eps)
{
    const Shape &sh = p.sh;
    const int ns = sh.n_static, dims = sh.dims, tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
    int *ireg = reinterpret_cast<int *>(reg);
    const GridLayout gl = grid_layout(ns);
    __shared__ int s_cnt[32 * 32 + 1];
    __shared__ float s_red[5][kSetupThreads / 32];
    __shared__ float s_geo[4];  // x0, y0, h, 1/h
    __shared__ int s_n[3];      // nx, ny, fullest cell
    if (ns < kGridMinStatic || !(sh.list_delta > 0.0)) {
        if (tid == 0) {
            for (int i = 0; i < 8; ++i) ireg[i] = 0;
        }
        return;
    }
    const float delta = float(sh.list_delta);
    // centre (x, y) relative to the origin and screening radius of obstacle j
    auto geometry = [&](int j, float &cx, float &cy) {
        const float a = float(p.semi[2 * j]), b = dims == 3 ? float(p.semi[2 * j + 1]) : a;
        const float kap = (a * a) / (b * b);
        float oo = 0.f;
        for (int ax = 0; ax < dims; ++ax) {
            const float c = float(p.center[j * dims + ax] - org[ax]);
            oo += (ax == 2 ? kap : 1.f) * c * c;
            if (ax == 0) cx = c;
            if (ax == 1) cy = c;
        }
        const float on = sqrtf(oo) * 1.001f + a + 1.f;  // as the record's margin
        const float margin = 64.f * eps * (4.f * on * on) * (dims == 3 ? 1.f + kap : 1.f);
        const float R = dims == 3 ? a * (1.f + delta * fmaxf(1.f / a, 1.f / b)) : a + delta;
        return sqrtf((R * R * (1.f + 1e-5f) + 2.f * margin) * (1.f + 1e-5f));
    };
    // extent of the screening discs and the largest radius (warp, then one warp over the warps)
    const float big = 3.0e38f;
    float v[5] = {big, big, -big, -big, 0.f};
    for (int j = tid; j < ns; j += T) {
        float cx = 0.f, cy = 0.f;
        const float r = geometry(j, cx, cy);
        v[0] = fminf(v[0], cx - r);
        v[1] = fminf(v[1], cy - r);
        v[2] = fmaxf(v[2], cx + r);
        v[3] = fmaxf(v[3], cy + r);
        v[4] = fmaxf(v[4], r);
    }
    for (int off = 16; off > 0; off >>= 1)
        for (int i = 0; i < 5; ++i) {
            const float o = __shfl_xor_sync(0xffffffffu, v[i], off);
            v[i] = i < 2 ? fminf(v[i], o) : fmaxf(v[i], o);
        }
    if (lane == 0)
        for (int i = 0; i < 5; ++i) s_red[i][tid >> 5] = v[i];
    for (int c = tid; c <= 32 * 32; c += T) s_cnt[c] = 0;
    __syncthreads();
    if (tid < 32) {
        const int nw = (T + 31) / 32;
        for (int i = 0; i < 5; ++i) v[i] = lane < nw ? s_red[i][lane] : (i < 2 ? big : (i < 4 ? -big : 0.f));
        for (int off = 16; off > 0; off >>= 1)
            for (int i = 0; i < 5; ++i) {
                const float o = __shfl_xor_sync(0xffffffffu, v[i], off);
                v[i] = i < 2 ? fminf(v[i], o) : fmaxf(v[i], o);
            }
        if (lane == 0) {
            const int gs = grid_side(ns);
            const float ext = fmaxf(v[2] - v[0], v[3] - v[1]);
            const float h = fmaxf(2.02f * v[4], ext / (float(gs) - 0.1f));
            const float x0 = v[0] - 0.02f * h, y0 = v[1] - 0.02f * h;
            s_geo[0] = x0;
            s_geo[1] = y0;
            s_geo[2] = h;
            s_geo[3] = 1.0f / h;
            s_n[0] = min(gs, max(1, int(ceilf((v[2] - x0) / h + 0.01f))));
            s_n[1] = min(gs, max(1, int(ceilf((v[3] - y0) / h + 0.01f))));
            s_n[2] = 0;
            // coordinates beyond FP32's range: no grid (the quads screen every static obstacle)
            if (!(h > 0.f) || !isfinite(h) || !isfinite(s_geo[3]) || !isfinite(x0) || !isfinite(y0) ||
                !isfinite(v[2] - x0) || !isfinite(v[3] - y0))
                s_n[0] = 0;
        }
    }
    __syncthreads();
    const float x0 = s_geo[0], y0 = s_geo[1], h = s_geo[2], ih = s_geo[3];
    const int nx = s_n[0], ny = s_n[1];
    if (nx == 0) {
        if (tid == 0) {
            for (int i = 0; i < 8; ++i) ireg[i] = 0;
        }
        return;
    }
    unsigned short *start = reinterpret_cast<unsigned short *>(reg + gl.start);
    unsigned short *ent = reinterpret_cast<unsigned short *>(reg + gl.ent);
    int *rng = reinterpret_cast<int *>(reg + gl.rng);
    // cell ranges (8 bits each: x0 x1 y0 y1, every bound clamped into the
    // grid, so the fill pass below decodes exactly the ranges counted here)
    // and counts
    auto cell = [](float u, int n) { return min(max(int(floorf(u)), 0), n - 1); };
    for (int j = tid; j < ns; j += T) {
        float cx = 0.f, cy = 0.f;
        const float r = geometry(j, cx, cy) + 1e-3f * h;
        const int ax0 = cell((cx - r - x0) * ih, nx), ax1 = cell((cx + r - x0) * ih, nx);
        const int ay0 = cell((cy - r - y0) * ih, ny), ay1 = cell((cy + r - y0) * ih, ny);
        rng[j] = ax0 | (ax1 << 8) | (ay0 << 16) | (ay1 << 24);
        for (int cy2 = ay0; cy2 <= ay1; ++cy2)
            for (int cx2 = ax0; cx2 <= ax1; ++cx2) atomicAdd(&s_cnt[cy2 * nx + cx2], 1);
    }
    __syncthreads();
    // cell starts (exclusive prefix sum by one warp) and the fullest cell
    const int nc = nx * ny;
    if (tid < 32) {
        const int per = (nc + 31) / 32, b0 = tid * per;
        int sum = 0, most = 0;
        for (int c = b0; c < min(nc, b0 + per); ++c) {
            sum += s_cnt[c];
            most = max(most, s_cnt[c]);
        }
        int inc = sum;
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, inc, off);
            if (tid >= off) inc += o;
        }
        for (int off = 16; off > 0; off >>= 1) most = max(most, __shfl_xor_sync(0xffffffffu, most, off));
        int run = inc - sum;
        for (int c = b0; c < min(nc, b0 + per); ++c) {
            const int n = s_cnt[c];
            start[c] = static_cast<unsigned short>(run);
            s_cnt[c] = run;  // fill cursor
            run += n;
        }
        if (tid == 31) {
            start[nc] = static_cast<unsigned short>(inc);
            s_n[2] = most;
            ireg[6] = inc;
        }
    }
    __syncthreads();
    if (s_n[2] > kGridCellMax) {
        if (tid == 0) {
            for (int i = 0; i < 8; ++i) ireg[i] = 0;
        }
        return;
    }
    for (int j = tid; j < ns; j += T) {
        const int g = rng[j];
        const int gx0 = g & 255, gx1 = (g >> 8) & 255, gy0 = (g >> 16) & 255, gy1 = (g >> 24) & 255;
        for (int cy2 = gy0; cy2 <= gy1; ++cy2)
            for (int cx2 = gx0; cx2 <= gx1; ++cx2)
                ent[atomicAdd(&s_cnt[cy2 * nx + cx2], 1)] = static_cast<unsigned short>(j);
    }
    __syncthreads();
    // entries of each cell in increasing obstacle order (insertion sort)
    for (int c = tid; c < nc; c += T) {
        const int e0 = start[c], e1 = start[c + 1];
        for (int e = e0 + 1; e < e1; ++e) {
            const unsigned short x = ent[e];
            int i = e - 1;
            while (i >= e0 && ent[i] > x) {
                ent[i + 1] = ent[i];
                --i;
            }
            ent[i + 1] = x;
        }
    }
    if (tid == 0) {
        reg[0] = s_geo[0];
        reg[1] = s_geo[1];
        reg[2] = s_geo[3];
        reg[3] = s_geo[2];
        ireg[4] = nx;
        ireg[5] = ny;
        ireg[7] = 0;
    }
}

template <typename Real>
__device__ void write_tables(const SetupParams &p, const double *src, size_t from, size_t to)
{
    Real *dst = reinterpret_cast<Real *>(p.tab);
    for (size_t i = from + threadIdx.x; i < to; i += blockDim.x) dst[i] = static_cast<Real>(src[i]);
}

__device__ void setup_body(const SetupParams &p, double *tab64)
{
    const Shape &sh = p.sh;
    const int tid = threadIdx.x, T = blockDim.x;
    const int n = sh.degree, nv = sh.nv, np_ = sh.n_p, dims = sh.dims, nf = sh.nf;
    const TableLayout lay = table_layout(dims, nv, nf, np_, sh.n_obs);
    double *basis = tab64 + lay.basis;
    double *base = tab64 + lay.base;
    double *W = tab64 + lay.W;
    double *obs = tab64 + lay.obs;
    double *tval = tab64 + lay.tval;

    __shared__ double s_cB[3][kMaxNv];
    __shared__ double s_G[3][kMaxNv][kMaxNv];
    __shared__ double s_M[kMaxNv][2 * kMaxNv];
    __shared__ double s_fcol[kMaxNv];
    __shared__ int s_flag;
    extern __shared__ double s_dyn[];  // D x D for the Cholesky, then the staged basis
    const size_t nbasis = size_t(3) * np_ * nv;
    const bool staged = nbasis * sizeof(double) <= kSetupBasisSmem;
    double *bsrc = staged ? s_dyn + size_t(sh.D) * sh.D : basis;  // where the sums read the basis

    double *gram = p.cB + 3 * kMaxNv;  // [3][kMaxNv][kMaxNv]
    // (1) basis rows and time stamps (once per problem shape; afterwards only
    //     staged back into shared memory)
    if (p.shape_ready) {
        if (staged)
            for (size_t e = tid; e < nbasis; e += T) bsrc[e] = basis[e];
    } else
    for (int t = tid; t < np_; t += T) {
        const double tau = double(t) / double(np_ - 1);
        double bn[kMaxNv], bn1[kMaxNv], bn2[kMaxNv];
        bernstein_levels(n, tau, bn, bn1, bn2);
        for (int j = 0; j < nv; ++j) {
            const double d1 = n * ((j >= 1 ? bn1[j - 1] : 0.0) - (j <= n - 1 ? bn1[j] : 0.0));
            const double d2 = n * (n - 1) *
                              ((j >= 2 ? bn2[j - 2] : 0.0) - 2.0 * (j >= 1 && j - 1 <= n - 2 ? bn2[j - 1] : 0.0) +
                               (j <= n - 2 ? bn2[j] : 0.0));
            basis[(0 * np_ + t) * nv + j] = bn[j];
            basis[(1 * np_ + t) * nv + j] = d1 / sh.horizon;
            basis[(2 * np_ + t) * nv + j] = d2 / (sh.horizon * sh.horizon);
            if (staged) {
                bsrc[(0 * np_ + t) * nv + j] = bn[j];
                bsrc[(1 * np_ + t) * nv + j] = d1 / sh.horizon;
                bsrc[(2 * np_ + t) * nv + j] = d2 / (sh.horizon * sh.horizon);
            }
        }
        tval[t] = sh.horizon * double(t) / double(np_ - 1);
    }
    __syncthreads();
    // (1b) packed free columns per time stamp: fb[t][q][f] = B_q[t][3 + f]
    if (!p.shape_ready) {
        const int nfp = nf_padded(nf), fbs = fb_stride(nf);
        double *fb = tab64 + lay.fb;
        for (int e = tid; e < np_ * fbs; e += T) {
            const int t = e / fbs, w = e - t * fbs, q = w / nfp, f = w - q * nfp;
            fb[e] = (q < 3 && f < nf) ? basis[(q * np_ + t) * nv + kFree0 + f] : 0.0;
        }
    }
    // (2) coefficients fixed by the boundary rows (closed form of A c = b)
    if (tid < dims) {
        const int ax = tid;
        const double Th = sh.horizon, nn = double(n), n2 = double(n) * double(n - 1);
        for (int j = 0; j < kMaxNv; ++j) s_cB[ax][j] = 0.0;
        s_cB[ax][0] = sh.b0[ax][0];
        s_cB[ax][1] = s_cB[ax][0] + Th * sh.b0[ax][1] / nn;
        s_cB[ax][2] = 2.0 * s_cB[ax][1] - s_cB[ax][0] + Th * Th * sh.b0[ax][2] / n2;
        if (sh.bc_mask & 1) s_cB[ax][n] = sh.bf[ax][0];
        if (sh.bc_mask & 2) s_cB[ax][n - 1] = s_cB[ax][n] - Th * sh.bf[ax][1] / nn;
        if (sh.bc_mask & 4) s_cB[ax][n - 2] = 2.0 * s_cB[ax][n - 1] - s_cB[ax][n] + Th * Th * sh.bf[ax][2] / n2;
        for (int j = 0; j < nv; ++j) p.cB[ax * kMaxNv + j] = s_cB[ax][j];
    }
    __syncthreads();
    // (3) fixed-coefficient part of position / velocity / acceleration; positions
    //     are expressed relative to the start-goal midpoint (the origin)
    __shared__ double s_org[3];
    if (tid < 3) s_org[tid] = (tid < dims) ? 0.5 * (sh.b0[tid][0] + sh.bf[tid][0]) : 0.0;
    __syncthreads();
    if (tid < 3) tab64[lay.origin + tid] = s_org[tid];
    const int f1 = kFree0 + nf;  // first fixed coefficient at the final end
    for (int e = tid; e < 3 * np_ * dims; e += T) {
        const int t = e % np_, qa = e / np_, q = qa / dims, ax = qa - q * dims;  // e = (q * dims + ax) * np_ + t
        double s = 0.0;
        for (int j = 0; j < nv; ++j)
            if (j < kFree0 || j >= f1) s += bsrc[(q * np_ + t) * nv + j] * s_cB[ax][j];
        base[e] = (q == 0) ? s - s_org[ax] : s;
    }
    // (4) Gram blocks of the free coefficients: G_q = B_q,F^T B_q,F (once per shape)
    for (int e = tid; e < 3 * nf * nf; e += T) {
        const int q = e / (nf * nf), i = (e / nf) % nf, j = e % nf;
        double s;
        if (p.shape_ready) {
            s = gram[(q * kMaxNv + i) * kMaxNv + j];
        } else {
            s = 0.0;
            for (int t = 0; t < np_; ++t)
                s += bsrc[(q * np_ + t) * nv + kFree0 + i] * bsrc[(q * np_ + t) * nv + kFree0 + j];
            gram[(q * kMaxNv + i) * kMaxNv + j] = s;
        }
        s_G[q][i][j] = s;
    }
    __syncthreads();
    // (5) H = I + rho Q_FF with Q = n_obs P^T P + Pd^T Pd + Pdd^T Pdd (+ 2 P^T P with
    //     the workspace rows -P, +P of eq. bound_con); W = H^-1 by Gauss-Jordan
    //     (H is symmetric positive definite, so no pivoting is needed).
    const double wP = double(sh.n_obs) + (sh.use_bounds ? 2.0 : 0.0);
    for (int e = tid; e < nf * 2 * nf; e += T) {
        const int i = e / (2 * nf), j = e % (2 * nf);
        double v;
        if (j < nf)
            v = (i == j ? 1.0 : 0.0) + sh.rho * (wP * s_G[0][i][j] + s_G[1][i][j] + s_G[2][i][j]);
        else
            v = (j - nf == i) ? 1.0 : 0.0;
        s_M[i][j] = v;
    }
    if (tid == 0) s_flag = 1;
    __syncthreads();
    __shared__ double s_ipiv;
    for (int k = 0; k < nf; ++k) {
        if (tid < nf) s_fcol[tid] = s_M[tid][k];
        if (tid == 0) {
            const double piv = s_M[k][k];
            if (!(piv > 0.0)) s_flag = 0;
            s_ipiv = (piv > 0.0) ? rcp_any(piv) : 1.0;
        }
        __syncthreads();
        for (int j = tid; j < 2 * nf; j += T) s_M[k][j] *= s_ipiv;
        __syncthreads();
        for (int e = tid; e < nf * 2 * nf; e += T) {
            const int i = e / (2 * nf), j = e % (2 * nf);
            if (i != k) s_M[i][j] -= s_fcol[i] * s_M[k][j];
        }
        __syncthreads();
    }
    if (tid == 0 && !s_flag) atomicOr(p.status, kStatusKkt);
    for (int e = tid; e < nf * nf; e += T) W[e] = s_M[e / nf][nf + e % nf];
    // (6) obstacle records, centres relative to the origin.  The first four
    //     values feed a conservative pre-filter: with p the point and o the
    //     centre, |p|^2 - 2 p.o < a^2 - |o|^2 (+ margin) whenever the scaled
    //     distance is below one; the exact test follows only for candidates.
    //     2-D: [-2 o_x, -2 o_y, thr, a | 1/a, -o_x/a, -o_y/a, 0 | -v_x/a, -v_y/a, 0, 0]
    //     3-D (kappa = a^2/b^2): [-2 o_x, -2 o_y, -2 kappa o_z, thr | kappa, a, b, 0 |
    //          1/a, -o_x/a, -o_y/a, -o_z/b | 1/b, -v_x/a, -v_y/a, -v_z/b]
    //     thr = a^2 - (o_x^2 + o_y^2 + kappa o_z^2) + margin, the margin covering
    //     the rounding of the expanded form in the working precision.
    const int st = obs_stride(dims);
    const double eps = p.real_is_double ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
    for (int j = tid; j < sh.n_obs; j += T) {
        const double a = p.semi[2 * j], b = (dims == 3) ? p.semi[2 * j + 1] : a;
        const double ia = rcp_any(a), ib = rcp_any(b), kap = (a * a) * (ib * ib);
        double *o = obs + size_t(j) * st;
        const double *v = p.vel + j * dims;
        double c[3];
        for (int ax = 0; ax < 3; ++ax) c[ax] = (ax < dims) ? p.center[j * dims + ax] - s_org[ax] : 0.0;
        const double oo = c[0] * c[0] + c[1] * c[1] + (dims == 3 ? kap * c[2] * c[2] : 0.0);
        const double thr = a * a - oo + screen_margin(oo, a, kap, dims, eps);
        if (dims == 2) {
            o[0] = -2.0 * c[0]; o[1] = -2.0 * c[1]; o[2] = thr; o[3] = a;
            o[4] = ia; o[5] = -c[0] * ia; o[6] = -c[1] * ia; o[7] = 0.0;
            o[8] = -v[0] * ia; o[9] = -v[1] * ia; o[10] = 0.0; o[11] = 0.0;
        } else {
            o[0] = -2.0 * c[0]; o[1] = -2.0 * c[1]; o[2] = -2.0 * kap * c[2]; o[3] = thr;
            o[4] = kap; o[5] = a; o[6] = b; o[7] = 0.0;
            o[8] = ia; o[9] = -c[0] * ia; o[10] = -c[1] * ia; o[11] = -c[2] * ib;
            o[12] = ib; o[13] = -v[0] * ia; o[14] = -v[1] * ia; o[15] = -v[2] * ib;
        }
    }
    // (7) full solve: default mean (straight-line coefficients) / covariance
    //     and the first factor chol(Sigma_0 + chol_eps tr(Sigma_0)/D I)
    if (p.L) {
        const int D = sh.D;
        if (p.default_mu)
            for (int e = tid; e < D; e += T) {
                const int ax = e / nv, k = e % nv;
                p.mu[e] = sh.b0[ax][0] + (sh.bf[ax][0] - sh.b0[ax][0]) * double(k) / double(n);
            }
        if (p.default_cov)
            for (int e = tid; e < D * D; e += T)
                p.cov[e] = (e / D == e % D) ? p.init_std * p.init_std : 0.0;
        __syncthreads();
        __shared__ double s_tr;
        if (tid < 32) {
            double tr = 0.0;
            for (int i = tid; i < D; i += 32) tr += p.cov[i * D + i];
            for (int off = 16; off > 0; off >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, off);
            if (tid == 0) s_tr = p.chol_eps * tr * rcp_fast(double(D));
        }
        __syncthreads();
        const double eps = s_tr;
        for (int e = tid; e < D * D; e += T) s_dyn[e] = p.cov[e] + ((e / D == e % D) ? eps : 0.0);
        __syncthreads();
        const bool ok = block_cholesky(s_dyn, D, &s_flag);
        for (int e = tid; e < D * D; e += T) p.L[e] = s_dyn[e];
        if (tid == 0 && !ok) atomicOr(p.status, kStatusCholesky);
    }
    __syncthreads();
    // (8) working-precision copy of the tables; (9) the static-obstacle grid
    if (!p.real_is_double) {
        build_grid(p, s_org, reinterpret_cast<float *>(p.tab) + lay.grid, float(eps));
        if (p.shape_ready)
            write_tables<float>(p, tab64, lay.base, lay.total);  // basis and packed basis unchanged
        else
            write_tables<float>(p, tab64, 0, lay.total);
    }
}

__global__ void __launch_bounds__(kSetupThreads) setup_kernel(SetupParams p, double *tab64)
{
    pdl_trigger();
    pdl_wait();
    setup_body(p, tab64);
}

// One CTA per problem.
__global__ void __launch_bounds__(kSetupThreads) setup_batch_kernel(const SetupParams *ps)
{
    const SetupParams p = ps[blockIdx.x];
    setup_body(p, p.tab64);
}

size_t setup_smem(const Shape &sh)
{
    const size_t nbasis = size_t(3) * sh.n_p * sh.nv * sizeof(double);
    return size_t(sh.D) * sh.D * sizeof(double) + (nbasis <= kSetupBasisSmem ? nbasis : 0);
}

}  // namespace

cudaError_t launch_setup_batch(const SetupParams *ps_dev, int n, size_t smem, cudaStream_t st)
{
    static size_t granted = 0;
    cudaError_t e = reserve_smem(setup_batch_kernel, smem, granted);
    if (e != cudaSuccess) return e;
    setup_batch_kernel<<<n, kSetupThreads, smem, st>>>(ps_dev);
    return cudaGetLastError();
}

size_t setup_smem_bytes(const Shape &sh) { return setup_smem(sh); }

cudaError_t launch_setup(const SetupParams &p, cudaStream_t st)
{
    const size_t nbasis = size_t(3) * p.sh.n_p * p.sh.nv * sizeof(double);
    const size_t dyn = size_t(p.sh.D) * p.sh.D * sizeof(double) + (nbasis <= kSetupBasisSmem ? nbasis : 0);
    static size_t granted = 0;
    cudaError_t e = reserve_smem(setup_kernel, dyn, granted);
    if (e != cudaSuccess) return e;
    setup_kernel<<<1, kSetupThreads, dyn, st>>>(p, p.tab64);
    return cudaGetLastError();
}

}  // namespace priest
