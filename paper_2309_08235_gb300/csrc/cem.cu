// cem.cu -- the CEM stages of Alg. 1 around the projection:
//   a10 ConstraintEliteSet (N_proj least r) and EliteSet (N_elite least
//       c_aug = c_1 + r among them), ties to the lower sample index: each set
//       by a bitwise threshold search (one block count per key bit), then a
//       bitonic sort of the N_elite survivors whose short-stride stages run
//       inside a warp on shuffles;
//   a11 MPPI-like refit (eqs. update_mean, update_covariance) in FP64 with
//       weights exp(-(c_aug - delta)/gamma), delta = min c_aug;
//   a12 the next sampling factor chol(Sigma' + eps I), eps = chol_eps tr(Sigma')/D,
//       by the last CTA of the refit grid.
#include <algorithm>

#include "block_linalg.cuh"
#include "priest_internal.cuh"

namespace priest {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSelectThreads = 1024;
constexpr int kRefitThreads = 256;

// Order-preserving map of an FP64 key to uint64 (NaN sorts after +inf).
__device__ __forceinline__ unsigned long long order_key(double x)
{
    long long b = __double_as_longlong(x);
    return (b < 0) ? ~static_cast<unsigned long long>(b) : (static_cast<unsigned long long>(b) | 0x8000000000000000ull);
}

__device__ __forceinline__ bool key_less(unsigned long long ka, int ia, unsigned long long kb, int ib)
{
    return ka < kb || (ka == kb && ia < ib);
}

// Ascending bitonic sort of n2 (power of two, >= 32) (key, index) pairs in
// shared memory.  Stages with partner distance >= 32 exchange through shared
// memory; the remaining stages of each merge run in registers with
// __shfl_xor_sync, one element per lane.
__device__ void bitonic_sort(unsigned long long *key, int *idx, int n2)
{
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31;
    for (int k = 2; k <= n2; k <<= 1) {
        int j = k >> 1;
        for (; j >= 32; j >>= 1) {
            __syncthreads();
            for (int e = tid; e < n2; e += T) {
                const int q = e ^ j;
                if (q > e) {
                    const bool asc = (e & k) == 0;
                    const unsigned long long ke = key[e], kq = key[q];
                    const int ie = idx[e], iq = idx[q];
                    const bool swap = asc ? key_less(kq, iq, ke, ie) : key_less(ke, ie, kq, iq);
                    if (swap) {
                        key[e] = kq;
                        key[q] = ke;
                        idx[e] = iq;
                        idx[q] = ie;
                    }
                }
            }
        }
        __syncthreads();
        // remaining distances j < 32: within aligned 32-element blocks
        for (int base = tid - lane; base < n2; base += T) {
            const int e = base + lane;
            unsigned long long ke = key[e];
            int ie = idx[e];
            const bool asc = (e & k) == 0;
            for (int jj = j; jj > 0; jj >>= 1) {
                const unsigned long long ko = __shfl_xor_sync(kFull, ke, jj);
                const int io = __shfl_xor_sync(kFull, ie, jj);
                const bool lower = (lane & jj) == 0;
                // lower element of the pair keeps the min when ascending
                const bool other_first = key_less(ko, io, ke, ie);
                const bool take = (lower == asc) ? other_first : !other_first;
                if (take) {
                    ke = ko;
                    ie = io;
                }
            }
            key[e] = ke;
            idx[e] = ie;
        }
        __syncthreads();
    }
}

__host__ __device__ inline int pow2_at_least(int n)
{
    int n2 = 32;
    while (n2 < n) n2 <<= 1;
    return n2;
}

// Number of elements over the block for which this thread counted c (one
// barrier).  Per-warp sums go to one of three counters by call parity: the
// counter of call n + 2 is cleared after the barrier of call n, when every
// read of it (call n - 1) is done.
__device__ __forceinline__ int block_count(int c, int *s_cnt, int &calls)
{
    const int w = __reduce_add_sync(kFull, c);
    const int slot = calls % 3;
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_cnt[slot], w);
    __syncthreads();
    const int total = s_cnt[slot];
    if (threadIdx.x == 0) s_cnt[(slot + 2) % 3] = 0;
    ++calls;
    return total;
}

// Exclusive prefix count of pred in thread order, and its total (two barriers).
__device__ __forceinline__ int block_scan(bool pred, int *s_warp, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned b = __ballot_sync(kFull, pred);
    if (lane == 0) s_warp[warp] = __popc(b);
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
        const int c = s_warp[w];
        before += (w < warp) ? c : 0;
        tot += c;
    }
    __syncthreads();
    total = tot;
    return before + __popc(b & ((1u << lane) - 1u));
}

// The k-th least key (1 <= k <= number of eligible elements) among the
// eligible elements of the block, and lt = how many eligible keys are below
// it.  Thread tid holds elements tid + e T (e < E, bit e of `elig`); the key of
// e = 0 is k0, the others are in keys[].  Bitwise: t is the largest value with
// #(key < t) < k, formed from the top bit down, one block count per bit.  The
// high word first; when the eligible keys with that high word share one low
// word (a lone key, or exact ties such as r = 0), that is the answer.
__device__ unsigned long long kth_key(const unsigned long long *keys, unsigned long long k0, unsigned elig, int E,
                                      int k, int *s_cnt, int &calls, unsigned *s_mm, int &lt)
{
    const int tid = threadIdx.x, T = blockDim.x;
    auto count_below = [&](unsigned long long trial) -> int {
        if (E == 1) return __syncthreads_count((elig & 1u) && k0 < trial);
        int c = 0;
        for (int e = 0; e < E; ++e)
            if ((elig >> e) & 1u) c += ((e == 0) ? k0 : keys[tid + e * T]) < trial;
        return block_count(c, s_cnt, calls);
    };
    unsigned long long t = 0;
    lt = 0;
    for (int b = 63; b >= 32; --b) {
        const unsigned long long trial = t | (1ull << b);
        const int c = count_below(trial);
        if (c < k) {
            t = trial;
            lt = c;
        }
    }
    for (int e = 0; e < E; ++e)
        if ((elig >> e) & 1u) {
            const unsigned long long v = (e == 0) ? k0 : keys[tid + e * T];
            if ((v >> 32) == (t >> 32)) {
                atomicMin(&s_mm[0], unsigned(v));
                atomicMax(&s_mm[1], unsigned(v));
            }
        }
    __syncthreads();
    if (s_mm[0] == s_mm[1]) return t | s_mm[0];
    for (int b = 31; b >= 0; --b) {
        const unsigned long long trial = t | (1ull << b);
        const int c = count_below(trial);
        if (c < k) {
            t = trial;
            lt = c;
        }
    }
    return t;
}

// ConstraintEliteSet: the n_proj least (r, index); EliteSet: the n_elite least
// (c_aug, index) among them, written in ascending order.  Each set is found by
// its threshold (kth_key) and the ties at the threshold taken by index, then
// the n_elite survivors are sorted (bitonic, padding entries carry the largest
// key and index).
__device__ void select_body(int N, const double *r, const double *c1, int n_proj, int n_elite, int *elite_idx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, T = blockDim.x, E = (N + T - 1) / T;
    const int n2e = pow2_at_least(n_elite);
    unsigned long long *key1 = reinterpret_cast<unsigned long long *>(smem_raw);  // N: order_key(r)
    unsigned long long *key2 = key1 + N;                                           // N: order_key(c_aug)
    unsigned long long *keyE = key2 + N;                                           // n2e
    int *idxE = reinterpret_cast<int *>(keyE + n2e);                               // n2e
    __shared__ int s_cnt[3], s_warp[32];
    __shared__ unsigned s_mm[4];
    if (tid < 3) s_cnt[tid] = 0;
    if (tid < 4) s_mm[tid] = (tid & 1) ? 0u : ~0u;
    unsigned long long k01 = ~0ull, k02 = ~0ull;
    unsigned valid = 0;
    for (int e = 0; e < E; ++e) {
        const int i = tid + e * T;
        if (i < N) {
            const double ri = r[i];
            const unsigned long long a = order_key(ri), b = order_key(c1[i] + ri);
            key1[i] = a;
            key2[i] = b;
            if (e == 0) {
                k01 = a;
                k02 = b;
            }
            valid |= 1u << e;
        }
    }
    __syncthreads();
    int calls = 0, lt = 0, base = 0, tot = 0;
    // ConstraintEliteSet
    const unsigned long long t1 = kth_key(key1, k01, valid, E, n_proj, s_cnt, calls, s_mm, lt);
    const int need1 = n_proj - lt;
    unsigned in1 = 0;
    for (int e = 0; e < E; ++e) {
        const unsigned long long v = (e == 0) ? k01 : (((valid >> e) & 1u) ? key1[tid + e * T] : ~0ull);
        const bool tie = ((valid >> e) & 1u) && v == t1;
        const int rank = base + block_scan(tie, s_warp, tot);
        base += tot;
        if (((valid >> e) & 1u) && (v < t1 || (tie && rank < need1))) in1 |= 1u << e;
    }
    // EliteSet among them
    const unsigned long long t2 = kth_key(key2, k02, in1, E, n_elite, s_cnt, calls, s_mm + 2, lt);
    const int need2 = n_elite - lt;
    base = 0;
    unsigned el = 0;
    for (int e = 0; e < E; ++e) {
        const unsigned long long v = (e == 0) ? k02 : (((in1 >> e) & 1u) ? key2[tid + e * T] : ~0ull);
        const bool tie = ((in1 >> e) & 1u) && v == t2;
        const int rank = base + block_scan(tie, s_warp, tot);
        base += tot;
        if (((in1 >> e) & 1u) && (v < t2 || (tie && rank < need2))) el |= 1u << e;
    }
    // compact the elites (index order), then sort them by (c_aug, index)
    base = 0;
    for (int e = 0; e < E; ++e) {
        const bool m = (el >> e) & 1u;
        const int pos = base + block_scan(m, s_warp, tot);
        base += tot;
        if (m) {
            keyE[pos] = (e == 0) ? k02 : key2[tid + e * T];
            idxE[pos] = tid + e * T;
        }
    }
    for (int p = n_elite + tid; p < n2e; p += T) {
        keyE[p] = ~0ull;
        idxE[p] = 0x7fffffff;
    }
    bitonic_sort(keyE, idxE, n2e);
    for (int e = tid; e < n_elite; e += T) elite_idx[e] = idxE[e];
}

__global__ void __launch_bounds__(kSelectThreads)
    select_kernel(int N, const double *r, const double *c1, int n_proj, int n_elite, int *elite_idx)
{
    pdl_trigger();
    pdl_wait();
    select_body(N, r, c1, n_proj, n_elite, elite_idx);
}

__global__ void __launch_bounds__(kSelectThreads) select_batch_kernel(const CemArgs *args)
{
    const CemArgs a = args[blockIdx.x];
    select_body(a.N, a.r, a.c1, a.n_proj, a.n_elite, a.elite);
}

// Elite rows staged in shared memory per chunk (all of them when they fit).
constexpr int kRefitChunkBytes = 96 * 1024;

// Dynamic shared memory the refit plans for: the per-elite arrays (weights,
// pre-weighted row entries: 8 + 8 bytes; indices: 4 bytes), the mean and
// the partial sums, and a staging area for a chunk of elite rows.
constexpr int kRefitSmemBudget = 200 * 1024;

// Elite rows staged per chunk: all of them when they fit in kRefitChunkBytes
// and in what the other arrays leave of kRefitSmemBudget.
__host__ __device__ inline int refit_chunk(int D, int n_elite)
{
    const int row = int(sizeof(double)) * D;
    const int room = (kRefitSmemBudget - 20 * n_elite - int(sizeof(double)) * (D + kRefitThreads)) / row;
    int c = kRefitChunkBytes / row;
    c = c < room ? c : room;
    c = c < n_elite ? c : n_elite;
    return c < 1 ? 1 : c;
}

// Doubles of the staging area: a chunk of elite rows, or the D x D matrix
// the last CTA factors.
__host__ __device__ inline int refit_stage_doubles(int D, int n_elite)
{
    const int c = refit_chunk(D, n_elite);
    return c * D > D * D ? c * D : D * D;
}

// Elite rows gathered per batch of loads in flight per thread.
constexpr int kStageBatch = 12;

// Row `row` of the refit of one problem; the last of its D CTAs (counted on
// *counter) publishes the mean, factors the covariance and writes the best elite.
// Global reads are grouped so that each phase waits for one round trip: the
// elite indices first (to shared memory), then the costs and the elite rows.
__device__ void refit_body(int D, int row, const double *xb, const double *r, const double *c1, const int *elite,
                           int n_elite, double sigma, double gamma, double chol_eps, double *mu, double *cov,
                           double *mu_new, double *Lout, unsigned *counter, int *status, double *best_out)
{
    extern __shared__ __align__(16) double s_dyn[];
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const int chunk = refit_chunk(D, n_elite);
    double *w = s_dyn;                 // n_elite weights
    double *wr = w + n_elite;          // n_elite: w_m (x_m,row - mu'_row)
    double *mnew = wr + n_elite;       // D
    double *part = mnew + D;           // T partial sums
    double *xe = part + T;             // chunk x D staged elite rows
    double *A = xe;                    // D x D (last CTA, reuses the staging area)
    int *eidx = reinterpret_cast<int *>(xe + refit_stage_doubles(D, n_elite));  // n_elite
    __shared__ double s_red[kRefitThreads / 32];
    __shared__ double s_isw, s_eps;
    __shared__ int s_last, s_flag;

    for (int m = tid; m < n_elite; m += T) eidx[m] = elite[m];
    double mu_t = 0.0, cov_t = 0.0;
    if (tid < D) {
        mu_t = mu[tid];
        cov_t = cov[row * D + tid];
    }
    __syncthreads();
    // elite rows m0 .. m0 + mc - 1 into xe (row-major), kStageBatch loads in
    // flight per thread; element e of the chunk is row e / D, column e % D
    auto stage = [&](int m0, int mc) {
        const int total = mc * D, dm = T / D, dq = T - dm * D;
        int m = tid / D, q = tid - (tid / D) * D;
        for (int e = tid; e < total; e += kStageBatch * T) {
            double v[kStageBatch];
#pragma unroll
            for (int u = 0; u < kStageBatch; ++u) {
                if (e + u * T < total) v[u] = xb[size_t(eidx[m0 + m]) * D + q];
                m += dm;
                q += dq;
                if (q >= D) {
                    q -= D;
                    ++m;
                }
            }
#pragma unroll
            for (int u = 0; u < kStageBatch; ++u)
                if (e + u * T < total) xe[e + u * T] = v[u];
        }
    };
    // weights w_m = exp(-(c_aug_m - delta) / gamma); the elites are sorted by
    // c_aug, so delta is the first one's.  The first T costs are loaded before
    // the staging so that both wait on the same round trip.
    const int e0 = eidx[0];
    const double c0 = c1[e0], r0 = r[e0];
    double cw = 0.0, rw = 0.0;
    if (tid < n_elite) {
        const int i = eidx[tid];
        cw = c1[i];
        rw = r[i];
    }
    stage(0, min(chunk, n_elite));
    double psum = 0.0;
    if (tid < n_elite) {
        const double delta = c0 + r0;
        const double ig = rcp_any(gamma);
        double wm = exp(-((cw + rw) - delta) * ig);
        w[tid] = wm;
        psum = wm;
        for (int m = tid + T; m < n_elite; m += T) {
            const int i = eidx[m];
            wm = exp(-((c1[i] + r[i]) - delta) * ig);
            w[m] = wm;
            psum += wm;
        }
    }
    for (int off = 16; off > 0; off >>= 1) psum += __shfl_xor_sync(kFull, psum, off);
    if (lane == 0) s_red[warp] = psum;
    __syncthreads();
    // 1 / (sum of the weights) on warp 0, beside pass 1
    if (warp == 0) {
        double sw = lane < nw ? s_red[lane] : 0.0;
        for (int off = kRefitThreads / 64; off > 0; off >>= 1) sw += __shfl_xor_sync(kFull, sw, off);
        if (lane == 0) s_isw = rcp_any(sw);
    }
    // thread (d, slice): column d, elites m = slice, slice + nslice, ...
    const int nslice = max(1, T / D);
    const int d = tid % D, slice = tid / D;
    const bool worker = slice < nslice;
    // pass 1: new mean (eq. update_mean); every CTA forms it, CTA 0 publishes it
    double acc = 0.0;
    for (int m0 = 0; m0 < n_elite; m0 += chunk) {
        const int mc = min(chunk, n_elite - m0);
        if (m0 > 0) {
            __syncthreads();
            stage(m0, mc);
            __syncthreads();
        }
        if (worker)
            for (int m = slice; m < mc; m += nslice) acc = fma(w[m0 + m], xe[m * D + d], acc);
    }
    part[tid] = worker ? acc : 0.0;
    __syncthreads();
    const double isw = s_isw;
    if (tid < D) {
        double s = 0.0;
        for (int k = 0; k < nslice; ++k) s += part[k * D + tid];
        mnew[tid] = (1.0 - sigma) * mu_t + sigma * (s * isw);
    }
    __syncthreads();
    // pass 2: row `row` of the new covariance (eq. update_covariance, around
    // the new mean), with w_m (x_m,row - mu'_row) formed once per elite
    acc = 0.0;
    const double mrow = mnew[row], md = mnew[d];
    for (int m0 = 0; m0 < n_elite; m0 += chunk) {
        const int mc = min(chunk, n_elite - m0);
        if (m0 > 0 || chunk < n_elite) {
            __syncthreads();
            stage(m0, mc);
            __syncthreads();
        }
        for (int m = tid; m < mc; m += T) wr[m0 + m] = w[m0 + m] * (xe[m * D + row] - mrow);
        __syncthreads();
        if (worker)
            for (int m = slice; m < mc; m += nslice) acc = fma(wr[m0 + m], xe[m * D + d] - md, acc);
    }
    part[tid] = worker ? acc : 0.0;
    __syncthreads();
    if (tid < D) {
        double s = 0.0;
        for (int k = 0; k < nslice; ++k) s += part[k * D + tid];
        cov[row * D + tid] = (1.0 - sigma) * cov_t + sigma * (s * isw);
    }
    if (row == 0)
        for (int q = tid; q < D; q += T) mu_new[q] = mnew[q];
    // last CTA: publish the mean, write the best elite, factor the new covariance
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(counter, 1u) == unsigned(D) - 1u);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int q = tid; q < D; q += T) {
        mu[q] = mnew[q];  // every CTA formed the same mean
        best_out[q] = (chunk >= n_elite) ? xe[q] : xb[size_t(e0) * D + q];
    }
    if (tid == 0) {
        best_out[D] = r0;
        best_out[D + 1] = c0;
        best_out[D + 2] = c0 + r0;
        best_out[D + 3] = double(e0);
    }
    __syncthreads();
    for (int i = warp; i < D; i += nw)
        for (int k = lane; k < D; k += 32) A[i * D + k] = __ldcg(cov + i * D + k);
    __syncthreads();
    // eps = chol_eps tr(Sigma') / D on the diagonal
    if (warp == 0) {
        double tr = 0.0;
        for (int i = lane; i < D; i += 32) tr += A[i * D + i];
        for (int off = 16; off > 0; off >>= 1) tr += __shfl_xor_sync(kFull, tr, off);
        if (lane == 0) s_eps = chol_eps * tr * rcp_fast(double(D));
    }
    __syncthreads();
    for (int i = tid; i < D; i += T) A[i * D + i] += s_eps;
    __syncthreads();
    const bool ok = block_cholesky(A, D, &s_flag);
    for (int e = tid; e < D * D; e += T) Lout[e] = A[e];
    if (tid == 0) {
        if (!ok) atomicOr(status, kStatusCholesky);
        *counter = 0u;
    }
}

__global__ void __launch_bounds__(kRefitThreads)
    refit_kernel(int D, const double *xb, const double *r, const double *c1, const int *elite, int n_elite,
                 double sigma, double gamma, double chol_eps, double *mu, double *cov, double *mu_new,
                 double *Lout, unsigned *counter, int *status, double *best_out)
{
    pdl_trigger();
    pdl_wait();
    refit_body(D, blockIdx.x, xb, r, c1, elite, n_elite, sigma, gamma, chol_eps, mu, cov, mu_new, Lout, counter,
               status, best_out);
}

// grid (max D, problems): CTAs past their problem's D return at once.
__global__ void __launch_bounds__(kRefitThreads) refit_batch_kernel(const CemArgs *args)
{
    const CemArgs a = args[blockIdx.y];
    if (int(blockIdx.x) >= a.D) return;
    refit_body(a.D, blockIdx.x, a.xb, a.r, a.c1, a.elite, a.n_elite, a.sigma, a.gamma, a.chol_eps, a.mu, a.cov,
               a.mu_new, a.L, a.counter, a.status, a.best_out);
}

// Diagnostic: block_cholesky on one CTA of any width (the refit runs it on
// 256 threads, the setup on 512).
__global__ void chol_selftest_kernel(double *A, int D, int *ok)
{
    extern __shared__ __align__(16) double s_a[];
    __shared__ int s_flag;
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) s_a[e] = A[e];
    __syncthreads();
    const bool good = block_cholesky(s_a, D, &s_flag);
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) A[e] = s_a[e];
    if (threadIdx.x == 0) *ok = good ? 1 : 0;
}

size_t refit_smem(int D, int n_elite)
{
    return (2 * size_t(n_elite) + D + kRefitThreads + refit_stage_doubles(D, n_elite)) * sizeof(double) +
           size_t(n_elite) * sizeof(int);
}

}  // namespace

size_t select_smem_bytes(int N)
{
    return 2 * size_t(N) * sizeof(unsigned long long) + size_t(pow2_at_least(N)) * (sizeof(unsigned long long) + sizeof(int));
}
size_t refit_smem_bytes(int D, int n_elite) { return refit_smem(D, n_elite); }

cudaError_t launch_select_batch(const CemArgs *args_dev, int n, size_t smem, cudaStream_t st)
{
    static size_t granted = 0;
    cudaError_t e = reserve_smem(select_batch_kernel, smem, granted);
    if (e != cudaSuccess) return e;
    select_batch_kernel<<<n, kSelectThreads, smem, st>>>(args_dev);
    return cudaGetLastError();
}

cudaError_t launch_refit_batch(const CemArgs *args_dev, int n, int D_max, size_t smem, cudaStream_t st)
{
    static size_t granted = 0;
    cudaError_t e = reserve_smem(refit_batch_kernel, smem, granted);
    if (e != cudaSuccess) return e;
    refit_batch_kernel<<<dim3(D_max, n), kRefitThreads, smem, st>>>(args_dev);
    return cudaGetLastError();
}

cudaError_t launch_select(int N, const double *r, const double *c1, int n_proj, int n_elite, int *elite_idx,
                          cudaStream_t st)
{
    const size_t smem = select_smem_bytes(N);
    static size_t granted = 0;
    cudaError_t e = reserve_smem(select_kernel, smem, granted);
    if (e != cudaSuccess) return e;
    return launch_pdl(select_kernel, dim3(1), dim3(kSelectThreads), smem, st, N, r, c1, n_proj, n_elite, elite_idx);
}

cudaError_t launch_refit(int D, const double *xb, const double *r, const double *c1, const int *elite,
                         int n_elite, double sigma, double gamma, double chol_eps, double *mu, double *cov,
                         double *mu_new, double *L, unsigned *counter, int *status, double *best_out,
                         cudaStream_t st)
{
    const size_t smem = refit_smem(D, n_elite);
    static size_t granted = 0;
    cudaError_t e = reserve_smem(refit_kernel, smem, granted);
    if (e != cudaSuccess) return e;
    return launch_pdl(refit_kernel, dim3(D), dim3(kRefitThreads), smem, st, D, xb, r, c1, elite, n_elite, sigma,
                      gamma, chol_eps, mu, cov, mu_new, L, counter, status, best_out);
}

}  // namespace priest

using namespace priest;

extern "C" priest_status priest_chol_selftest(int D, int threads, const double *a_host, double *l_host)
{
    if (D < 1 || D > PRIEST_MAX_D || threads < 32 || threads > 1024 || threads % 32 || !a_host || !l_host)
        return PRIEST_ERR_INVALID;
    const size_t bytes = sizeof(double) * D * D;
    double *A = nullptr;
    int *ok = nullptr;
    cudaError_t e = cudaMalloc(&A, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&ok, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(A, a_host, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ok, 0, sizeof(int));
    if (e == cudaSuccess) {
        chol_selftest_kernel<<<1, threads, bytes>>>(A, D, ok);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int hok = 0;
    if (e == cudaSuccess) e = cudaMemcpy(l_host, A, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hok, ok, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(A);
    cudaFree(ok);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PRIEST_ERR_CUDA;
    }
    return hok ? PRIEST_OK : PRIEST_ERR_NUMERIC;
}
