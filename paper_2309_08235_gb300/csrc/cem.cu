// cem.cu -- the CEM stages of Alg. 1 around the projection:
//   a10 ConstraintEliteSet (N_proj least r) and EliteSet (N_elite least
//       c_aug = c_1 + r among them), ties to the lower sample index, by a
//       bitonic sort whose short-stride stages run inside a warp on shuffles;
//   a11 MPPI-like refit (eqs. update_mean, update_covariance) in FP64 with
//       weights exp(-(c_aug - delta)/gamma), delta = min c_aug;
//   a12 the next sampling factor chol(Sigma' + eps I), eps = chol_eps tr(Sigma')/D,
//       by the last CTA of the refit grid.
#include "block_linalg.cuh"
#include "priest_internal.cuh"

namespace priest {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSelectThreads = 1024;
constexpr int kRefitThreads = 128;

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

__global__ void __launch_bounds__(kSelectThreads)
    select_kernel(int N, const double *r, const double *c1, int n_proj, int n_elite, int *elite_idx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int n2 = 32;
    while (n2 < N) n2 <<= 1;
    unsigned long long *key = reinterpret_cast<unsigned long long *>(smem_raw);
    int *idx = reinterpret_cast<int *>(key + n2);
    const int tid = threadIdx.x, T = blockDim.x;
    // ConstraintEliteSet: sort by (r, index)
    for (int e = tid; e < n2; e += T) {
        key[e] = (e < N) ? order_key(r[e]) : ~0ull;
        idx[e] = e;
    }
    bitonic_sort(key, idx, n2);
    // EliteSet: the first n_proj re-keyed by c_aug = c_1 + r
    int m2 = 32;
    while (m2 < n_proj) m2 <<= 1;
    for (int e = tid; e < m2; e += T) {
        if (e < n_proj) {
            const int i = idx[e];
            key[e] = order_key(c1[i] + r[i]);
        } else {
            key[e] = ~0ull;
            idx[e] = 0x7fffffff;
        }
    }
    bitonic_sort(key, idx, m2);
    for (int e = tid; e < n_elite; e += T) elite_idx[e] = idx[e];
}

__global__ void __launch_bounds__(kRefitThreads)
    refit_kernel(int D, const double *xb, const double *r, const double *c1, const int *elite, int n_elite,
                 double sigma, double gamma, double chol_eps, double *mu, double *cov, double *mu_new,
                 double *Lout, unsigned *counter, int *status, double *best_out)
{
    extern __shared__ __align__(16) double s_dyn[];
    double *w = s_dyn;                 // n_elite
    double *mnew = w + n_elite;        // D
    double *A = mnew + D;              // D x D (last CTA)
    __shared__ double s_red[kRefitThreads / 32];
    __shared__ double s_sw;
    __shared__ int s_last, s_flag;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int row = blockIdx.x;

    // weights: elites are sorted by c_aug, so delta = c_aug of the first
    const int e0 = elite[0];
    const double delta = c1[e0] + r[e0];
    double part = 0.0;
    for (int m = tid; m < n_elite; m += T) {
        const int i = elite[m];
        const double wm = exp(-((c1[i] + r[i]) - delta) / gamma);
        w[m] = wm;
        part += wm;
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(kFull, part, off);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    if (tid == 0) {
        double sw = 0.0;
        for (int k = 0; k < T / 32; ++k) sw += s_red[k];
        s_sw = sw;
    }
    __syncthreads();
    const double sw = s_sw;
    // new mean (eq. update_mean); every CTA forms it, CTA 0 publishes it
    for (int d = tid; d < D; d += T) {
        double s = 0.0;
        for (int m = 0; m < n_elite; ++m) s += w[m] * xb[size_t(elite[m]) * D + d];
        mnew[d] = (1.0 - sigma) * mu[d] + sigma * (s / sw);
    }
    __syncthreads();
    // row `row` of the new covariance (eq. update_covariance, around the new mean)
    for (int j = tid; j < D; j += T) {
        double s = 0.0;
        for (int m = 0; m < n_elite; ++m) {
            const double *x = xb + size_t(elite[m]) * D;
            s += w[m] * ((x[row] - mnew[row]) * (x[j] - mnew[j]));
        }
        cov[row * D + j] = (1.0 - sigma) * cov[row * D + j] + sigma * (s / sw);
    }
    if (row == 0)
        for (int d = tid; d < D; d += T) mu_new[d] = mnew[d];
    // last CTA: publish the mean, factor the new covariance, write the best elite
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int d = tid; d < D; d += T) mu[d] = mu_new[d];
    __shared__ double s_tr;
    if (tid == 0) {
        double tr = 0.0;
        for (int i = 0; i < D; ++i) tr += cov[i * D + i];
        s_tr = tr;
    }
    __syncthreads();
    const double eps = chol_eps * s_tr / double(D);
    for (int e = tid; e < D * D; e += T) A[e] = cov[e] + ((e / D == e % D) ? eps : 0.0);
    __syncthreads();
    const bool ok = block_cholesky(A, D, &s_flag);
    for (int e = tid; e < D * D; e += T) Lout[e] = A[e];
    if (tid == 0) {
        if (!ok) atomicOr(status, kStatusCholesky);
        *counter = 0u;
    }
    for (int d = tid; d < D; d += T) best_out[d] = xb[size_t(e0) * D + d];
    if (tid == 0) {
        best_out[D] = r[e0];
        best_out[D + 1] = c1[e0];
        best_out[D + 2] = c1[e0] + r[e0];
        best_out[D + 3] = double(e0);
    }
}

}  // namespace

cudaError_t launch_select(int N, const double *r, const double *c1, int n_proj, int n_elite, int *elite_idx,
                          cudaStream_t st)
{
    int n2 = 32;
    while (n2 < N) n2 <<= 1;
    const size_t smem = size_t(n2) * (sizeof(unsigned long long) + sizeof(int));
    static size_t granted = 0;
    cudaError_t e = reserve_smem(select_kernel, smem, granted);
    if (e != cudaSuccess) return e;
    select_kernel<<<1, kSelectThreads, smem, st>>>(N, r, c1, n_proj, n_elite, elite_idx);
    return cudaGetLastError();
}

cudaError_t launch_refit(int D, const double *xb, const double *r, const double *c1, const int *elite,
                         int n_elite, double sigma, double gamma, double chol_eps, double *mu, double *cov,
                         double *mu_new, double *L, unsigned *counter, int *status, double *best_out,
                         cudaStream_t st)
{
    const size_t smem = (size_t(n_elite) + D + size_t(D) * D) * sizeof(double);
    static size_t granted = 0;
    cudaError_t e = reserve_smem(refit_kernel, smem, granted);
    if (e != cudaSuccess) return e;
    refit_kernel<<<D, kRefitThreads, smem, st>>>(D, xb, r, c1, elite, n_elite, sigma, gamma, chol_eps, mu, cov,
                                                  mu_new, L, counter, status, best_out);
    return cudaGetLastError();
}

}  // namespace priest
