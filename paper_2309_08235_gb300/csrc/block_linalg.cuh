// block_linalg.cuh -- small FP64 dense factorisations run by one CTA.
//
// FP64 issues slowly on this part, so the serial chain is kept short: square
// roots and reciprocals start from the FP32 hardware estimate and are refined
// by Newton-Raphson steps in FP64 (each step doubles the correct bits:
// 2^-23 -> 2^-46 -> beyond FP64), and per-column scalars are formed by one
// thread and shared.
#pragma once

#include <cuda_runtime.h>

namespace priest {

// The FP32 estimate needs x inside the FP32 normal range; outside it the
// plain FP64 operation is used.
__device__ __forceinline__ bool fp32_range(double x)
{
    const double ax = fabs(x);
    return ax > 1e-30 && ax < 1e30;
}

// 1/sqrt(x) for x > 0: FP32 estimate, then y <- y (3 - x y^2) / 2 twice.
__device__ __forceinline__ double rsqrt_nr(double x)
{
    if (!fp32_range(x)) return 1.0 / sqrt(x);
    double y = double(rsqrtf(float(x)));
    y = y * (1.5 - 0.5 * x * y * y);
    y = y * (1.5 - 0.5 * x * y * y);
    return y;
}

// 1/x for x != 0: FP32 estimate, then y <- y (2 - x y) twice.
__device__ __forceinline__ double rcp_nr(double x)
{
    if (!fp32_range(x)) return 1.0 / x;
    double y = double(1.0f / float(x));
    y = y * (2.0 - x * y);
    y = y * (2.0 - x * y);
    return y;
}

// In-place Cholesky of the D x D symmetric matrix A (row-major, shared
// memory): on return the lower triangle holds L with A = L L^T and the strict
// upper triangle is zeroed.  Right-looking: per column one square root, a
// parallel scaling of the column and a parallel rank-1 update of the trailing
// lower triangle.  Returns false (to every thread) on a non-positive pivot.
// All threads of the CTA call it.
__device__ inline bool block_cholesky(double *A, int D, int *flag_smem)
{
    __shared__ double s_inv;
    const int tid = threadIdx.x, T = blockDim.x;
    if (tid == 0) *flag_smem = 1;
    __syncthreads();
    for (int j = 0; j < D; ++j) {
        if (tid == 0) {
            double s = A[j * D + j];
            if (!(s > 0.0) || !(s < 1e300)) {
                *flag_smem = 0;
                s = 1.0;
            }
            const double y = rsqrt_nr(s);
            A[j * D + j] = s * y;  // sqrt(s)
            s_inv = y;             // 1 / sqrt(s)
        }
        __syncthreads();
        const double inv = s_inv;
        for (int i = j + 1 + tid; i < D; i += T) A[i * D + j] *= inv;
        __syncthreads();
        // trailing update A[i][k] -= L[i][j] L[k][j] for j < k <= i
        const int m = D - j - 1;
        for (int e = tid; e < m * m; e += T) {
            const int i = j + 1 + e / m, k = j + 1 + e % m;
            if (k <= i) A[i * D + k] -= A[i * D + j] * A[k * D + j];
        }
        __syncthreads();
    }
    for (int e = tid; e < D * D; e += T)
        if ((e % D) > (e / D)) A[e] = 0.0;
    __syncthreads();
    return *flag_smem != 0;
}

}  // namespace priest
