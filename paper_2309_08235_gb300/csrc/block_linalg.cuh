// block_linalg.cuh -- small FP64 dense factorisations run by one CTA.
#pragma once

#include <cuda_runtime.h>

namespace priest {

// In-place Cholesky of the D x D symmetric matrix A (row-major, shared
// memory): on return the lower triangle holds L with A = L L^T and the strict
// upper triangle is zeroed.  Right-looking: per column one square root, a
// parallel scaling of the column and a parallel rank-1 update of the trailing
// lower triangle, so the serial chain is one sqrt and one division per
// column.  Returns false (to every thread) on a non-positive pivot.  All
// threads of the CTA call it.
__device__ inline bool block_cholesky(double *A, int D, int *flag_smem)
{
    const int tid = threadIdx.x, T = blockDim.x;
    if (tid == 0) *flag_smem = 1;
    __syncthreads();
    for (int j = 0; j < D; ++j) {
        if (tid == 0) {
            double s = A[j * D + j];
            if (!(s > 0.0)) {
                *flag_smem = 0;
                s = 1.0;
            }
            A[j * D + j] = sqrt(s);
        }
        __syncthreads();
        const double inv = 1.0 / A[j * D + j];
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
