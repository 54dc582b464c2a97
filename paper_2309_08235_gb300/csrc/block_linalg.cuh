// block_linalg.cuh -- small FP64 dense factorisations run by one CTA.
//
// FP64 issues slowly on this part (64 cycles per dependent FMA), so the
// serial chains are kept short: reciprocals and reciprocal square roots start
// from the PTX FP64 estimates (relative error below 2^-19 measured) and are
// refined by Newton-Raphson steps in FP64, and per-column scalars are formed
// by one thread and shared.
#pragma once

#include <cuda_runtime.h>

#include "priest.h"

namespace priest {

// x is positive, normal, and far enough from the top of the range that 1/x
// and 1/sqrt(x) are normal too: a test of the exponent bits on the integer
// pipe (the sign bit makes a negative x fail it).
__device__ __forceinline__ bool positive_normal(double x)
{
    const unsigned hi = unsigned(__double2hiint(x));
    return (hi >> 20) - 1u < 0x7fcu;
}

// 1/x for positive_normal(x): the FP64 estimate of the PTX approximate
// reciprocal (relative error below 2^-19 on this part), then one third-order
// step: with e = 1 - x y, 1/x = y (1 + e + e^2 + ...), so y (1 + e + e^2)
// leaves an error of e^3 < 2^-57 before the final rounding.
__device__ __forceinline__ double rcp_fast(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// 1/sqrt(x) for positive_normal(x): the PTX approximate reciprocal square
// root, then two Newton-Raphson steps e = 1/2 - (x/2) y^2, y <- y + y e.
__device__ __forceinline__ double rsqrt_fast(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double h = 0.5 * x;
    double e = fma(-h, y * y, 0.5);
    y = fma(y, e, y);
    e = fma(-h, y * y, 0.5);
    return fma(y, e, y);
}

// 1/x for any x: rcp_fast where it applies, else the plain division.
__device__ __forceinline__ double rcp_any(double x) { return positive_normal(x) ? rcp_fast(x) : 1.0 / x; }

constexpr int kCholMaxD = PRIEST_MAX_D;

// In-place Cholesky of the D x D symmetric matrix A (row-major, shared
// memory, D <= kCholMaxD): on return the lower triangle holds L with
// A = L L^T and the strict upper triangle is zeroed.  Returns false (to every
// thread) on a pivot that is not a positive normal number; that pivot is
// taken as 1 and the factorisation runs on.  All threads of the CTA call it.
//
// Right-looking, in the unscaled form: step j updates the trailing lower
// triangle, A[i][k] -= A[i][j] A[k][j] / A[j][j] for j < k <= i, which is the
// rank-1 update of the textbook form (L[i][j] = A[i][j] / sqrt(A[j][j]))
// without scaling column j first; L follows at the end in one pass,
// L[i][k] = A[i][k] / sqrt(A[k][k]).  The thread that updates the next pivot
// (a thread of its own) forms its reciprocal at once, column j + 1 is copied
// into a contiguous buffer as it is written and the square of its entry in
// row j + 2 is kept, so each column costs one barrier and the serial chain per
// column is one fused multiply-add and one reciprocal.  Each thread keeps the
// same elements at every step: the triangle is numbered by columns from the
// last one back (column k holds rows k..D-1), so the elements of step j are
// the first (D-1-j)(D-j)/2 numbers.
__device__ inline bool block_cholesky(double *A, int D, int *flag_smem)
{
    __shared__ double s_col[2][kCholMaxD];  // column j (unscaled), by step parity
    __shared__ double s_rcp[kCholMaxD];     // 1 / pivot
    __shared__ double s_sq[2];              // A[j+1][j]^2, by step parity
    __shared__ unsigned short s_tab[kCholMaxD * (kCholMaxD + 1) / 2];  // (i << 8) | k
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const int ntri = D * (D + 1) / 2;
    for (int p = tid; p < ntri; p += T) {
        // q(q+1)/2 <= p < (q+1)(q+2)/2: the block of column k = D-1-q
        int q = int((sqrtf(float(8 * p + 1)) - 1.0f) * 0.5f);
        if ((q + 1) * (q + 2) / 2 <= p) ++q;
        if (q * (q + 1) / 2 > p) --q;
        const int k = D - 1 - q, i = k + (p - q * (q + 1) / 2);
        s_tab[p] = static_cast<unsigned short>((i << 8) | k);
    }
    if (tid == 0) {
        int ok = 1;
        double v = A[0];
        if (!positive_normal(v)) {
            ok = 0;
            v = 1.0;
            A[0] = v;
        }
        *flag_smem = ok;
        s_rcp[0] = rcp_fast(v);
    }
    for (int i = 1 + tid; i < D; i += T) {
        const double v = A[i * D];
        s_col[0][i] = v;
        if (i == 1) s_sq[0] = v * v;
    }
    __syncthreads();
    // the next pivot and its reciprocal on lane 0 of the last warp, which
    // takes no part in the update, so no other element waits behind the chain
    const int Tw = nw > 1 ? T - 32 : T, tp = nw > 1 ? T - 32 : 0;
    for (int j = 0; j + 1 < D; ++j) {
        const int m = D - 1 - j, cnt = m * (m + 1) / 2;
        const double r = s_rcp[j];
        const double *col = s_col[j & 1];
        double *nxt = s_col[(j + 1) & 1];
        if (tid == tp) {
            const int q = (j + 1) * (D + 1);
            double v = fma(-s_sq[j & 1], r, A[q]);
            if (!positive_normal(v)) {
                *flag_smem = 0;
                v = 1.0;
            }
            s_rcp[j + 1] = rcp_fast(v);
            A[q] = v;
        }
        if (tid < Tw)
            for (int p = tid; p < cnt; p += Tw) {
                const int ik = s_tab[p], i = ik >> 8, k = ik & 255;
                if (i == k && k == j + 1) continue;  // the pivot, above
                const double v = fma(-col[i], col[k] * r, A[i * D + k]);
                if (k == j + 1) {
                    nxt[i] = v;
                    if (i == k + 1) s_sq[(j + 1) & 1] = v * v;
                }
                A[i * D + k] = v;
            }
        __syncthreads();
    }
    double *rsq = s_col[0];  // free after the last step's barrier
    for (int k = tid; k < D; k += T) rsq[k] = rsqrt_fast(A[k * D + k]);
    __syncthreads();
    for (int i = warp; i < D; i += nw)
        for (int k = lane; k < D; k += 32) A[i * D + k] = (k <= i) ? A[i * D + k] * rsq[k] : 0.0;
    __syncthreads();
    return *flag_smem != 0;
}

}  // namespace priest
