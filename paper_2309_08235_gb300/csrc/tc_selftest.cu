// tc_selftest.cu -- a diagnostic of the tensor-core path (tc.cuh): one
// D = A B^T product, A 128 x K and B N x K in BF16, D in FP32, through
// shared-memory descriptors, tcgen05.mma, an mbarrier and TMEM loads.  The
// projection's pair-distance products use the same pieces; this entry point
// lets a test compare them with an exact host product (small integers make
// every product and sum exact in FP32).
#include <cuda_runtime.h>

#include "priest_internal.cuh"
#include "tc.cuh"

namespace priest {
namespace {

__global__ void __launch_bounds__(128) tc_selftest_kernel(const uint16_t *A, const uint16_t *B, int N, int K,
                                                          int swap, uint32_t ncols, float *D, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *sA = sm, *sB = sm + 128 * K * 2;
    for (int e = tid; e < 128 * K; e += blockDim.x)
        *reinterpret_cast<uint16_t *>(sA + tc::offset(e / K, e % K, K)) = A[e];
    for (int e = tid; e < N * K; e += blockDim.x)
        *reinterpret_cast<uint16_t *>(sB + tc::offset(e / K, e % K, K)) = B[e];
    tc::fence_async_smem();
    if (warp == 0) tc::tmem_alloc(&tmem_base, ncols);
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    // swap == 2: no product and no completion signal, so the bounded wait below
    // runs out (the time-out path, with no asynchronous work in flight)
    if (tid == 0 && swap != 2) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, N);
        const uint32_t lbo = swap ? tc::sbo(K) : tc::kLbo, sbo = swap ? tc::kLbo : tc::sbo(K);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t a = tc::smem_desc(tc::smem_u32(sA) + ks * 2 * tc::kLbo, lbo, sbo);
            const uint64_t b = tc::smem_desc(tc::smem_u32(sB) + ks * 2 * tc::kLbo, lbo, sbo);
            tc::mma_bf16(tbase, a, b, idesc, ks > 0 ? 1u : 0u);
        }
        tc::mma_commit(&mbar);
    }
    __syncwarp();
    bool ok = tc::mbar_wait_bounded(&mbar, 0, 1000000000ull);
    if (!ok) {
        if (lane == 0) atomicOr(err, 1);
        tc::mbar_wait_bounded(&mbar, 0, 1000000000ull);  // let work in flight finish before freeing TMEM
    }
    tc::fence_after_sync();
    if (ok) {
        for (int c = 0; c < N; c += 16) {
            uint32_t v[16];
            tc::tmem_ld16(tbase + (uint32_t(warp * 32) << 16) + uint32_t(c), v);
            tc::tmem_wait_ld();
            for (int i = 0; i < 16; ++i) D[(warp * 32 + lane) * N + c + i] = __uint_as_float(v[i]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

}  // namespace
}  // namespace priest

using namespace priest;

extern "C" priest_status priest_tc_selftest(int n, int k, int swap, const uint16_t *a_host, const uint16_t *b_host,
                                           float *d_host)
{
    if (n < 16 || n > 256 || n % 16 || k < 16 || k > 64 || k % 16 || swap < 0 || swap > 2 || !a_host || !b_host ||
        !d_host)
        return PRIEST_ERR_INVALID;
    uint32_t ncols = 32;
    while (ncols < uint32_t(n)) ncols <<= 1;
    uint16_t *A = nullptr, *B = nullptr;
    float *D = nullptr;
    int *err = nullptr;
    cudaError_t e = cudaMalloc(&A, sizeof(uint16_t) * 128 * k);
    if (e == cudaSuccess) e = cudaMalloc(&B, sizeof(uint16_t) * n * k);
    if (e == cudaSuccess) e = cudaMalloc(&D, sizeof(float) * 128 * n);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(A, a_host, sizeof(uint16_t) * 128 * k, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B, b_host, sizeof(uint16_t) * n * k, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(D, 0, sizeof(float) * 128 * n);
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    const size_t smem = size_t(128 + n) * k * 2;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) {
        tc_selftest_kernel<<<1, 128, smem>>>(A, B, n, k, swap, ncols, D, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(d_host, D, sizeof(float) * 128 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(A);
    cudaFree(B);
    cudaFree(D);
    cudaFree(err);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PRIEST_ERR_CUDA;
    }
    return herr ? PRIEST_ERR_TIMEOUT : PRIEST_OK;
}
