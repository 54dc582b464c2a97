// rng.cu -- the standard-normal stream of Alg. 1's sampling step, drawn on
// the device.
//
// The stream is the one the host produces for priest_plan: SplitMix64
// (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014) seeded with `seed`, 53-bit uniforms u = (x >> 11) 2^-53 and the
// Box-Muller transform on (1 - u1, u2) giving r cos(2 pi u2), then
// r sin(2 pi u2).  SplitMix64 is counter based -- its k-th state is
// seed + k * 0x9E3779B97F4A7C15 (mod 2^64) -- so value i of the stream needs
// only states 2 floor(i/2) + 1 and + 2 and every thread computes its values
// independently.  The uniforms are bit-identical to the host's; log, sqrt,
// cos and sin are the device's FP64 functions, so the values agree with the
// host stream to within a few units in the last place.
#include <cuda_runtime.h>

#include "priest_internal.cuh"

namespace priest {
namespace {

constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ull;
constexpr int kRngThreads = 256;
constexpr int kPairsPerThread = 4;

__device__ __forceinline__ unsigned long long splitmix_at(unsigned long long seed, unsigned long long k)
{
    unsigned long long z = seed + k * kGolden;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Writes job j's values; the pairs of values are spread over blockIdx.x.
__device__ __forceinline__ void normal_run(const GaussJob &j)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (j.status) *j.status = 0;
        if (j.counter) *j.counter = 0u;
    }
    const long long n_pairs = (j.count + 1) / 2;
    const double two_pi = 6.283185307179586476925286766559;
    const double inv53 = 1.0 / 9007199254740992.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n_pairs;
         q += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = 2ull * (unsigned long long)q;
        const double u1 = double(splitmix_at(j.seed, k + 1) >> 11) * inv53;
        const double u2 = double(splitmix_at(j.seed, k + 2) >> 11) * inv53;
        const double rad = sqrt(-2.0 * log(1.0 - u1));
        const double th = two_pi * u2;
        const long long i = 2 * q;
        j.out[i] = rad * cos(th);
        if (i + 1 < j.count) j.out[i + 1] = rad * sin(th);
    }
}

// One job per blockIdx.y.
__global__ void __launch_bounds__(kRngThreads) normal_kernel(const GaussJob *jobs) { normal_run(jobs[blockIdx.y]); }

__global__ void __launch_bounds__(kRngThreads) normal_single_kernel(const GaussJob job) { normal_run(job); }

unsigned blocks_for(long long count)
{
    const long long pairs = (count + 1) / 2;
    long long bx = (pairs + (long long)kRngThreads * kPairsPerThread - 1) / ((long long)kRngThreads * kPairsPerThread);
    return unsigned(bx < 1 ? 1 : (bx > 65535 ? 65535 : bx));
}

}  // namespace

cudaError_t launch_normal_batch(const GaussJob *jobs_dev, int n_jobs, long long max_count, cudaStream_t st)
{
    if (n_jobs <= 0) return cudaSuccess;
    const unsigned bx = blocks_for(max_count);
    for (int y0 = 0; y0 < n_jobs; y0 += 65535) {
        const int ny = (n_jobs - y0) < 65535 ? (n_jobs - y0) : 65535;
        normal_kernel<<<dim3(bx, unsigned(ny)), kRngThreads, 0, st>>>(jobs_dev + y0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_normal(unsigned long long seed, long long count, double *out_dev, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    GaussJob j;
    j.seed = seed;
    j.count = count;
    j.out = out_dev;
    j.status = nullptr;
    j.counter = nullptr;
    normal_single_kernel<<<blocks_for(count), kRngThreads, 0, st>>>(j);
    return cudaGetLastError();
}

}  // namespace priest
