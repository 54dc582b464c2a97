// project_f32_2d.cu -- explicit instantiations of the fused projection kernel (FP32, 2-D).
#include "project_kernel.cuh"

namespace priest {

template cudaError_t launch_variant<float, 2, 4, 512>(const ProjParams<float> &, const Tiling &, cudaStream_t);
template cudaError_t launch_variant<float, 2, 5, 512>(const ProjParams<float> &, const Tiling &, cudaStream_t);

template cudaError_t launch_variant_batch<float, 2, 5, 512>(const ProjParams<float> *, const int2 *, int, int *,
                                                              int, int, int, size_t, int, cudaStream_t);

}  // namespace priest
