// project_f32_2d_wide.cu -- explicit instantiations of the fused projection kernel (FP32, 2-D,
// eight points per item or 1024-thread CTAs).
#include "project_kernel.cuh"

namespace priest {

template cudaError_t launch_variant<float, 2, 8, 512>(const ProjParams<float> &, const Tiling &, cudaStream_t);
template cudaError_t launch_variant<float, 2, 5, 1024>(const ProjParams<float> &, const Tiling &, cudaStream_t);

}  // namespace priest
