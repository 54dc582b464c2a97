// project_f64.cu -- explicit instantiations of the fused projection kernel (FP64 check mode).
#include "project_kernel.cuh"

namespace priest {

template cudaError_t launch_variant<double, 2, 4, 256>(const ProjParams<double> &, const Tiling &,
                                                         cudaStream_t);
template cudaError_t launch_variant<double, 3, 4, 256>(const ProjParams<double> &, const Tiling &,
                                                         cudaStream_t);

template cudaError_t launch_variant_batch<double, 2, 4, 256>(const ProjParams<double> *, const int2 *, int, int *,
                                                              int, int, int, size_t, int, cudaStream_t);
template cudaError_t launch_variant_batch<double, 3, 4, 256>(const ProjParams<double> *, const int2 *, int, int *,
                                                              int, int, int, size_t, int, cudaStream_t);

}  // namespace priest
