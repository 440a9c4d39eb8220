// FP32 instantiation of the fused stage kernel.
#include "mhd_stage_impl.cuh"

namespace mhd {
// compiled in mhd_stage_halo_f32.cu
extern template cudaError_t launch_stage_halo<float>(const Grid&, int, const float*, const float*, float*,
                                                  const StepScalars*, unsigned long long*,
                                                  unsigned long long*, cudaStream_t, double,
                                                  double, const float* const*, unsigned int*, int,
                                                  int, int);
extern template cudaError_t prepare_stage_kernels_halo<float>(const Grid&);
template cudaError_t launch_stage<float>(const Grid&, int, const float*, const float*, float*,
                                         const StepScalars*, unsigned long long*,
                                         unsigned long long*, cudaStream_t, double, double,
                                         const float* const*, float*, int, int, int,
                                          unsigned int*);
template void stage_shape<float>(const Grid&, size_t*, int*, int*);
template cudaError_t prepare_stage_kernels<float>(const Grid&, bool);
}  // namespace mhd
