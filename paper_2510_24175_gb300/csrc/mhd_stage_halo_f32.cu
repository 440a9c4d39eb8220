// FP32 instantiation of the stage kernels with halo faces (decomposed grids).
#include "mhd_stage_impl.cuh"

namespace mhd {
template cudaError_t launch_stage_halo<float>(const Grid&, int, const float*, const float*, float*,
                                           const StepScalars*, unsigned long long*,
                                           unsigned long long*, cudaStream_t, double, double,
                                           const float* const*, unsigned int*, int, int,
                                           int);
template cudaError_t prepare_stage_kernels_halo<float>(const Grid&);
}  // namespace mhd
