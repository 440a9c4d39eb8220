// FP64 instantiation of the stage kernels with halo faces (decomposed grids).
#include "mhd_stage_impl.cuh"

namespace mhd {
template cudaError_t launch_stage_halo<double>(const Grid&, int, const double*, const double*, double*,
                                           const StepScalars*, unsigned long long*,
                                           unsigned long long*, cudaStream_t, double, double,
                                           const double* const*, unsigned int*, int, int,
                                           int);
template cudaError_t prepare_stage_kernels_halo<double>(const Grid&);
}  // namespace mhd
