// FP64 instantiation of the fused stage kernel.
#include "mhd_stage_impl.cuh"

namespace mhd {
// compiled in mhd_stage_halo_f64.cu
extern template cudaError_t launch_stage_halo<double>(const Grid&, int, const double*, const double*, double*,
                                                  const StepScalars*, unsigned long long*,
                                                  unsigned long long*, cudaStream_t, double,
                                                  double, const double* const*, unsigned int*, int,
                                                  int, int);
extern template cudaError_t prepare_stage_kernels_halo<double>(const Grid&);
template cudaError_t launch_stage<double>(const Grid&, int, const double*, const double*, double*,
                                          const StepScalars*, unsigned long long*,
                                          unsigned long long*, cudaStream_t, double, double,
                                          const double* const*, double*, int, int, int,
                                          unsigned int*);
template void stage_shape<double>(const Grid&, size_t*, int*, int*);
template cudaError_t prepare_stage_kernels<double>(const Grid&, bool);
}  // namespace mhd
