// Discrete adjoint of the RK2 step (reverse-mode derivative with dt and c_h
// frozen).
#include <cstdio>

#include "mhd_internal.h"

namespace mhd {

size_t adjoint_scratch_bytes(const Grid& g) { return 256; }

int adjoint_step(const Grid& g, double dt, double ch, double glm_alpha, double dh_min,
                 const double* U_n, const double* lam_np1, double* lam_n, void* scratch,
                 size_t scratch_bytes, cudaStream_t stream, char* err, size_t errlen) {
  snprintf(err, errlen, "adjoint not available in this build");
  return -6;
}

}  // namespace mhd
