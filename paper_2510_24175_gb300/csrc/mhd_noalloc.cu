// Conservation sums for callers that cannot allocate device memory.
//
// Some callers of this library can't call cudaMalloc: a host application
// whose device memory is all owned by another allocator (for example a
// framework's caching allocator that reserved the GPU at start-up), a code
// whose policy forbids allocations once its time loop runs, or a diagnostic
// hook that runs while the caller is capturing a stream (where cudaMalloc is
// not allowed in the default capture mode).  mhd_conserved_sums_noalloc()
// serves them: it needs no context and no workspace.  Its scratch (per-block
// partial sums and the 8 results) lives in a file-scope __device__ array of
// fixed size that every GPU loading this library holds until the process
// exits.  It calls no cudaMalloc, cudaFree or allocating library routine.
#include <cstdio>
#include <mutex>

#include "../../include/mhd.h"
#include "mhd_internal.h"

namespace {

constexpr long long kCellsPerPartial = 32768;
constexpr int kMaxPartials = 16384;  // => at most 16384 * 32768 cells
constexpr int kMaxDevices = 64;

// 16384 x 8 partials + 8 results = 1 MiB of FP64 scratch per device.
static __device__ __align__(256) double g_sums_scratch[kMaxPartials * 8 + 8];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sums_scratch on the current device, looked up once per
// device (host code cannot use the symbol itself as a device pointer).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return mhd::free_fail(MHD_ERR_CUDA, "mhd_conserved_sums_noalloc: no usable device");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sums_scratch);
    if (e != cudaSuccess || !p) {
      return mhd::free_fail(MHD_ERR_CUDA,
                            "mhd_conserved_sums_noalloc: cudaGetSymbolAddress failed: %s",
                            cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MHD_OK;
}

}  // namespace

extern "C" int mhd_conserved_sums_noalloc(const mhd_config* cfg, const void* U, double out[8],
                                          void* stream) {
  if (!cfg || !U || !out)
    return mhd::free_fail(MHD_ERR_INVALID, "mhd_conserved_sums_noalloc: null argument");
  size_t unused = 0;
  if (mhd_workspace_bytes(cfg, &unused) != MHD_OK) return MHD_ERR_INVALID;  // its message
  mhd::Grid g{};
  long long ncell = 1;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = cfg->n[d];
    g.dx[d] = (cfg->xmax[d] - cfg->xmin[d]) / cfg->n[d];
    ncell *= cfg->n[d];
  }
  g.ncell = ncell;
  const long long nparts = (ncell + kCellsPerPartial - 1) / kCellsPerPartial;
  if (nparts > kMaxPartials) {
    return mhd::free_fail(MHD_ERR_NOMEM,
                          "mhd_conserved_sums_noalloc: %lld cells exceed the fixed scratch (at "
                          "most %lld cells); use mhd_conserved_sums with a workspace",
                          ncell, (long long)kMaxPartials * kCellsPerPartial);
  }
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != MHD_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Pass 1 writes every partial pass 2 reads, and pass 2 writes all 8
  // results, so nothing left in the scratch by an earlier call is used.
  double* results = scratch + (size_t)kMaxPartials * 8;
  cudaError_t e;
  if (cfg->precision == MHD_FP64)
    e = mhd::launch_sums<double>(g, static_cast<const double*>(U), scratch, (int)nparts, results,
                                 s);
  else
    e = mhd::launch_sums<float>(g, static_cast<const float*>(U), scratch, (int)nparts, results,
                                s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, results, 8 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return mhd::free_fail(MHD_ERR_CUDA, "mhd_conserved_sums_noalloc: %s", cudaGetErrorString(e));
  return MHD_OK;
}
