// Conservation sums for callers that cannot allocate device memory.
//
// Some callers of this library can't call cudaMalloc: a host application
// whose device memory is all owned by another allocator (for example a
// framework's caching allocator that reserved the GPU at start-up), or a code
// whose policy forbids allocations once its time loop runs.
// mhd_conserved_sums_noalloc() serves them: it needs no context and no
// workspace.  Its scratch (per-block partial sums and the 8 results) lives in
// a file-scope __device__ array of fixed size that every GPU loading this
// library holds until the process exits.  It calls no cudaMalloc, cudaFree or
// allocating library routine.
#include <cstdio>

#include "../../include/mhd.h"
#include "mhd_internal.h"

namespace {

constexpr long long kCellsPerPartial = 32768;
constexpr int kMaxPartials = 16384;  // => at most 16384 * 32768 cells

// 16384 x 8 partials + 8 results = 1 MiB of FP64 scratch per device.
static __device__ __align__(256) double g_sums_scratch[kMaxPartials * 8 + 8];

// Device address of g_sums_scratch on the current device.  Host code cannot
// use the symbol itself as a device pointer.  The address is looked up on
// every call (a cheap runtime query), so nothing cached can go stale, e.g.
// after a cudaDeviceReset or on another device.
int scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_sums_scratch);
  if (e != cudaSuccess || !p) {
    return mhd::free_fail(MHD_ERR_CUDA,
                          "mhd_conserved_sums_noalloc: cudaGetSymbolAddress failed: %s",
                          cudaGetErrorString(e));
  }
  *out = static_cast<double*>(p);
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
    g.dx[d] = cfg->dx[d] > 0.0 ? cfg->dx[d] : (cfg->xmax[d] - cfg->xmin[d]) / cfg->n[d];
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The call ends with a copy to pageable host memory and a stream
  // synchronisation, neither of which a capturing stream accepts: refuse it
  // before anything is enqueued, so the caller's capture stays intact.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess)
    return mhd::free_fail(MHD_ERR_CUDA, "mhd_conserved_sums_noalloc: %s", cudaGetErrorString(e));
  if (cs != cudaStreamCaptureStatusNone)
    return mhd::free_fail(MHD_ERR_INVALID,
                          "mhd_conserved_sums_noalloc: the stream is capturing; this call "
                          "synchronises its stream");
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != MHD_OK) return rc;
  // Pass 1 writes every partial pass 2 reads, and pass 2 writes all 8
  // results, so nothing left in the scratch by an earlier call is used.
  double* results = scratch + (size_t)kMaxPartials * 8;
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
