// Auxiliary kernels of the hot path: the per-step prepare kernel (CFL time
// step from the reduced max wave speed, GLM c_h and damping factor), the
// max-wave-speed reduction, deterministic FP64 conservation sums, state
// conversions and the batched interface-flux kernel.
#include "mhd_internal.h"

namespace mhd {

template <class T>
Phys<T> make_phys(const Grid& g) {
  Phys<T> ph;
  ph.gamma = T(g.gamma);
  ph.gm1 = T(g.gamma - 1.0);
  ph.gm1i = T(1.0 / (g.gamma - 1.0));
  ph.rho_floor = T(g.rho_floor);
  ph.p_floor = T(g.p_floor);
  ph.gamma_d = g.gamma;
  ph.rho_floor_d = g.rho_floor;
  ph.p_floor_d = g.p_floor;
  return ph;
}
template Phys<double> make_phys<double>(const Grid&);
template Phys<float> make_phys<float>(const Grid&);

// ---------------------------------------------------------------- prepare --
// One thread.  dt rule: c_h = lambda (max |v_d| + c_f,d of the state),
// dt = cfl / (c_h sum_active 1/dx_d), clamped so the step ends at t_end.
// A non-finite or non-positive dt / c_h sets status bit 1 and turns the step
// into a no-op (dt = 0, damping 1), so the state is preserved for inspection.
__global__ void prep_kernel(const PrepArgs a, StepScalars* sc, unsigned long long* lam_bits,
                            unsigned int* est_bits, unsigned int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double lam = __longlong_as_double((long long)*lam_bits);
  double ch = a.ch_req > 0.0 ? a.ch_req : lam;
  double dt = a.dt_req;
  const double t = sc->t;
  if (!(dt > 0.0)) {
    dt = a.cfl / (ch * a.inv_dx_sum);
    if (a.t_end > 0.0) dt = fmin(dt, a.t_end - t);
  }
  bool bad = !(ch > 0.0) || !(ch < INFINITY) || !(dt >= 0.0) || !(dt < INFINITY);
  if (bad) {
    atomicOr(status, 1u);
    dt = 0.0;
    ch = 1.0;
  }
  sc->dt = dt;
  sc->ch = ch;
  for (int d = 0; d < 3; ++d) sc->dtdx[d] = a.active[d] ? dt / a.dx[d] : 0.0;
  sc->damp = exp(-a.glm_alpha * ch * dt / a.dh_min);
  sc->t = t + dt;
  sc->lam = lam;
  sc->steps += 1.0;
  *lam_bits = 0ull;  // the last stage accumulates lambda of the new state
  *est_bits = 0u;
}

cudaError_t launch_prep(const PrepArgs& a, StepScalars* sc, unsigned long long* lam_bits,
                        unsigned int* est_bits, unsigned int* status, cudaStream_t stream) {
  prep_kernel<<<1, 32, 0, stream>>>(a, sc, lam_bits, est_bits, status);
  return cudaGetLastError();
}

// (t, dt, c_h, steps) of the last step into a caller's device array.
__global__ void step_record_kernel(const StepScalars* sc, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  out[0] = sc->t;
  out[1] = sc->dt;
  out[2] = sc->ch;
  out[3] = sc->steps;
}

cudaError_t launch_step_record(const StepScalars* sc, double* out, cudaStream_t stream) {
  step_record_kernel<<<1, 32, 0, stream>>>(sc, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------- max wave speed --
// Block maximum of a non-negative (or NaN) double per thread; thread 0 gets it.
__device__ __forceinline__ double block_speed_max(double lam) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lam = nan_max(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  __shared__ double w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = lam;
  __syncthreads();
  double m = w[0];
  if (threadIdx.x == 0)
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = nan_max(m, w[i]);
  return m;
}

// FP32 states: every cell's speed.
__global__ void __launch_bounds__(256) max_speed_f32_kernel(const float* __restrict__ U,
                                                            long long ncell, int ndim,
                                                            Phys<float> ph,
                                                            unsigned long long* lam_bits) {
  unsigned flags = 0;  // not counted: floors are counted per stage input
  SpeedMax<float> smax(ph);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    float u[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) u[k] = U[k * ncell + c];
    smax.update(u, true, ph, ndim, flags);
  }
  const double m = block_speed_max(smax.value());
  if (threadIdx.x == 0) SpeedMax<float>::publish(m, lam_bits, nullptr);
}

// FP64 pass 1 over cells [c0, c1): the maximum reliable FP32 estimate.
__global__ void __launch_bounds__(256) speed_estimate_kernel(const double* __restrict__ U,
                                                             long long ncell, long long c0,
                                                             long long c1, int ndim,
                                                             Phys<double> ph,
                                                             unsigned int* est_bits) {
  unsigned flags = 0;
  SpeedMax<double> smax(ph);
  for (long long c = c0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; c < c1;
       c += (long long)gridDim.x * blockDim.x) {
    double u[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) u[k] = U[k * ncell + c];
    smax.update(u, true, ph, ndim, flags);
  }
  const double m = block_speed_max(smax.value());
  if (threadIdx.x == 0) SpeedMax<double>::publish(m, nullptr, est_bits);
}

// FP64 pass 2: the exact speed of every cell whose estimate reaches 0.999 of
// the maximum reliable estimate or is not reliable (mhd_physics.cuh).  The
// trip count is warp-uniform so that the FP64 evaluation can sit behind a
// warp-uniform branch.
__global__ void __launch_bounds__(256) speed_exact_kernel(const double* __restrict__ U,
                                                          long long ncell, int ndim,
                                                          Phys<double> ph,
                                                          const unsigned int* est_bits,
                                                          unsigned long long* lam_bits) {
  unsigned flags = 0;  // not counted: floors are counted per stage input
  const SpeedEstimator estimate(ph);
  const float thr = 0.999f * __uint_as_float(*est_bits);
  double lam = 0.0;
  const long long lane = threadIdx.x & 31;
  for (long long w = blockIdx.x * (long long)blockDim.x + (threadIdx.x - lane); w < ncell;
       w += (long long)gridDim.x * blockDim.x) {
    const long long c = w + lane;
    const bool valid = c < ncell;
    double u[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) u[k] = valid ? U[k * ncell + c] : 0.0;
    bool ok = true;
    const float e = estimate(u, ndim, ok);
    const bool cand = valid && (!ok || e >= thr);
    if (__any_sync(0xffffffffu, cand)) {
      if (cand) lam = nan_max(lam, cell_max_speed(u, ph, ndim, flags));
    }
  }
  const double m = block_speed_max(lam);
  if (threadIdx.x == 0) SpeedMax<float>::publish(m, lam_bits, nullptr);
}

static unsigned speed_blocks(const Grid& g, long long n) {
  long long blocks = (n + 255) / 256;
  const long long cap = (long long)g.nsm * 8;
  if (blocks > cap) blocks = cap;
  return (unsigned)(blocks < 1 ? 1 : blocks);
}

cudaError_t launch_speed_estimate(const Grid& g, const double* U, long long c0, long long c1,
                                  unsigned int* est_bits, cudaStream_t stream) {
  if (c0 < 0 || c1 > g.ncell || c0 >= c1) return cudaErrorInvalidValue;
  speed_estimate_kernel<<<speed_blocks(g, c1 - c0), 256, 0, stream>>>(
      U, g.ncell, c0, c1, g.ndim, make_phys<double>(g), est_bits);
  return cudaGetLastError();
}

cudaError_t launch_speed_exact(const Grid& g, const double* U, const unsigned int* est_bits,
                               unsigned long long* lam_bits, cudaStream_t stream) {
  speed_exact_kernel<<<speed_blocks(g, g.ncell), 256, 0, stream>>>(
      U, g.ncell, g.ndim, make_phys<double>(g), est_bits, lam_bits);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_max_speed(const Grid& g, const T* U, unsigned long long* lam_bits,
                             unsigned int* est_bits, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(lam_bits, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  if constexpr (sizeof(T) == 8) {
    if (!est_bits) return cudaErrorInvalidValue;
    e = cudaMemsetAsync(est_bits, 0, sizeof(unsigned int), stream);
    if (e == cudaSuccess) e = launch_speed_estimate(g, U, 0, g.ncell, est_bits, stream);
    if (e == cudaSuccess) e = launch_speed_exact(g, U, est_bits, lam_bits, stream);
    return e;
  } else {
    max_speed_f32_kernel<<<speed_blocks(g, g.ncell), 256, 0, stream>>>(
        U, g.ncell, g.ndim, make_phys<float>(g), lam_bits);
    return cudaGetLastError();
  }
}
template cudaError_t launch_max_speed<double>(const Grid&, const double*, unsigned long long*,
                                              unsigned int*, cudaStream_t);
template cudaError_t launch_max_speed<float>(const Grid&, const float*, unsigned long long*,
                                             unsigned int*, cudaStream_t);

// ------------------------------------------------------ conservation sums --
// Pass 1: CTA b sums the contiguous cell range [b*chunk, (b+1)*chunk) of the
// eight conserved quantities in FP64, threads strided, then a fixed-shape
// shared-memory tree.  Pass 2: one CTA reduces the partials the same way.
// The order depends only on (ncell, nblocks): results are bitwise repeatable.
__device__ __forceinline__ void tree_sum8(double (*s)[8], int tid) {
  for (int h = 128; h > 0; h >>= 1) {
    __syncthreads();
    if (tid < h)
      for (int q = 0; q < 8; ++q) s[tid][q] += s[tid + h][q];
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(256) sums_pass1(const T* __restrict__ U, long long ncell,
                                                  long long chunk, double* partials) {
  __shared__ double s[256][8];
  const int vars[8] = {kRHO, kVX, kVY, kVZ, kPRS, kBX, kBY, kBZ};
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long lo = blockIdx.x * chunk;
  const long long hi = min(lo + chunk, ncell);
  for (long long c = lo + threadIdx.x; c < hi; c += 256)
    for (int q = 0; q < 8; ++q) acc[q] += (double)U[vars[q] * ncell + c];
  for (int q = 0; q < 8; ++q) s[threadIdx.x][q] = acc[q];
  tree_sum8(s, threadIdx.x);
  if (threadIdx.x == 0)
    for (int q = 0; q < 8; ++q) partials[blockIdx.x * 8 + q] = s[0][q];
}

__global__ void __launch_bounds__(256) sums_pass2(const double* partials, int nblocks,
                                                  double vol, double* out8) {
  __shared__ double s[256][8];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblocks; b += 256)
    for (int q = 0; q < 8; ++q) acc[q] += partials[b * 8 + q];
  for (int q = 0; q < 8; ++q) s[threadIdx.x][q] = acc[q];
  tree_sum8(s, threadIdx.x);
  if (threadIdx.x == 0)
    for (int q = 0; q < 8; ++q) out8[q] = s[0][q] * vol;
}

template <class T>
cudaError_t launch_sums(const Grid& g, const T* U, double* partials, int nblocks, double* out8,
                        cudaStream_t stream) {
  const long long chunk = (g.ncell + nblocks - 1) / nblocks;
  double vol = 1.0;
  for (int d = 0; d < 3; ++d)
    if (g.n[d] > 1) vol *= g.dx[d];
  sums_pass1<T><<<nblocks, 256, 0, stream>>>(U, g.ncell, chunk, partials);
  sums_pass2<<<1, 256, 0, stream>>>(partials, nblocks, vol, out8);
  return cudaGetLastError();
}
template cudaError_t launch_sums<double>(const Grid&, const double*, double*, int, double*,
                                         cudaStream_t);
template cudaError_t launch_sums<float>(const Grid&, const float*, double*, int, double*,
                                        cudaStream_t);

// ------------------------------------------------------------ conversions --
static inline unsigned grid_for(long long n, int nsm) {
  long long b = (n + 255) / 256;
  const long long cap = (long long)nsm * 16;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------ halo faces --
// One thread per halo element, in the destination's order: the source is the
// cell whose coordinate along the face normal d is the layer (low face) or
// n_d - gh + layer (high face).
template <class T>
__global__ void halo_pack_kernel(const T* __restrict__ W, T* __restrict__ dst, int n0, int n1,
                                 int n2, long long ncell, int d, int hi, int gh) {
  const int e0 = d == 0 ? gh : n0, e1 = d == 1 ? gh : n1, e2 = d == 2 ? gh : n2;
  const long long per_var = (long long)e0 * e1 * e2;
  const long long total = 9 * per_var;
  const int n_d = d == 0 ? n0 : (d == 1 ? n1 : n2);
  const int shift = hi ? n_d - gh : 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(q / per_var);
    long long r = q - v * per_var;
    int c0 = (int)(r % e0);
    r /= e0;
    int c1 = (int)(r % e1);
    int c2 = (int)(r / e1);
    if (d == 0) c0 += shift;
    if (d == 1) c1 += shift;
    if (d == 2) c2 += shift;
    dst[q] = W[v * ncell + ((long long)c2 * n1 + c1) * n0 + c0];
  }
}

template <class T>
cudaError_t launch_halo_pack(const Grid& g, const T* W, int face, int gh, T* dst,
                             cudaStream_t stream) {
  const int d = face >> 1;
  if (face < 0 || face > 5 || gh < 1 || gh > g.n[d]) return cudaErrorInvalidValue;
  long long area = 1;
  for (int e = 0; e < 3; ++e) area *= e == d ? gh : g.n[e];
  halo_pack_kernel<T><<<grid_for(9 * area, g.nsm), 256, 0, stream>>>(
      W, dst, g.n[0], g.n[1], g.n[2], g.ncell, d, face & 1, gh);
  return cudaGetLastError();
}
template cudaError_t launch_halo_pack<double>(const Grid&, const double*, int, int, double*,
                                              cudaStream_t);
template cudaError_t launch_halo_pack<float>(const Grid&, const float*, int, int, float*,
                                             cudaStream_t);

// The wave-speed maxima of subdomains combine by an integer maximum of their
// bit patterns (non-negative doubles order like their patterns; the
// canonical quiet NaN orders above +inf, also as a signed 64-bit integer).
__global__ void lambda_max_into_kernel(const unsigned long long* lam_bits,
                                       unsigned long long* dst) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long b = *lam_bits;
  if ((b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull)
    b = 0x7ff8000000000000ull;  // NaN (either sign)
  else if (b >> 63)
    b = 0ull;  // -0 (wave speeds are not negative)
  atomicMax(dst, b);
}

cudaError_t launch_lambda_max_into(const unsigned long long* lam_bits, unsigned long long* dst,
                                   cudaStream_t stream) {
  lambda_max_into_kernel<<<1, 32, 0, stream>>>(lam_bits, dst);
  return cudaGetLastError();
}


template <class T>
__global__ void prim_to_cons_kernel(const double* __restrict__ V, T* __restrict__ U,
                                    long long ncell, Phys<double> ph) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double v[kNV], u[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) v[k] = V[k * ncell + c];
    prim_to_cons(v, u, ph);
#pragma unroll
    for (int k = 0; k < kNV; ++k) U[k * ncell + c] = (T)u[k];
  }
}

template <class T>
__global__ void prim_to_cons_inplace_kernel(T* U, long long ncell, Phys<double> ph) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double v[kNV], u[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) v[k] = (double)U[k * ncell + c];
    prim_to_cons(v, u, ph);
#pragma unroll
    for (int k = 0; k < kNV; ++k) U[k * ncell + c] = (T)u[k];
  }
}

template <class T>
__global__ void cons_to_prim_kernel(const T* __restrict__ U, double* __restrict__ V,
                                    long long ncell, Phys<T> ph) {
  unsigned flags = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    T u[kNV], v[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) u[k] = U[k * ncell + c];
    cons_to_prim(u, v, ph, flags);
#pragma unroll
    for (int k = 0; k < kNV; ++k) V[k * ncell + c] = (double)v[k];
  }
}

template <class T>
cudaError_t launch_prim_to_cons(const Grid& g, const double* V, T* U, cudaStream_t stream) {
  prim_to_cons_kernel<T><<<grid_for(g.ncell, g.nsm), 256, 0, stream>>>(V, U, g.ncell,
                                                                        make_phys<double>(g));
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_prim_to_cons_inplace(const Grid& g, T* U, cudaStream_t stream) {
  prim_to_cons_inplace_kernel<T><<<grid_for(g.ncell, g.nsm), 256, 0, stream>>>(
      U, g.ncell, make_phys<double>(g));
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_cons_to_prim(const Grid& g, const T* U, double* V, cudaStream_t stream) {
  cons_to_prim_kernel<T><<<grid_for(g.ncell, g.nsm), 256, 0, stream>>>(U, V, g.ncell,
                                                                        make_phys<T>(g));
  return cudaGetLastError();
}
template cudaError_t launch_prim_to_cons<double>(const Grid&, const double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_prim_to_cons<float>(const Grid&, const double*, float*,
                                                cudaStream_t);
template cudaError_t launch_prim_to_cons_inplace<double>(const Grid&, double*, cudaStream_t);
template cudaError_t launch_prim_to_cons_inplace<float>(const Grid&, float*, cudaStream_t);
template cudaError_t launch_cons_to_prim<double>(const Grid&, const double*, double*,
                                                 cudaStream_t);
template cudaError_t launch_cons_to_prim<float>(const Grid&, const float*, double*,
                                                cudaStream_t);

__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out,
                                  long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void f32_to_f64_kernel(const float* __restrict__ in, double* __restrict__ out,
                                  long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
cudaError_t launch_f64_to_f32(const double* in, float* out, long long n, cudaStream_t stream) {
  f64_to_f32_kernel<<<grid_for(n, 152), 256, 0, stream>>>(in, out, n);
  return cudaGetLastError();
}
cudaError_t launch_f32_to_f64(const float* in, double* out, long long n, cudaStream_t stream) {
  f32_to_f64_kernel<<<grid_for(n, 152), 256, 0, stream>>>(in, out, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------ flux batch --
template <class T>
__global__ void flux_batch_kernel(const T* __restrict__ VL, const T* __restrict__ VR,
                                  T* __restrict__ F, long long nface, int dir, T ch, T half_chi,
                                  Phys<T> ph) {
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nface;
       f += (long long)gridDim.x * blockDim.x) {
    T vl[kNV], vr[kNV], out[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
      vl[k] = VL[k * nface + f];
      vr[k] = VR[k * nface + f];
    }
    glm_hlld_flux_dir(vl, vr, dir, ch, half_chi, ph, out);
#pragma unroll
    for (int k = 0; k < kNV; ++k) F[k * nface + f] = out[k];
  }
}

template <class T>
cudaError_t launch_flux_batch(const T* VL, const T* VR, T* F, long long nface, int dir,
                              double ch, double gamma, cudaStream_t stream) {
  Grid g{};
  g.gamma = gamma;
  g.rho_floor = 0.0;
  g.p_floor = 0.0;
  flux_batch_kernel<T><<<grid_for(nface, 152), 256, 0, stream>>>(
      VL, VR, F, nface, dir, T(ch), T(0.5 / ch), make_phys<T>(g));
  return cudaGetLastError();
}
template cudaError_t launch_flux_batch<double>(const double*, const double*, double*, long long,
                                               int, double, double, cudaStream_t);
template cudaError_t launch_flux_batch<float>(const float*, const float*, float*, long long, int,
                                              double, double, cudaStream_t);

// FP64 throughput probe: every thread of the warps selected by warp_mask
// (bit w: warp w of the 8) runs 16 independent fused multiply-add chains
// (a <- a b + c) for `iters` rounds.  The chains converge to c / (1 - b) and
// stay finite; the sums are stored so that no chain is dead code.
__global__ void __launch_bounds__(256, 1) fma_rate_kernel(double* out, int iters,
                                                          unsigned warp_mask) {
  double a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = 1.0 + 1e-9 * (threadIdx.x + i);
  const double b = 0.999999999, c = 1e-12;
  const int n = (warp_mask >> (threadIdx.x >> 5)) & 1u ? iters : 0;
  for (int it = 0; it < n; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += a[i];
  out[blockIdx.x * 256 + threadIdx.x] = s;
}

cudaError_t measure_fma_rate(cudaStream_t stream, unsigned warp_mask, double out[3]) {
  warp_mask &= 0xffu;
  if (!warp_mask) warp_mask = 0xffu;
  int dev = 0, nsm = 0, khz = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) return e;
  double* buf = nullptr;
  e = cudaMalloc(&buf, (size_t)nsm * 256 * sizeof(double));
  if (e != cudaSuccess) return e;
  // one CTA per SM: its shared-memory request leaves no room for a second
  const int smem = 160 * 1024;
  const int iters = 20000;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaFuncSetAttribute(fma_rate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fma_rate_kernel<<<nsm, 256, smem, stream>>>(buf, iters / 10, warp_mask);  // warm-up
    cudaEventRecord(e0, stream);
    fma_rate_kernel<<<nsm, 256, smem, stream>>>(buf, iters, warp_mask);
    cudaEventRecord(e1, stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  }
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return e;
  const double lanes = (double)nsm * 32.0 * __builtin_popcount(warp_mask) * iters * 16.0;
  out[0] = lanes / (ms * 1e-3);
  out[1] = out[0] / nsm / (khz * 1e3);
  out[2] = ms;
  return cudaSuccess;
}

}  // namespace mhd
