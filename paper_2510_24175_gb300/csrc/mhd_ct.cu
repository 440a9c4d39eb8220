// Constrained transport: the div-B control of the paper's weak-scaling runs
// (Section 4.2, after Evans & Hawley 1988 and Londrillo & Del Zanna 2004).
// The magnetic field lives on cell faces (b_d on each cell's lower d-face)
// and is advanced by Faraday's law in circulation form,
//   d b_d / dt = -(curl E)_d,  (curl E)_d = dE_b/da - dE_a/db, (d, a, b) cyclic,
// with the electric field on cell edges, so the face divergence
// sum_d (b_d(+1/2) - b_d(-1/2)) / dx_d is preserved to round-off.  The edge
// field is the upwind "CT-contact" average of Gardiner & Stone (2005): the
// mean of the four face values around the edge plus upwinded differences of
// edge-to-cell derivatives, the upwind side given by the sign of the face
// mass flux.
//
// A CT step runs, per Runge-Kutta stage, the fused stage kernel instantiated
// with CT = true (rho, m, E; face and cell electric fields into the CT
// buffer), then the three kernels here: edge fields, face update (with the
// Runge-Kutta combination), and the cell-centred B = mean of the cell's two
// faces (plus, after the last stage, the next step's wave-speed reduction).
// Three active dimensions, periodic boundaries.  All kernels are
// elementwise over cells with neighbour reads at offset -1 / +1 (L1/L2
// serve the reuse); a thread owns one cell.
#include <cuda_runtime.h>

#include "mhd_internal.h"

namespace mhd {

namespace {

constexpr int kCtThreads = 256;

struct CellIndex {
  int i, j, k, im, jm, km, ip, jp, kp;
  __device__ __forceinline__ CellIndex(long long c, int nx, int ny, int nz) {
    const long long pl = (long long)nx * ny;
    k = (int)(c / pl);
    const long long r = c - (long long)k * pl;
    j = (int)(r / nx);
    i = (int)(r - (long long)j * nx);
    im = i ? i - 1 : nx - 1;
    jm = j ? j - 1 : ny - 1;
    km = k ? k - 1 : nz - 1;
    ip = i + 1 < nx ? i + 1 : 0;
    jp = j + 1 < ny ? j + 1 : 0;
    kp = k + 1 < nz ? k + 1 : 0;
  }
};

template <class T>
__device__ __forceinline__ T ct_upwind(T f, T from_lo, T from_hi) {
  return f > T(0) ? from_lo : (f < T(0) ? from_hi : T(0.5) * (from_lo + from_hi));
}

// Edge field from the two a-faces (ea0: on the low-b side, ea1: high-b side,
// mass fluxes fa0, fa1), the two b-faces (eb0: low-a side, eb1: high-a side,
// fb0, fb1) and the four cells c[a side][b side] around the edge.
template <class T>
__device__ __forceinline__ T ct_contact(T ea0, T ea1, T fa0, T fa1, T eb0, T eb1, T fb0, T fb1,
                                        T c00, T c01, T c10, T c11) {
  const T mean = T(0.25) * (ea0 + ea1 + eb0 + eb1);
  const T db_lo = ct_upwind(fa0, eb0 - c00, eb1 - c10);
  const T db_hi = ct_upwind(fa1, c01 - eb0, c11 - eb1);
  const T da_lo = ct_upwind(fb0, ea0 - c00, ea1 - c01);
  const T da_hi = ct_upwind(fb1, c10 - ea0, c11 - ea1);
  return mean + T(0.25) * (db_lo - db_hi) + T(0.25) * (da_lo - da_hi);
}

// Edge fields of each cell: E_x on its (y-, z-) edge, E_y on its (z-, x-)
// edge, E_z on its (x-, y-) edge (low corners).
template <class T>
__global__ void __launch_bounds__(kCtThreads) ct_edge_kernel(const T* __restrict__ f,
                                                               T* __restrict__ edge, int nx,
                                                               int ny, int nz, long long nc) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    const CellIndex q(c, nx, ny, nz);
    auto at = [&](int plane, int i, int j, int k) -> T {
      return f[plane * nc + ((long long)k * ny + j) * nx + i];
    };
    const int i = q.i, j = q.j, k = q.k;
    // E_z at (i-1/2, j-1/2): a = x, b = y
    edge[2 * nc + c] = ct_contact(
        at(kCtXEz, i, q.jm, k), at(kCtXEz, i, j, k), at(kCtXFm, i, q.jm, k), at(kCtXFm, i, j, k),
        at(kCtYEz, q.im, j, k), at(kCtYEz, i, j, k), at(kCtYFm, q.im, j, k), at(kCtYFm, i, j, k),
        at(kCtEcz, q.im, q.jm, k), at(kCtEcz, q.im, j, k), at(kCtEcz, i, q.jm, k),
        at(kCtEcz, i, j, k));
    // E_x at (j-1/2, k-1/2): a = y, b = z
    edge[c] = ct_contact(
        at(kCtYEx, i, j, q.km), at(kCtYEx, i, j, k), at(kCtYFm, i, j, q.km), at(kCtYFm, i, j, k),
        at(kCtZEx, i, q.jm, k), at(kCtZEx, i, j, k), at(kCtZFm, i, q.jm, k), at(kCtZFm, i, j, k),
        at(kCtEcx, i, q.jm, q.km), at(kCtEcx, i, q.jm, k), at(kCtEcx, i, j, q.km),
        at(kCtEcx, i, j, k));
    // E_y at (k-1/2, i-1/2): a = z, b = x
    edge[nc + c] = ct_contact(
        at(kCtZEy, q.im, j, k), at(kCtZEy, i, j, k), at(kCtZFm, q.im, j, k), at(kCtZFm, i, j, k),
        at(kCtXEy, i, j, q.km), at(kCtXEy, i, j, k), at(kCtXFm, i, j, q.km), at(kCtXFm, i, j, k),
        at(kCtEcy, q.im, j, q.km), at(kCtEcy, i, j, q.km), at(kCtEcy, q.im, j, k),
        at(kCtEcy, i, j, k));
  }
}

// Faraday's law on each cell's three lower faces and the Runge-Kutta
// combination: bout = a_n bn + a_w (bw - dt curl E) (STAGE 1: bw - dt curl E).
// bout may alias bn or bw (each thread reads only its own faces of those).
template <class T>
__global__ void __launch_bounds__(kCtThreads) ct_face_kernel(
    const T* __restrict__ edge, const T* bw, const T* bn, T* bout, int nx, int ny, int nz,
    long long nc, const StepScalars* __restrict__ scp, int first, T a_n, T a_w) {
  const StepScalars& sc = *scp;
  const T dtdx = T(sc.dtdx[0]), dtdy = T(sc.dtdx[1]), dtdz = T(sc.dtdx[2]);
  const bool frozen = !(sc.dt != 0.0);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    const CellIndex q(c, nx, ny, nz);
    auto E = [&](int e, int i, int j, int k) -> T {
      return edge[e * nc + ((long long)k * ny + j) * nx + i];
    };
    const int i = q.i, j = q.j, k = q.k;
    const T ex = E(0, i, j, k), ey = E(1, i, j, k), ez = E(2, i, j, k);
    T db[3];
    db[0] = dtdy * (E(2, i, q.jp, k) - ez) - dtdz * (E(1, i, j, q.kp) - ey);
    db[1] = dtdz * (E(0, i, j, q.kp) - ex) - dtdx * (E(2, q.ip, j, k) - ez);
    db[2] = dtdx * (E(1, q.ip, j, k) - ey) - dtdy * (E(0, i, q.jp, k) - ex);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T s1 = bw[d * nc + c] - (frozen ? T(0) : db[d]);
      bout[d * nc + c] = first ? s1 : a_n * bn[d * nc + c] + a_w * s1;
    }
  }
}

// Cell-centred B of U = mean of the cell's two faces; LAST: also the max
// wave speed of the new state (NaN-sticky; one FP64-bit atomicMax per CTA).
// Floors are counted by the stage kernels (per stage input), not here.
template <class T, bool LAST>
__global__ void __launch_bounds__(kCtThreads) ct_cell_kernel(const T* __restrict__ b, T* U,
                                                               int nx, int ny, int nz,
                                                               long long nc, Phys<T> ph,
                                                               unsigned long long* lam_bits) {
  __shared__ double wmax[kCtThreads / 32];
  T lam = T(0);
  unsigned flags = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    const CellIndex q(c, nx, ny, nz);
    const long long row = ((long long)q.k * ny + q.j) * nx;
    const T bx = T(0.5) * (b[c] + b[row + q.ip]);
    const T by = T(0.5) * (b[nc + c] + b[nc + ((long long)q.k * ny + q.jp) * nx + q.i]);
    const T bz = T(0.5) * (b[2 * nc + c] + b[2 * nc + ((long long)q.kp * ny + q.j) * nx + q.i]);
    U[kBX * nc + c] = bx;
    U[kBY * nc + c] = by;
    U[kBZ * nc + c] = bz;
    if constexpr (LAST) {
      T u[kNV];
#pragma unroll
      for (int v = 0; v < kNV; ++v) u[v] = U[v * nc + c];
      u[kBX] = bx;
      u[kBY] = by;
      u[kBZ] = bz;
      lam = nan_max(lam, cell_max_speed(u, ph, 3, flags));
    }
  }
  if constexpr (LAST) {
    double l = (double)lam;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l = nan_max(l, __shfl_xor_sync(0xffffffffu, l, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = wmax[0];
      for (int w = 1; w < kCtThreads / 32; ++w) m = nan_max(m, wmax[w]);
      unsigned long long bits = (unsigned long long)__double_as_longlong(m);
      if (m != m) bits = 0x7ff8000000000000ull;
      atomicMax(lam_bits, bits);
    }
  }
}

// After the caller set the face field: cell-centred B := face means, with the
// total energy adjusted (in FP64) so that the pressure is unchanged.  A cell
// whose B already equals its face means keeps its energy bit for bit.
template <class T>
__global__ void __launch_bounds__(kCtThreads) ct_set_cells_kernel(const T* __restrict__ b,
                                                                    T* U, int nx, int ny,
                                                                    int nz, long long nc) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    const CellIndex q(c, nx, ny, nz);
    const long long row = ((long long)q.k * ny + q.j) * nx;
    const T bn[3] = {T(0.5) * (b[c] + b[row + q.ip]),
                     T(0.5) * (b[nc + c] + b[nc + ((long long)q.k * ny + q.jp) * nx + q.i]),
                     T(0.5) * (b[2 * nc + c] +
                               b[2 * nc + ((long long)q.kp * ny + q.j) * nx + q.i])};
    double dE = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double o = (double)U[(kBX + d) * nc + c], nw = (double)bn[d];
      dE += 0.5 * (nw * nw - o * o);
      U[(kBX + d) * nc + c] = bn[d];
    }
    if (dE != 0.0) U[kPRS * nc + c] = T((double)U[kPRS * nc + c] + dE);
  }
}

// max over cells of |sum_d (b_d(+1/2) - b_d(-1/2)) / dx_d| (FP64), as bits.
template <class T>
__global__ void __launch_bounds__(kCtThreads) ct_divb_kernel(const T* __restrict__ b, int nx,
                                                               int ny, int nz, long long nc,
                                                               double idx, double idy,
                                                               double idz,
                                                               unsigned long long* out_bits) {
  __shared__ double wmax[kCtThreads / 32];
  double m = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    const CellIndex q(c, nx, ny, nz);
    const long long row = ((long long)q.k * ny + q.j) * nx;
    const double dv =
        ((double)b[row + q.ip] - (double)b[c]) * idx +
        ((double)b[nc + ((long long)q.k * ny + q.jp) * nx + q.i] - (double)b[nc + c]) * idy +
        ((double)b[2 * nc + ((long long)q.kp * ny + q.j) * nx + q.i] - (double)b[2 * nc + c]) *
            idz;
    m = nan_max(m, fabs(dv));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = nan_max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = wmax[0];
    for (int w = 1; w < kCtThreads / 32; ++w) r = nan_max(r, wmax[w]);
    unsigned long long bits = (unsigned long long)__double_as_longlong(r);
    if (r != r) bits = 0x7ff8000000000000ull;
    atomicMax(out_bits, bits);
  }
}

inline int ct_blocks(const Grid& g) {
  const long long need = (g.ncell + kCtThreads - 1) / kCtThreads;
  const long long cap = (long long)g.nsm * 8;
  return (int)(need < cap ? need : cap);
}

}  // namespace

template <class T>
cudaError_t launch_ct_edges(const Grid& g, const T* ctf, T* edge, cudaStream_t s) {
  ct_edge_kernel<T><<<ct_blocks(g), kCtThreads, 0, s>>>(ctf, edge, g.n[0], g.n[1], g.n[2],
                                                         g.ncell);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_ct_faces(const Grid& g, bool first, const T* edge, const T* bw, const T* bn,
                            T* bout, const StepScalars* sc, double a_n, double a_w,
                            cudaStream_t s) {
  ct_face_kernel<T><<<ct_blocks(g), kCtThreads, 0, s>>>(edge, bw, bn ? bn : bw, bout, g.n[0],
                                                         g.n[1], g.n[2], g.ncell, sc,
                                                         first ? 1 : 0, T(a_n), T(a_w));
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_ct_cells(const Grid& g, bool last, const T* b, T* U,
                            unsigned long long* lam_bits, cudaStream_t s) {
  const Phys<T> ph = make_phys<T>(g);
  if (last)
    ct_cell_kernel<T, true><<<ct_blocks(g), kCtThreads, 0, s>>>(
        b, U, g.n[0], g.n[1], g.n[2], g.ncell, ph, lam_bits);
  else
    ct_cell_kernel<T, false><<<ct_blocks(g), kCtThreads, 0, s>>>(
        b, U, g.n[0], g.n[1], g.n[2], g.ncell, ph, lam_bits);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_ct_set_cells(const Grid& g, const T* b, T* U, cudaStream_t s) {
  ct_set_cells_kernel<T><<<ct_blocks(g), kCtThreads, 0, s>>>(b, U, g.n[0], g.n[1], g.n[2],
                                                              g.ncell);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_ct_divb(const Grid& g, const T* b, unsigned long long* out_bits,
                           cudaStream_t s) {
  ct_divb_kernel<T><<<ct_blocks(g), kCtThreads, 0, s>>>(
      b, g.n[0], g.n[1], g.n[2], g.ncell, 1.0 / g.dx[0], 1.0 / g.dx[1], 1.0 / g.dx[2],
      out_bits);
  return cudaGetLastError();
}

#define MHD_CT_INSTANTIATE(T)                                                                \
  template cudaError_t launch_ct_edges<T>(const Grid&, const T*, T*, cudaStream_t);          \
  template cudaError_t launch_ct_faces<T>(const Grid&, bool, const T*, const T*, const T*,   \
                                          T*, const StepScalars*, double, double,            \
                                          cudaStream_t);                                     \
  template cudaError_t launch_ct_cells<T>(const Grid&, bool, const T*, T*,                   \
                                          unsigned long long*, cudaStream_t);                \
  template cudaError_t launch_ct_set_cells<T>(const Grid&, const T*, T*, cudaStream_t);      \
  template cudaError_t launch_ct_divb<T>(const Grid&, const T*, unsigned long long*,         \
                                         cudaStream_t);
MHD_CT_INSTANTIATE(double)
MHD_CT_INSTANTIATE(float)
#undef MHD_CT_INSTANTIATE

}  // namespace mhd
