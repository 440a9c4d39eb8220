// Fused RK2 stage kernel: one launch performs, for its tile of cells, the five
// per-stage steps of Section 3.2 (boundary calculation, cons->prim,
// reconstruction, Riemann solver, right-hand side) and the Runge-Kutta
// combination; stage 2 also applies the GLM damping (Mignone & Tzeferacos
// 2010, Eq. 27) and reduces the next step's max wave speed.
//
// Decomposition: a CTA owns a 32 x TY column tile in (x, y) and marches in z
// over p.tz planes.  Primitive variables of the current plane and its
// (x, y) halo live in a 4-plane shared-memory ring (planes k-1 .. k+2 feed the
// z faces of plane k).  Ghost zones are never stored: the boundary
// calculation is an index remap at load time (periodic: wrap; outflow: clamp
// to the nearest interior cell), so the state arrays are interior-only SoA.
// Each face flux of the tile is computed once and kept in shared memory;
// work items are grouped so that every warp handles faces of one direction.
#pragma once

#include "mhd_physics.cuh"

namespace mhd {

// Per-step scalars written on the device by the step-prepare kernel.
struct StepScalars {
  double dt;         // time step of the step in progress
  double ch;         // GLM cleaning speed c_h
  double dtdx[3];    // dt / dx_d
  double damp;       // exp(-alpha c_h dt / dh_min)
  double t;          // time after this step
  double lam;        // max wave speed the step's dt was taken from
  double steps;      // number of steps since set_state
};

template <class T>
struct StageParams {
  const T* win;   // stage input W (U^n or U1)
  const T* un;    // U^n (stage 2); may alias uout
  T* uout;        // stage output
  int n[3];
  long long sy, sz, sv;  // strides of y, z, var in elements
  int bc_lo[3], bc_hi[3];
  int limiter;
  int tz;         // planes per CTA
  Phys<T> ph;
  const StepScalars* sc;
  unsigned long long* lam_bits;   // stage 2: max wave speed as FP64 bits
  unsigned long long* floor_cnt;  // [2] floor activations
};

// Remaps a possibly out-of-range index (>= -2) into [0, n): periodic wraps,
// outflow clamps.  Indices beyond n+1 only occur in the unused part of a
// ragged tile and are folded to n+1 first, so every load stays in bounds.
__device__ __forceinline__ int remap(int i, int n, int lo, int hi) {
  i = min(i, n + 1);
  if (i < 0) return lo == kBcPeriodic ? i + n : 0;
  if (i >= n) return hi == kBcPeriodic ? i - n : n - 1;
  return i;
}

template <int TY, bool ZACT>
struct TileGeom {
  static constexpr int TX = 32;
  static constexpr int GX = 2;
  static constexpr int GY = TY > 1 ? 2 : 0;
  static constexpr int SX = TX + 2 * GX;
  static constexpr int SY = TY + 2 * GY;
  static constexpr int PLANE = SX * SY;               // ring cells per plane
  static constexpr int NRING = ZACT ? 4 : 1;
  static constexpr int NCROSS = TY * SX + 2 * GY * TX;  // cells loaded per plane
  static constexpr int FX = TY * (TX + 1);            // x faces per plane
  static constexpr int FY = GY ? (TY + 1) * TX : 0;   // y faces per plane
  static constexpr int FZ = ZACT ? TY * TX : 0;       // z faces per plane
  // shared-memory words
  static constexpr int RING_W = NRING * kNV * PLANE;
  static constexpr int FX_W = kNV * FX;
  static constexpr int FY_W = kNV * FY;
  static constexpr int FZ_W = 2 * kNV * FZ;
  static constexpr int WORDS = RING_W + FX_W + FY_W + FZ_W;
  // flux work items: warp-aligned segments [x main][y][z][x right edge]
  static constexpr int IT_X = TY * TX;
  static constexpr int IT_Y = FY;
  static constexpr int IT_Z = FZ;
  static constexpr int IT_XE = TY;
  static constexpr int ITEMS = IT_X + IT_Y + IT_Z + IT_XE;
};

template <class T, int TY, int NW, int STAGE, bool ZACT>
__global__ void __launch_bounds__(NW * 32, 1) rk_stage_kernel(const StageParams<T> p) {
  using G = TileGeom<TY, ZACT>;
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);
  T* Fx = ring + G::RING_W;
  T* Fy = Fx + G::FX_W;
  T* Fz = Fy + G::FY_W;

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * G::TX;
  const int y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * p.tz;
  const int z1 = min(z0 + p.tz, p.n[2]);
  const int nx = p.n[0], ny = p.n[1], nz = p.n[2];

  const StepScalars sc = *p.sc;
  const T ch = T(sc.ch);
  const T half_chi = T(0.5 / sc.ch);
  const T dtdx = T(sc.dtdx[0]), dtdy = T(sc.dtdx[1]), dtdz = T(sc.dtdx[2]);
  const T damp = T(sc.damp);
  const int lim = p.limiter;
  const Phys<T> ph = p.ph;
  unsigned flags = 0;

  // ---- load one plane (cons -> prim) into a ring slot -------------------
  auto load_plane = [&](int zz, int slot) {
    const int gz = ZACT ? remap(zz, nz, p.bc_lo[2], p.bc_hi[2]) : 0;
    T* dst = ring + slot * (kNV * G::PLANE);
    for (int it = tid; it < G::NCROSS; it += NT) {
      int r, c;
      if (it < TY * G::SX) {
        r = it / G::SX;
        c = it - r * G::SX - G::GX;
      } else {
        const int j = it - TY * G::SX;
        const int hr = j / G::TX;
        r = hr < G::GY ? hr - G::GY : TY + hr - G::GY;
        c = j - hr * G::TX;
      }
      const int gx = remap(x0 + c, nx, p.bc_lo[0], p.bc_hi[0]);
      const int gy = G::GY ? remap(y0 + r, ny, p.bc_lo[1], p.bc_hi[1]) : 0;
      const long long off = (long long)gz * p.sz + (long long)gy * p.sy + gx;
      T u[kNV], v[kNV];
#pragma unroll
      for (int k = 0; k < kNV; ++k) u[k] = p.win[k * p.sv + off];
      cons_to_prim(u, v, ph, flags);
      const int s = (r + G::GY) * G::SX + (c + G::GX);
#pragma unroll
      for (int k = 0; k < kNV; ++k) dst[k * G::PLANE + s] = v[k];
    }
  };

  // ---- face fluxes of plane k (x, y) and of face k+1/2 (z) --------------
  auto flux_items = [&](int k, bool z_only) {
    const int lo = z_only ? G::IT_X + G::IT_Y : 0;
    const int hi = z_only ? G::IT_X + G::IT_Y + G::IT_Z : G::ITEMS;
    const T* cur = ring + ((k & (G::NRING - 1)) * kNV * G::PLANE);
    for (int it = lo + tid; it < hi; it += NT) {
      T vl[kNV], vr[kNV], F[kNV];
      int dir;
      T* out;
      int ostride;
      if (it < G::IT_X || it >= G::IT_X + G::IT_Y + G::IT_Z) {
        int r, fi;
        if (it < G::IT_X) {
          r = it / G::TX;
          fi = it - r * G::TX;
        } else {
          r = it - (G::IT_X + G::IT_Y + G::IT_Z);
          fi = G::TX;
        }
        // face between tile cells fi-1 and fi: ring cols fi .. fi+3
        const T* b = cur + (r + G::GY) * G::SX + fi;
        plm_face_pair(b, b + 1, b + 2, b + 3, G::PLANE, lim, vl, vr);
        dir = 0;
        out = Fx + r * (G::TX + 1) + fi;
        ostride = G::FX;
      } else if (it < G::IT_X + G::IT_Y) {
        const int j = it - G::IT_X;
        const int fj = j / G::TX, c = j - fj * G::TX;
        const T* b = cur + fj * G::SX + (c + G::GX);
        plm_face_pair(b, b + G::SX, b + 2 * G::SX, b + 3 * G::SX, G::PLANE, lim, vl, vr);
        dir = 1;
        out = Fy + fj * G::TX + c;
        ostride = G::FY;
      } else {
        const int j = it - G::IT_X - G::IT_Y;
        const int r = j / G::TX, c = j - r * G::TX;
        const int s = (r + G::GY) * G::SX + (c + G::GX);
        const T* b0 = ring + (((k - 1) & 3) * kNV * G::PLANE) + s;
        const T* b1 = ring + (((k) & 3) * kNV * G::PLANE) + s;
        const T* b2 = ring + (((k + 1) & 3) * kNV * G::PLANE) + s;
        const T* b3 = ring + (((k + 2) & 3) * kNV * G::PLANE) + s;
        plm_face_pair(b0, b1, b2, b3, G::PLANE, lim, vl, vr);
        dir = 2;
        out = Fz + (k & 1) * (kNV * G::FZ) + j;
        ostride = G::FZ;
      }
      glm_hlld_flux(vl, vr, dir, ch, half_chi, ph, F);
#pragma unroll
      for (int q = 0; q < kNV; ++q) out[q * ostride] = F[q];
    }
  };

  if constexpr (ZACT) {
    for (int zz = z0 - 2; zz < z0 + 2; ++zz) load_plane(zz, zz & 3);
    __syncthreads();
    flux_items(z0 - 1, true);  // face z0 - 1/2
    __syncthreads();
  }

  T lam = T(0);
  for (int k = z0; k < z1; ++k) {
    if constexpr (ZACT) {
      load_plane(k + 2, (k + 2) & 3);
    } else {
      load_plane(0, 0);
    }
    __syncthreads();
    flux_items(k, false);
    __syncthreads();

    // ---- right-hand side and RK combination for plane k ------------------
    for (int it = tid; it < TY * G::TX; it += NT) {
      const int r = it / G::TX, c = it - r * G::TX;
      const int gx = x0 + c, gy = y0 + r;
      if (gx >= nx || gy >= ny) continue;
      const long long off = (long long)k * p.sz + (long long)gy * p.sy + gx;
      T unew[kNV];
#pragma unroll
      for (int q = 0; q < kNV; ++q) {
        const T* fx = Fx + q * G::FX + r * (G::TX + 1) + c;
        T du = (fx[1] - fx[0]) * dtdx;
        if constexpr (G::GY > 0) {
          const T* fy = Fy + q * G::FY + r * G::TX + c;
          du += (fy[G::TX] - fy[0]) * dtdy;
        }
        if constexpr (ZACT) {
          const T fp = Fz[(k & 1) * (kNV * G::FZ) + q * G::FZ + it];
          const T fm = Fz[((k - 1) & 1) * (kNV * G::FZ) + q * G::FZ + it];
          du += (fp - fm) * dtdz;
        }
        const T s1 = p.win[q * p.sv + off] - du;
        if constexpr (STAGE == 1) {
          unew[q] = s1;
        } else {
          unew[q] = T(0.5) * (p.un[q * p.sv + off] + s1);
        }
      }
      if constexpr (STAGE == 2) unew[kPSI] *= damp;
#pragma unroll
      for (int q = 0; q < kNV; ++q) p.uout[q * p.sv + off] = unew[q];
      if constexpr (STAGE == 2) {
        const int ndim = 1 + (G::GY > 0) + (ZACT ? 1 : 0);
        const T s = cell_max_speed(unew, ph, ndim, flags);
        if (!(s <= lam)) lam = s;  // keeps NaN
      }
    }
  }

  if constexpr (STAGE == 2) {
    // block max of the wave speed -> one FP64-bit atomicMax per CTA
    double l = (double)lam;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, l, o);
      if (!(other <= l)) l = other;
    }
    __shared__ double wmax[NW];
    __syncthreads();
    if ((tid & 31) == 0) wmax[tid >> 5] = l;
    __syncthreads();
    if (tid == 0) {
      double m = wmax[0];
      for (int w = 1; w < NW; ++w)
        if (!(wmax[w] <= m)) m = wmax[w];
      unsigned long long bits = (unsigned long long)__double_as_longlong(m);
      if (m != m) bits = 0x7ff8000000000000ull;
      atomicMax(p.lam_bits, bits);
    }
  }
  if (flags) {
    if (flags & kFloorRho) atomicAdd(&p.floor_cnt[0], 1ull);
    if (flags & kFloorP) atomicAdd(&p.floor_cnt[1], 1ull);
  }
}

}  // namespace mhd
