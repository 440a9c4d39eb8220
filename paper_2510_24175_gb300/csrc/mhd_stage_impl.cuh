// Launch-shape selection and instantiation of the fused stage kernel for one
// arithmetic type.  Included once per type by mhd_stage_f64.cu / _f32.cu.
#pragma once

#include "mhd_internal.h"
#include "mhd_stage_weno.cuh"

namespace mhd {

// Tile shapes: 3-D grids use 32 x 8 column tiles marching in z.  FP64 runs
// 16 warps per CTA (one CTA per SM: 201 KB of shared memory): the SM's FP64
// unit is shared by all its warps and one warp issues an FP64 instruction at
// most every 64 clocks, so the unit saturates only when at least four warps
// have FP64 work; 16 warps (8 helper warps, 8 column owners) keep more warps
// busy through the phases than 13 and cap registers at 128 as 13 do (four
// warps per scheduler).  FP32 runs 8 warps and two CTAs per SM.  2-D grids
// use the same tile with a single plane; 1-D grids a 32-cell row.
template <class T>
struct StageShape3D {
  static constexpr int TY = 8;
  static constexpr int NW = sizeof(T) == 8 ? 16 : 8;
};

// The dynamic shared-memory limit of a kernel is set once per device (a
// driver call per launch costs more than a small grid's kernel).  One flag
// word per kernel: the template argument is the kernel itself.
template <auto KERN>
static cudaError_t set_smem_once(size_t smem) {
  static unsigned long long done = 0;  // bit d: set on device d (d < 64)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(KERN, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done |= bit;
  return e;
}

template <class T, int TY, int NW, int STAGE, bool ZACT, bool CT = false, bool HALO = false>
static cudaError_t launch_one(const StageParams<T>& p, dim3 grid, cudaStream_t s) {
  using G = TileGeom<TY, ZACT>;
  const size_t smem = (size_t)G::WORDS * sizeof(T);
  auto kern = rk_stage_kernel<T, TY, NW, STAGE, ZACT, CT, HALO>;
  cudaError_t e = set_smem_once<rk_stage_kernel<T, TY, NW, STAGE, ZACT, CT, HALO>>(smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NW * 32, smem, s>>>(p);
  return cudaGetLastError();
}

template <class T, int TY, int NW, int STAGE, bool ZACT, bool CT = false, bool HALO = false>
static cudaError_t launch_weno(const StageParams<T>& p, dim3 grid, cudaStream_t s) {
  using G = WenoGeom<TY, ZACT>;
  const size_t smem = (size_t)G::WORDS * sizeof(T);
  auto kern = rk_stage_weno_kernel<T, TY, NW, STAGE, ZACT, CT, HALO>;
  cudaError_t e = set_smem_once<rk_stage_weno_kernel<T, TY, NW, STAGE, ZACT, CT, HALO>>(smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NW * 32, smem, s>>>(p);
  return cudaGetLastError();
}

// WENO-Z tiles of 3-D grids.  FP64: 32 x 4 columns, 8 warps (the
// face-value phase gives every warp two cells' worth of work), one CTA per
// SM (166 KB of shared memory).  FP32: 32 x 8 columns, 16 warps (8 helper
// warps, 8 column owners), one CTA per SM (154 KB): the three-deep y halo
// is then 6 rows per 8 instead of per 4, and the kernel ran 8 % faster with
// GLM and 5 % with constrained transport than with 32 x 4 tiles at two
// 8-warp CTAs per SM.  2-D grids use 32 x 4 tiles with a single plane.
template <class T>
struct WenoShape3D {
  static constexpr int TY = sizeof(T) == 8 ? 4 : 8;
  static constexpr int NW = sizeof(T) == 8 ? 8 : 16;
};

template <class T>
void stage_shape(const Grid& g, size_t* smem, int* threads, int* ty) {
  if (g.limiter == kLimWenoz) {
    if (g.ndim == 3) {
      using WS = WenoShape3D<T>;
      *smem = (size_t)WenoGeom<WS::TY, true>::WORDS * sizeof(T);
      *threads = WS::NW * 32;
      *ty = WS::TY;
    } else if (g.ndim == 2) {
      *smem = (size_t)WenoGeom<4, false>::WORDS * sizeof(T);
      *threads = 256;
      *ty = 4;
    } else {
      *smem = (size_t)WenoGeom<1, false>::WORDS * sizeof(T);
      *threads = 32;
      *ty = 1;
    }
    return;
  }
  if (g.ndim == 3) {
    using S = StageShape3D<T>;
    *smem = (size_t)TileGeom<S::TY, true>::WORDS * sizeof(T);
    *threads = S::NW * 32;
    *ty = S::TY;
  } else if (g.ndim == 2) {
    *smem = (size_t)TileGeom<8, false>::WORDS * sizeof(T);
    *threads = 8 * 32;
    *ty = 8;
  } else {
    *smem = (size_t)TileGeom<1, false>::WORDS * sizeof(T);
    *threads = 32;
    *ty = 1;
  }
}

// Sets the shared-memory limit of every stage-kernel variant a grid launches
// (stages 1, 2, 3; constrained transport or not), so that no launch needs the
// driver call later, e.g. while a stream is being captured.
template <class T>
cudaError_t prepare_stage_kernels(const Grid& g, bool ct) {
  cudaError_t e = cudaSuccess;
  // the three stages of one variant <TY, NW, 3-D, CT> with geometry G
#define MHD_SET1(KERN, G, TY_, NW_, S_, Z_, CT_) \
  if (e == cudaSuccess) e = set_smem_once<KERN<T, TY_, NW_, S_, Z_, CT_>>((size_t)G::WORDS * sizeof(T))
#define MHD_SET3(KERN, G, TY_, NW_, Z_, CT_)   \
  MHD_SET1(KERN, G, TY_, NW_, 1, Z_, CT_);     \
  MHD_SET1(KERN, G, TY_, NW_, 2, Z_, CT_);     \
  MHD_SET1(KERN, G, TY_, NW_, 3, Z_, CT_)
  using S = StageShape3D<T>;
  using WS = WenoShape3D<T>;
  using W3 = WenoGeom<WS::TY, true>;
  using W2 = WenoGeom<4, false>;
  using W1 = WenoGeom<1, false>;
  using P3 = TileGeom<S::TY, true>;
  using P2 = TileGeom<8, false>;
  using P1 = TileGeom<1, false>;
  if (ct) {
    if (g.limiter == kLimWenoz) {
      MHD_SET3(rk_stage_weno_kernel, W3, WS::TY, WS::NW, true, true);
    } else {
      MHD_SET3(rk_stage_kernel, P3, S::TY, S::NW, true, true);
    }
  } else if (sizeof(T) == 8 && g.ndim == 3) {
    e = prepare_stage_kernels_halo<T>(g);  // FP64 3-D GLM: the halo-capable kernels
  } else if (g.limiter == kLimWenoz) {
    if (g.ndim == 3) {
      if constexpr (sizeof(T) == 4) {
        MHD_SET3(rk_stage_weno_kernel, W3, WS::TY, WS::NW, true, false);
      }
    } else if (g.ndim == 2) {
      MHD_SET3(rk_stage_weno_kernel, W2, 4, 8, false, false);
    } else {
      MHD_SET3(rk_stage_weno_kernel, W1, 1, 1, false, false);
    }
  } else if (g.ndim == 3) {
    if constexpr (sizeof(T) == 4) {
      MHD_SET3(rk_stage_kernel, P3, S::TY, S::NW, true, false);
    }
  } else if (g.ndim == 2) {
    MHD_SET3(rk_stage_kernel, P2, 8, 8, false, false);
  } else {
    MHD_SET3(rk_stage_kernel, P1, 1, 1, false, false);
  }
#undef MHD_SET3
#undef MHD_SET1
  return e;
}

// Kernel parameters shared by launch_stage and launch_stage_halo; returns
// cudaErrorInvalidValue for a bad z range.
template <class T>
static cudaError_t stage_params(StageParams<T>& p, const Grid& g, const T* win,
                                const T* un, T* uout, const StepScalars* sc,
                                unsigned long long* lam_bits, unsigned long long* floor_cnt,
                                double a_n, double a_w, int zlo, int zhi, int tz,
                                unsigned int* est_bits) {
  p.a_n = T(a_n);
  p.a_w = T(a_w);
  p.win = win;
  p.un = un;
  p.uout = uout;
  for (int d = 0; d < 3; ++d) {
    p.n[d] = g.n[d];
    p.bc_lo[d] = g.bc_lo[d];
    p.bc_hi[d] = g.bc_hi[d];
  }
  p.sy = g.n[0];
  p.sz = (long long)g.n[0] * g.n[1];
  p.sv = g.ncell;
  p.limiter = g.limiter;
  p.tz = g.ndim == 3 ? (tz > 0 ? tz : g.tz) : 1;
  p.zlo = g.ndim == 3 ? zlo : 0;
  p.zhi = g.ndim == 3 && zhi >= 0 ? zhi : g.n[2];
  if (p.zlo < 0 || p.zhi > g.n[2] || p.zlo >= p.zhi) return cudaErrorInvalidValue;
  p.ph = make_phys<T>(g);
  p.sc = sc;
  p.lam_bits = lam_bits;
  p.est_bits = est_bits;
  p.floor_cnt = floor_cnt;
  for (int d = 0; d < 3; ++d) p.bw[d] = nullptr;
  p.ctf = nullptr;
  for (int f = 0; f < 6; ++f) p.halo[f] = nullptr;
  return cudaSuccess;
}

template <class T>
cudaError_t launch_stage(const Grid& g, int stage, const T* win, const T* un, T* uout,
                         const StepScalars* sc, unsigned long long* lam_bits,
                         unsigned long long* floor_cnt, cudaStream_t stream, double a_n,
                         double a_w, const T* const* bw, T* ctf, int zlo, int zhi, int tz,
                         unsigned int* est_bits) {
  StageParams<T> p;
  cudaError_t pe = stage_params(p, g, win, un, uout, sc, lam_bits, floor_cnt, a_n, a_w, zlo,
                                zhi, tz, est_bits);
  if (pe != cudaSuccess) return pe;
  const int nzc = (p.zhi - p.zlo + p.tz - 1) / p.tz;  // z chunks of this launch
  // the FP64 last stage publishes the maximum speed estimate (speed_exact
  // finishes the maximum); it needs the estimate word
  if (sizeof(T) == 8 && stage == 2 && !ctf && !est_bits) return cudaErrorInvalidValue;
  for (int d = 0; d < 3; ++d) p.bw[d] = bw ? bw[d] : nullptr;
  p.ctf = ctf;
  if (ctf) {
    // constrained transport: 3-D grids only (checked when the context is made)
    if (g.ndim != 3 || !bw) return cudaErrorInvalidValue;
    if (g.limiter == kLimWenoz) {
      using WS = WenoShape3D<T>;
      dim3 grid((g.n[0] + 31) / 32, (g.n[1] + WS::TY - 1) / WS::TY, nzc);
      if (stage == 1) return launch_weno<T, WS::TY, WS::NW, 1, true, true>(p, grid, stream);
      if (stage == 2) return launch_weno<T, WS::TY, WS::NW, 2, true, true>(p, grid, stream);
      return launch_weno<T, WS::TY, WS::NW, 3, true, true>(p, grid, stream);
    }
    using S = StageShape3D<T>;
    dim3 grid((g.n[0] + 31) / 32, (g.n[1] + S::TY - 1) / S::TY, nzc);
    if (stage == 1) return launch_one<T, S::TY, S::NW, 1, true, true>(p, grid, stream);
    if (stage == 2) return launch_one<T, S::TY, S::NW, 2, true, true>(p, grid, stream);
    return launch_one<T, S::TY, S::NW, 3, true, true>(p, grid, stream);
  }
  if constexpr (sizeof(T) == 8) {
    // FP64 3-D GLM: always the halo-capable kernels (no halo faces here), so
    // that a grid and the blocks of its decomposition run the same code
    if (g.ndim == 3)
      return launch_stage_halo<T>(g, stage, win, un, uout, sc, lam_bits, floor_cnt, stream, a_n,
                                  a_w, nullptr, est_bits, zlo, zhi, tz);
  }
  if (g.limiter == kLimWenoz) {
    if constexpr (sizeof(T) == 4) {
      if (g.ndim == 3) {
        using WS = WenoShape3D<T>;
        dim3 grid((g.n[0] + 31) / 32, (g.n[1] + WS::TY - 1) / WS::TY, nzc);
        if (stage == 1) return launch_weno<T, WS::TY, WS::NW, 1, true>(p, grid, stream);
        if (stage == 2) return launch_weno<T, WS::TY, WS::NW, 2, true>(p, grid, stream);
        return launch_weno<T, WS::TY, WS::NW, 3, true>(p, grid, stream);
      }
    }
    if (g.ndim == 2) {
      dim3 grid((g.n[0] + 31) / 32, (g.n[1] + 3) / 4, 1);
      if (stage == 1) return launch_weno<T, 4, 8, 1, false>(p, grid, stream);
      if (stage == 2) return launch_weno<T, 4, 8, 2, false>(p, grid, stream);
      return launch_weno<T, 4, 8, 3, false>(p, grid, stream);
    }
    dim3 grid((g.n[0] + 31) / 32, 1, 1);
    if (stage == 1) return launch_weno<T, 1, 1, 1, false>(p, grid, stream);
    if (stage == 2) return launch_weno<T, 1, 1, 2, false>(p, grid, stream);
    return launch_weno<T, 1, 1, 3, false>(p, grid, stream);
  }
  if constexpr (sizeof(T) == 4) {
    if (g.ndim == 3) {
      using S = StageShape3D<T>;
      dim3 grid((g.n[0] + 31) / 32, (g.n[1] + S::TY - 1) / S::TY, nzc);
      if (stage == 1) return launch_one<T, S::TY, S::NW, 1, true>(p, grid, stream);
      if (stage == 2) return launch_one<T, S::TY, S::NW, 2, true>(p, grid, stream);
      return launch_one<T, S::TY, S::NW, 3, true>(p, grid, stream);
    }
  }
  if (g.ndim == 2) {
    dim3 grid((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, 1);
    if (stage == 1) return launch_one<T, 8, 8, 1, false>(p, grid, stream);
    if (stage == 2) return launch_one<T, 8, 8, 2, false>(p, grid, stream);
    return launch_one<T, 8, 8, 3, false>(p, grid, stream);
  }
  dim3 grid((g.n[0] + 31) / 32, 1, 1);
  if (stage == 1) return launch_one<T, 1, 1, 1, false>(p, grid, stream);
  if (stage == 2) return launch_one<T, 1, 1, 2, false>(p, grid, stream);
  return launch_one<T, 1, 1, 3, false>(p, grid, stream);
}

// Halo faces (3-D GLM grids with kBcHalo sides): the HALO variants of the
// 3-D stage kernels, the ghost cells of those sides read from halo[f].
// Instantiated in mhd_stage_halo_f64.cu / _f32.cu only.
template <class T>
cudaError_t launch_stage_halo(const Grid& g, int stage, const T* win, const T* un, T* uout,
                              const StepScalars* sc, unsigned long long* lam_bits,
                              unsigned long long* floor_cnt, cudaStream_t stream, double a_n,
                              double a_w, const T* const* halo, unsigned int* est_bits, int zlo,
                              int zhi, int tz) {
  if (g.ndim != 3) return cudaErrorInvalidValue;
  StageParams<T> p;
  cudaError_t pe = stage_params(p, g, win, un, uout, sc, lam_bits, floor_cnt, a_n, a_w, zlo, zhi,
                                tz, est_bits);
  if (pe != cudaSuccess) return pe;
  if (sizeof(T) == 8 && stage == 2 && !est_bits) return cudaErrorInvalidValue;
  for (int f = 0; f < 6; ++f) {
    const bool lo = (f & 1) == 0;
    const int bc = lo ? g.bc_lo[f >> 1] : g.bc_hi[f >> 1];
    if (bc == kBcHalo && (!halo || !halo[f])) return cudaErrorInvalidValue;
    p.halo[f] = bc == kBcHalo ? halo[f] : nullptr;
  }
  const int nzc = (p.zhi - p.zlo + p.tz - 1) / p.tz;
  if (g.limiter == kLimWenoz) {
    using WS = WenoShape3D<T>;
    dim3 grid((g.n[0] + 31) / 32, (g.n[1] + WS::TY - 1) / WS::TY, nzc);
    if (stage == 1) return launch_weno<T, WS::TY, WS::NW, 1, true, false, true>(p, grid, stream);
    if (stage == 2) return launch_weno<T, WS::TY, WS::NW, 2, true, false, true>(p, grid, stream);
    return launch_weno<T, WS::TY, WS::NW, 3, true, false, true>(p, grid, stream);
  }
  using S = StageShape3D<T>;
  dim3 grid((g.n[0] + 31) / 32, (g.n[1] + S::TY - 1) / S::TY, nzc);
  if (stage == 1) return launch_one<T, S::TY, S::NW, 1, true, false, true>(p, grid, stream);
  if (stage == 2) return launch_one<T, S::TY, S::NW, 2, true, false, true>(p, grid, stream);
  return launch_one<T, S::TY, S::NW, 3, true, false, true>(p, grid, stream);
}

// The shared-memory limits of the HALO variants (set once, outside any capture).
template <class T>
cudaError_t prepare_stage_kernels_halo(const Grid& g) {
  cudaError_t e = cudaSuccess;
  using S = StageShape3D<T>;
  using WS = WenoShape3D<T>;
  using W3 = WenoGeom<WS::TY, true>;
  using P3 = TileGeom<S::TY, true>;
  const size_t sw = (size_t)W3::WORDS * sizeof(T), sp = (size_t)P3::WORDS * sizeof(T);
  if (g.limiter == kLimWenoz) {
    if (e == cudaSuccess) e = set_smem_once<rk_stage_weno_kernel<T, WS::TY, WS::NW, 1, true, false, true>>(sw);
    if (e == cudaSuccess) e = set_smem_once<rk_stage_weno_kernel<T, WS::TY, WS::NW, 2, true, false, true>>(sw);
    if (e == cudaSuccess) e = set_smem_once<rk_stage_weno_kernel<T, WS::TY, WS::NW, 3, true, false, true>>(sw);
  } else {
    if (e == cudaSuccess) e = set_smem_once<rk_stage_kernel<T, S::TY, S::NW, 1, true, false, true>>(sp);
    if (e == cudaSuccess) e = set_smem_once<rk_stage_kernel<T, S::TY, S::NW, 2, true, false, true>>(sp);
    if (e == cudaSuccess) e = set_smem_once<rk_stage_kernel<T, S::TY, S::NW, 3, true, false, true>>(sp);
  }
  return e;
}

}  // namespace mhd
