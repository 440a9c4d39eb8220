// Fused Runge-Kutta stage kernel: one launch performs, for its tile of cells,
// the five per-stage steps of Section 3.2 (boundary calculation,
// cons->prim, reconstruction, Riemann solver, right-hand side) and the
// Runge-Kutta combination.  STAGE 1: out = W + dt L(W); STAGE 2 (last stage):
// out = a_n U^n + a_w (W + dt L(W)), then the GLM damping (Mignone &
// Tzeferacos 2010, Eq. 27) and the next step's max-wave-speed reduction;
// STAGE 3 (SSP-RK3 middle stage): the combination without the epilogue.
//
// Decomposition: a CTA owns a 32 x TY column tile in (x, y) and marches in z
// over p.tz planes.  Ghost zones are never stored: the boundary calculation
// is an index remap at load time (periodic: wrap; outflow: clamp to the
// nearest interior cell), so the state arrays are interior-only SoA.
//
// Per plane k, four phases separated by CTA barriers:
//   A  load + cons->prim: the tile interior of plane k+2 (into a 3-plane
//      ring) and the (x, y) halo of plane k (into halo buffers);
//   B  limited slopes, each cell and direction once: x slopes of the 34
//      cells per row, y slopes of the TY+2 rows, and -- by the thread that
//      owns the column -- the z slope of cell k+1;
//   C  face fluxes (PLM face states V -/+ sigma/2, GLM, HLLD), each face of
//      the tile once, warp-uniform direction; the column owner also computes
//      the z face k+1/2 and keeps the z data (slope, face state, flux) of its
//      column in per-owner shared slots across planes;
//   D  the column owner applies the flux divergence and the RK combination.
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
  int zlo, zhi;   // z planes [zlo, zhi) of this launch (blockIdx.z counts tz-plane chunks)
  T a_n, a_w;     // combining stages: out = a_n U^n + a_w (W + dt L(W))
  Phys<T> ph;
  const StepScalars* sc;
  unsigned long long* lam_bits;   // stage 2: max wave speed as FP64 bits (FP32 path)
  unsigned int* est_bits;         // stage 2, FP64: max reliable FP32 speed estimate
  unsigned long long* floor_cnt;  // [3] floor activations (see count_floors)
  // constrained transport (kernels instantiated with CT = true)
  const T* bw[3];  // the stage input's face field: b_d on each cell's lower d-face
  T* ctf;          // kCtPlanes planes of ncell values (layout below)
  // halo faces (kernels instantiated with HALO = true): ghost cells beyond a
  // side whose bc is kBcHalo, per face x-, x+, y-, y+, z-, z+ (layout at
  // halo_cell below)
  const T* halo[6];
};

// HALO kernels: the address of variable 0 of cell (i, j, k) of the stage
// input and the variable stride, for indices up to GH cells outside the grid
// (GH = ghost width: 2 for PLM, 3 for WENO-Z).  A cell beyond a kBcHalo side
// comes from that face's halo buffer, which has the grid's SoA layout over
// the ghost slab: extent GH along the face normal (layer l = ghost index + GH
// on the low side, ghost index - n on the high side), the grid's extents
// along the two others.  Other out-of-range indices wrap (periodic) or clamp
// (outflow) as in remap().  The stage kernels never use a cell outside the
// grid along two axes at once, so when the chosen face's tangential indices
// are out of range the load is of an unused value and is clamped into the
// buffer; indices beyond n + GH - 1 (the unused part of a ragged tile) are
// folded first.  Every load stays in bounds.
template <int GH, class T>
__device__ __forceinline__ const T* halo_cell(const StageParams<T>& p, int i, int j, int k,
                                              long long& sv) {
  const int n0 = p.n[0], n1 = p.n[1], n2 = p.n[2];
  i = min(i, n0 + GH - 1);
  j = min(j, n1 + GH - 1);
  k = min(k, n2 + GH - 1);
  int f = -1, l = 0;
  if (k < 0 && p.bc_lo[2] == kBcHalo) {
    f = 4;
    l = k + GH;
  } else if (k >= n2 && p.bc_hi[2] == kBcHalo) {
    f = 5;
    l = k - n2;
  } else if (j < 0 && p.bc_lo[1] == kBcHalo) {
    f = 2;
    l = j + GH;
  } else if (j >= n1 && p.bc_hi[1] == kBcHalo) {
    f = 3;
    l = j - n1;
  } else if (i < 0 && p.bc_lo[0] == kBcHalo) {
    f = 0;
    l = i + GH;
  } else if (i >= n0 && p.bc_hi[0] == kBcHalo) {
    f = 1;
    l = i - n0;
  }
  if (f < 0) {
    auto wrap = [](int x, int n, int lo, int hi) {
      if (x < 0) return lo == kBcPeriodic ? x + n : 0;
      if (x >= n) return hi == kBcPeriodic ? x - n : n - 1;
      return x;
    };
    const int gx = wrap(i, n0, p.bc_lo[0], p.bc_hi[0]);
    const int gy = wrap(j, n1, p.bc_lo[1], p.bc_hi[1]);
    const int gz = wrap(k, n2, p.bc_lo[2], p.bc_hi[2]);
    sv = p.sv;
    return p.win + (long long)gz * p.sz + (long long)gy * p.sy + gx;
  }
  const int d = f >> 1;
  const int c0 = d == 0 ? l : min(max(i, 0), n0 - 1);
  const int c1 = d == 1 ? l : min(max(j, 0), n1 - 1);
  const int c2 = d == 2 ? l : min(max(k, 0), n2 - 1);
  const int e0 = d == 0 ? GH : n0, e1 = d == 1 ? GH : n1;
  const int e2 = d == 2 ? GH : n2;
  sv = (long long)e0 * e1 * e2;
  return p.halo[f] + ((long long)c2 * e1 + c1) * e0 + c0;
}

// Planes of the constrained-transport buffer written by a CT stage kernel,
// per cell: the electric field E = -v x B on the cell's lower x, y and z
// faces (the two components after the face normal in cyclic order, from the
// face flux: on a d-face E_{d+1} = F[B_{d+2}] and E_{d+2} = -F[B_{d+1}]), the
// mass flux through each of those faces (set to zero when
// |F_rho| <= delta c_h rho, delta = 1e-12 in FP64 and 1e-4 in FP32, so that
// round-off cannot pick an upwind side), and the cell-centred E.
enum : int {
  kCtXEy = 0, kCtXEz, kCtXFm, kCtYEz, kCtYEx, kCtYFm, kCtZEx, kCtZEy, kCtZFm,
  kCtEcx, kCtEcy, kCtEcz, kCtPlanes
};

template <class T>
__device__ __forceinline__ T ct_mass_flux(T f, T rho, T ch) {
  const T thr = T(sizeof(T) == 8 ? 1e-12 : 1e-4) * ch * rho;
  return tabs(f) > thr ? f : T(0);
}

// Constrained-transport data of the cell a column owner updates: the
// cell-centred E and rho (read in phase C, before the next plane's loads may
// reuse the ring slot) and the z flux through the cell's lower face.
template <class T>
struct CtCell {
  T ex, ey, ez, rho;
  T fz_bx, fz_by, fz_rho;
  __device__ __forceinline__ void from_prims(const T* v, int st) {
    const T vx = v[kVX * st], vy = v[kVY * st], vz = v[kVZ * st];
    const T bx = v[kBX * st], by = v[kBY * st], bz = v[kBZ * st];
    ex = vz * by - vy * bz;
    ey = vx * bz - vz * bx;
    ez = vy * bx - vx * by;
    rho = v[kRHO * st];
  }
  // fx / fy: the x and y fluxes of the cell's lower faces (variables sx / sy
  // apart)
  __device__ __forceinline__ void write(T* ctf, long long sv, long long off, const T* fx,
                                        int sx, const T* fy, int sy, T ch) const {
    ctf[kCtXEy * sv + off] = fx[kBZ * sx];
    ctf[kCtXEz * sv + off] = -fx[kBY * sx];
    ctf[kCtXFm * sv + off] = ct_mass_flux(fx[kRHO * sx], rho, ch);
    ctf[kCtYEz * sv + off] = fy[kBX * sy];
    ctf[kCtYEx * sv + off] = -fy[kBZ * sy];
    ctf[kCtYFm * sv + off] = ct_mass_flux(fy[kRHO * sy], rho, ch);
    ctf[kCtZEx * sv + off] = fz_by;
    ctf[kCtZEy * sv + off] = -fz_bx;
    ctf[kCtZFm * sv + off] = ct_mass_flux(fz_rho, rho, ch);
    ctf[kCtEcx * sv + off] = ex;
    ctf[kCtEcy * sv + off] = ey;
    ctf[kCtEcz * sv + off] = ez;
  }
};

// Constrained transport: both sides of a d-face carry the staggered normal
// field and psi = 0 (the GLM interface step is then the identity).
template <class T>
__device__ __forceinline__ void ct_face_field(T vl[kNV], T vr[kNV], int d, T bn) {
  vl[kBX + d] = vr[kBX + d] = bn;
  vl[kPSI] = vr[kPSI] = T(0);
}

// Remaps a possibly out-of-range index (>= -2) into [0, n): periodic wraps,
// outflow clamps.  Indices beyond n+1 only occur in the unused part of a
// ragged tile and are folded to n+1 first, so every load stays in bounds.
__host__ __device__ __forceinline__ int remap(int i, int n, int lo, int hi) {
  i = min(i, n + 1);
  if (i < 0) return lo == kBcPeriodic ? i + n : 0;
  if (i >= n) return hi == kBcPeriodic ? i - n : n - 1;
  return i;
}

// Same for a three-cell-deep halo (WENO-Z; active dimensions need n >= 3).
__host__ __device__ __forceinline__ int remap3(int i, int n, int lo, int hi) {
  i = min(i, n + 2);
  if (i < 0) return lo == kBcPeriodic ? i + n : 0;
  if (i >= n) return hi == kBcPeriodic ? i - n : n - 1;
  return i;
}

template <int TY, bool ZACT>
struct TileGeom {
  static constexpr int TX = 32;
  static constexpr int GY = TY > 1 ? 2 : 0;
  static constexpr int NINT = TY * TX;             // interior cells per plane
  static constexpr int NXH = 4 * TY;               // x halo: columns -2, -1, 32, 33
  static constexpr int NYH = GY ? 4 * TX : 0;      // y halo: rows -2, -1, TY, TY+1
  static constexpr int NRING = ZACT ? 3 : 1;
  // shared-memory words
  // Variable stride PS of the ring slots and of the halo buffer: the x and y
  // halo cells share one buffer (x halo items first, then y halo items) with
  // the ring's stride, so every cell of the current plane is reached at a
  // compile-time stride; PS = NINT unless the halo cells are more (TY = 4)
  static constexpr int PS = NINT > NXH + NYH ? NINT : NXH + NYH;
  static constexpr int RING_W = NRING * kNV * PS;
  static constexpr int HB_W = kNV * PS;
  static constexpr int SXN = TY * (TX + 2);         // x slopes, columns -1..32
  static constexpr int SYN = GY ? (TY + 2) * TX : 0;  // y slopes, rows -1..TY
  static constexpr int FXN = TY * (TX + 1);
  static constexpr int FYN = GY ? (TY + 1) * TX : 0;
  static constexpr int Z_W = ZACT ? 3 * kNV * NINT : 0;  // z slope, z face state, z flux
  static constexpr int WORDS =
      RING_W + HB_W + kNV * SXN + kNV * SYN + kNV * FXN + kNV * FYN + Z_W;
  // phase-A items: interior, x halo, y halo
  static constexpr int NLOAD = NINT + NXH + NYH;
  // phase-C flux items, warp-aligned segments [x main][y][x right edge]
  static constexpr int IT_X = TY * TX;
  static constexpr int IT_Y = FYN;
  static constexpr int IT_XE = TY;
  static constexpr int ITEMS = IT_X + IT_Y + IT_XE;
};

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// FP32 limited slopes of two variables at once: the one-sided differences,
// their product, the doubled minimum and the halved sum in packed FP32; the
// per-lane comparisons, minima and sign choices as limited_slope<float>
// takes them (the same values).
__device__ __forceinline__ float2 limited_slope2(float2 dm, float2 dp, int lim) {
  const float2 pr = mul2(dm, dp);
  float2 mag = pk(fminf(fabsf(dm.x), fabsf(dp.x)), fminf(fabsf(dm.y), fabsf(dp.y)));
  if (lim == kLimMC) {
    const float2 two = mul2(pk1(2.0f), mag);
    const float2 sum = add2(dm, dp);
    const float2 cen = mul2(pk1(0.5f), pk(fabsf(sum.x), fabsf(sum.y)));
    mag = pk(fminf(two.x, cen.x), fminf(two.y, cen.y));
  }
  const bool okx = lim != kLimFlat && pr.x > 0.0f, oky = lim != kLimFlat && pr.y > 0.0f;
  return pk(okx ? (dm.x > 0.0f ? mag.x : -mag.x) : 0.0f,
            oky ? (dm.y > 0.0f ? mag.y : -mag.y) : 0.0f);
}
#endif

// Limited slopes of the 9 primitives of one cell from its two neighbours
// along a direction, with the zero-slope fallback when a face density or
// pressure would be non-positive.  PAIRED: FP32 on the device pairs the
// variables (0, 1) ... (6, 7) in packed instructions (the same values; fewer
// instructions, more registers live).
template <class T, bool PAIRED = true>
__device__ __forceinline__ void cell_slopes(const T* m, int sm, const T* c, int sc, const T* p,
                                            int sp, int lim, T sig[kNV]) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  if constexpr (PAIRED && sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k + 1 < kNV; k += 2) {
      const float2 q = pk(c[k * sc], c[(k + 1) * sc]);
      const float2 dm = sub2(q, pk(m[k * sm], m[(k + 1) * sm]));
      const float2 dp = sub2(pk(p[k * sp], p[(k + 1) * sp]), q);
      const float2 s2 = limited_slope2(dm, dp, lim);
      sig[k] = s2.x;
      sig[k + 1] = s2.y;
    }
    {
      const T q = c[(kNV - 1) * sc];
      sig[kNV - 1] = limited_slope(q - m[(kNV - 1) * sm], p[(kNV - 1) * sp] - q, lim);
    }
    const bool ok = gt0(c[kRHO * sc] - T(0.5) * tabs(sig[kRHO])) &&
                    gt0(c[kPRS * sc] - T(0.5) * tabs(sig[kPRS]));
    if (!ok) {
#pragma unroll
      for (int k = 0; k < kNV; ++k) sig[k] = T(0);
    }
    return;
  }
#endif
#pragma unroll
  for (int k = 0; k < kNV; ++k) {
    const T q = c[k * sc];
    sig[k] = limited_slope(q - m[k * sm], p[k * sp] - q, lim);
  }
  const bool ok = gt0(c[kRHO * sc] - T(0.5) * tabs(sig[kRHO])) &&
                  gt0(c[kPRS * sc] - T(0.5) * tabs(sig[kPRS]));
  if (!ok) {
#pragma unroll
    for (int k = 0; k < kNV; ++k) sig[k] = T(0);
  }
}

// One tile (bx, by, bz) of one RK stage; called by every thread of a CTA of
// NW warps.  smem_raw: TileGeom::WORDS elements of T; wmax: NW doubles.
// CT (constrained transport, 3-D only): face-normal fields from p.bw, only
// rho, m and E are updated (psi is written as 0; the magnetic field is left to
// the face update), the face / cell electric fields go to p.ctf, and the last
// stage has no damping and no wave-speed reduction (done after the face update).
// HALO (3-D, not CT): ghost cells of kBcHalo sides from p.halo (halo_cell).
template <class T, int TY, int NW, int STAGE, bool ZACT, bool CT = false, bool HALO = false,
          bool PREFETCH = true>
__device__ __forceinline__ void stage_tile(const StageParams<T>& p, const StepScalars& sc,
                                           int bx, int by, int bz, unsigned char* smem_raw,
                                           double* wmax) {
  using G = TileGeom<TY, ZACT>;
  constexpr int NT = NW * 32;
  constexpr int TX = G::TX;
  constexpr int ZT0 = NT - G::NINT;  // threads ZT0.. own one tile column each
  static_assert(ZT0 >= 0, "need one thread per tile column");
  T* ring = reinterpret_cast<T*>(smem_raw);
  T* xh = ring + G::RING_W;  // x halo items (variable stride G::PS)
  T* yh = xh + G::NXH;        // y halo items (same buffer and stride)
  T* sxs = xh + G::HB_W;
  T* sys = sxs + kNV * G::SXN;
  T* Fx = sys + kNV * G::SYN;
  T* Fy = Fx + kNV * G::FXN;
  T* zS = Fy + kNV * G::FYN;  // per owner: z slope of cell k+1
  T* zP = zS + kNV * G::NINT;  // per owner: face state V_k + sigma_k / 2
  T* zF = zP + kNV * G::NINT;  // per owner: z flux at face k-1/2

  const int tid = threadIdx.x;
  const int x0 = bx * TX;
  const int y0 = by * TY;
  const int z0 = p.zlo + bz * p.tz;
  const int z1 = min(z0 + p.tz, p.zhi);
  const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
  const bool owner = tid >= ZT0;
  const int oidx = tid - ZT0;  // owned column = interior cell index r * TX + c
  const int orow = oidx / TX, ocol = oidx - (oidx / TX) * TX;

  const T ch = T(sc.ch);
  const T half_chi = T(0.5 / sc.ch);
  const T dtdx = T(sc.dtdx[0]), dtdy = T(sc.dtdx[1]), dtdz = T(sc.dtdx[2]);
  const T damp = T(sc.damp);
  // dt == 0 (a step at t_end, or one the prepare kernel turned into a no-op
  // after a non-finite wave speed): the state is copied through unchanged,
  // even where fluxes are not finite
  const bool frozen = !(sc.dt != 0.0);
  const int lim = p.limiter;
  const Phys<T> ph = p.ph;
  unsigned flags = 0;  // of the wave-speed conversions (not counted)

  auto slot = [](int zz) { return ZACT ? ((zz % 3) + 3) % 3 : 0; };
  auto ring_plane = [&](int zz) { return ring + slot(zz) * (kNV * G::PS); };

  // Floor activations are counted once per stage for each cell the tile
  // updates, from that cell's own conversion of the stage input; halo copies
  // converted by neighbouring tiles are not counted, so the counts do not
  // depend on the decomposition.  Rare: one atomic per flagged cell.
  auto count_floors = [&](unsigned fl, int zz, int r, int c) {
    if (zz < z0 || zz >= z1 || x0 + c >= nx || (G::GY && y0 + r >= ny)) return;
    if (fl & kFloorRho) atomicAdd(&p.floor_cnt[0], 1ull);
    if (fl & kFloorP) atomicAdd(&p.floor_cnt[1], 1ull);
    if (fl & kPressF64) atomicAdd(&p.floor_cnt[2], 1ull);
  };
  // cons -> prim of cell (r, c) of plane zz into dst (variables dst_stride
  // apart); own: an interior item of the tile (counted if the tile updates it)
  auto load_cell = [&](int zz, int r, int c, T* dst, int dst_stride, bool own) {
    T u[kNV], v[kNV];
    if constexpr (HALO) {
      long long hs;
      const T* a = halo_cell<2>(p, x0 + c, y0 + r, zz, hs);
#pragma unroll
      for (int k = 0; k < kNV; ++k) u[k] = a[k * hs];
    } else {
      const int gz = ZACT ? remap(zz, nz, p.bc_lo[2], p.bc_hi[2]) : 0;
      const int gx = remap(x0 + c, nx, p.bc_lo[0], p.bc_hi[0]);
      const int gy = G::GY ? remap(y0 + r, ny, p.bc_lo[1], p.bc_hi[1]) : 0;
      const long long off = (long long)gz * p.sz + (long long)gy * p.sy + gx;
#pragma unroll
      for (int k = 0; k < kNV; ++k) u[k] = p.win[k * p.sv + off];
    }
    unsigned fl = 0;
    cons_to_prim(u, v, ph, fl);
    if (fl && own) count_floors(fl, zz, r, c);
#pragma unroll
    for (int k = 0; k < kNV; ++k) dst[k * dst_stride] = v[k];
  };
  // FP32 kernels without halo faces or constrained transport, one thread per
  // interior column (NT = NINT): each thread's interior item of the next
  // iteration (plane k + 3) is fetched into registers one iteration ahead, so
  // that its global-load latency overlaps this plane's slope, flux and update
  // phases.  The same cells are read as without it, and converted by the same
  // code.  (PREFETCH = false: not done, for callers short of registers.)
  // The slopes are paired in packed FP32 where the prefetch is not done;
  // with the prefetch, pairing them as well (still within the 128 registers
  // of two CTAs per SM) ran slower than scalar slopes.
  constexpr bool PREF = PREFETCH && ZACT && !HALO && !CT && sizeof(T) == 4 && NT == G::NINT;
  T pre[kNV];
  auto fetch_interior = [&](int zz) {
    const int r = tid / TX, c = tid - (tid / TX) * TX;
    const int gz = remap(zz, nz, p.bc_lo[2], p.bc_hi[2]);
    const int gx = remap(x0 + c, nx, p.bc_lo[0], p.bc_hi[0]);
    const int gy = G::GY ? remap(y0 + r, ny, p.bc_lo[1], p.bc_hi[1]) : 0;
    const long long off = (long long)gz * p.sz + (long long)gy * p.sy + gx;
#pragma unroll
    for (int k = 0; k < kNV; ++k) pre[k] = p.win[k * p.sv + off];
  };
  auto convert_interior = [&](int zz) {
    const int r = tid / TX, c = tid - (tid / TX) * TX;
    T v[kNV];
    unsigned fl = 0;
    cons_to_prim(pre, v, ph, fl);
    if (fl) count_floors(fl, zz, r, c);
    T* dst = ring_plane(zz) + tid;
#pragma unroll
    for (int k = 0; k < kNV; ++k) dst[k * G::PS] = v[k];
  };
  // phase-A item: interior cell of plane zi or halo cell of plane zh
  auto load_item = [&](int it, int zi, int zh) {
    if (it < G::NINT) {
      const int r = it / TX, c = it - (it / TX) * TX;
      load_cell(zi, r, c, ring_plane(zi) + it, G::PS, true);
    } else if (it < G::NINT + G::NXH) {
      const int j = it - G::NINT;
      const int r = j >> 2, q = j & 3;
      const int c = q < 2 ? q - 2 : TX + q - 2;
      load_cell(zh, r, c, xh + j, G::PS, false);
    } else {
      const int j = it - G::NINT - G::NXH;
      const int hr = j / TX, c = j - (j / TX) * TX;
      const int r = hr < 2 ? hr - 2 : TY + hr - 2;
      load_cell(zh, r, c, yh + j, G::PS, false);
    }
  };
  // primitives of cell (r, c) of the current plane (interior in ring slot,
  // halo in the halo buffers); returns the pointer, stride in *st
  auto cell_ptr = [&](const T* cur, int r, int c, int* st) -> const T* {
    if (c < 0 || c >= TX) {
      *st = G::PS;
      return xh + r * 4 + (c < 0 ? c + 2 : c - TX + 2);
    }
    if (r < 0 || r >= TY) {
      *st = G::PS;
      return yh + (r < 0 ? r + 2 : r - TY + 2) * TX + c;
    }
    *st = G::PS;
    return cur + r * TX + c;
  };
  static_assert(!CT || ZACT, "constrained transport is 3-D only");
  static_assert(!HALO || (ZACT && !CT), "halo faces: 3-D GLM kernels only");
  // staggered normal field on the lower d-face of tile cell (r, c) of plane zz
  auto bface = [&](int d, int zz, int r, int c) -> T {
    const int gz = remap(zz, nz, p.bc_lo[2], p.bc_hi[2]);
    const int gx = remap(x0 + c, nx, p.bc_lo[0], p.bc_hi[0]);
    const int gy = remap(y0 + r, ny, p.bc_lo[1], p.bc_hi[1]);
    return p.bw[d][(long long)gz * p.sz + (long long)gy * p.sy + gx];
  };
  CtCell<T> ctc;

  // The z march: one loop body for every plane, so that each cell's
  // conversion, slopes and z fluxes come from the same code wherever a z
  // chunk (or a block of a decomposed grid, or a launch's z range) starts --
  // a cell's result must not depend on that decomposition.  Iterations
  // k < z0 warm up: k = z0-4 and z0-3 only load planes z0-2 and z0-1 into the
  // ring, k = z0-2 sets the column owners' face state of cell z0-1, k = z0-1
  // their flux through face z0-1/2; the x, y work and the update start at
  // k = z0.  (Unrolling, and with it the peeling of warm-up iterations into
  // separate copies, is disabled.)
  constexpr int NWARM = ZACT ? 4 : 0;
  SpeedMax<T> smax(ph);  // last stage: the new state's maximum wave speed
#pragma unroll 1
  for (int k = z0 - NWARM; k < z1; ++k) {
    const bool main = k >= z0;
    // FP32 (two CTAs per SM): the item loops of phases A-C start at a
    // thread index rotated by (k mod 4) whole warps.  A phase's items do not
    // divide evenly among the warps; without the rotation the warps left with
    // one item more are always the first ones, on the same schedulers in
    // both CTAs of an SM, and rotated they change from plane to plane.
    // Which thread takes an item does not change its result.
    const int rtid = sizeof(T) == 4 ? (tid + 32 * (k & 3)) % NT : tid;
    // ---- A: loads ---------------------------------------------------------
    const int nload = main ? G::NLOAD : G::NINT;
    if constexpr (PREF) {
      // interior item (it = tid) from the registers fetched last iteration
      if (k > z0 - NWARM) {
        convert_interior(k + 2);
      } else {
        fetch_interior(k + 2);
        convert_interior(k + 2);
      }
      for (int it = rtid + NT; it < nload; it += NT) load_item(it, k, k);
    } else {
      for (int it = rtid; it < nload; it += NT) {
        if (ZACT && it < G::NINT)
          load_item(it, k + 2, k);
        else
          load_item(it, k, k);
      }
    }
    __syncthreads();
    if constexpr (PREF) {
      if (k + 1 < z1) fetch_interior(k + 3);
    }
    if (ZACT && k < z0 - 2) continue;
    const T* cur = ring_plane(k);

    // ---- B: slopes --------------------------------------------------------
    for (int it = rtid; main && it < G::SXN + G::SYN; it += NT) {
      T sig[kNV];
      T* dst;
      int ds;
      int s0, s1, s2;
      const T *m, *c, *pp;
      if (it < G::SXN) {
        const int r = it / (TX + 2), cc = it - r * (TX + 2) - 1;
        m = cell_ptr(cur, r, cc - 1, &s0);
        c = cell_ptr(cur, r, cc, &s1);
        pp = cell_ptr(cur, r, cc + 1, &s2);
        dst = sxs + it;
        ds = G::SXN;
      } else {
        const int j = it - G::SXN;
        const int rr = j / TX - 1, cc = j - (j / TX) * TX;
        m = cell_ptr(cur, rr - 1, cc, &s0);
        c = cell_ptr(cur, rr, cc, &s1);
        pp = cell_ptr(cur, rr + 1, cc, &s2);
        dst = sys + j;
        ds = G::SYN;
      }
      cell_slopes<T, !PREF>(m, s0, c, s1, pp, s2, lim, sig);
#pragma unroll
      for (int q = 0; q < kNV; ++q) dst[q * ds] = sig[q];
    }
    if (ZACT && owner) {
      T sig[kNV];
      cell_slopes<T, !PREF>(cur + oidx, G::PS, ring_plane(k + 1) + oidx, G::PS,
                            ring_plane(k + 2) + oidx, G::PS, lim, sig);
#pragma unroll
      for (int q = 0; q < kNV; ++q) zS[q * G::NINT + oidx] = sig[q];
    }
    __syncthreads();

    // ---- C: fluxes --------------------------------------------------------
    for (int it = rtid; main && it < G::ITEMS; it += NT) {
      T vl[kNV], vr[kNV], F[kNV];
      int dir;
      T* out;
      int os;
      if (it < G::IT_X || it >= G::IT_X + G::IT_Y) {
        int r, fi;
        if (it < G::IT_X) {
          r = it / TX;
          fi = it - r * TX;
        } else {
          r = it - (G::IT_X + G::IT_Y);
          fi = TX;
        }
        int sa, sb;
        const T* a = cell_ptr(cur, r, fi - 1, &sa);
        const T* b = cell_ptr(cur, r, fi, &sb);
        const T* ga = sxs + r * (TX + 2) + fi;      // slope of cell fi-1
        const T* gb = ga + 1;                        // slope of cell fi
#pragma unroll
        for (int q = 0; q < kNV; ++q) {
          vl[q] = a[q * sa] + T(0.5) * ga[q * G::SXN];
          vr[q] = b[q * sb] - T(0.5) * gb[q * G::SXN];
        }
        if constexpr (CT) ct_face_field(vl, vr, 0, bface(0, k, r, fi));
        dir = 0;
        out = Fx + r * (TX + 1) + fi;
        os = G::FXN;
      } else {
        const int j = it - G::IT_X;
        const int fj = j / TX, c = j - (j / TX) * TX;
        int sa, sb;
        const T* a = cell_ptr(cur, fj - 1, c, &sa);
        const T* b = cell_ptr(cur, fj, c, &sb);
        const T* ga = sys + fj * TX + c;             // slope of row fj-1
        const T* gb = ga + TX;                       // slope of row fj
#pragma unroll
        for (int q = 0; q < kNV; ++q) {
          vl[q] = a[q * sa] + T(0.5) * ga[q * G::SYN];
          vr[q] = b[q * sb] - T(0.5) * gb[q * G::SYN];
        }
        if constexpr (CT) ct_face_field(vl, vr, 1, bface(1, k, fj, c));
        dir = 1;
        out = Fy + j;
        os = G::FYN;
      }
      // warp-uniform branch to the compile-time direction
      if (dir == 0)
        glm_hlld_flux<0>(vl, vr, ch, half_chi, ph, F);
      else
        glm_hlld_flux<1>(vl, vr, ch, half_chi, ph, F);
#pragma unroll
      for (int q = 0; q < kNV; ++q) out[q * os] = F[q];
    }
    T dUz[kNV];
    if constexpr (ZACT) {
      if (owner) {
        T vl[kNV], vr[kNV], F[kNV];
        const T* c = ring_plane(k + 1) + oidx;
#pragma unroll
        for (int q = 0; q < kNV; ++q) {
          vl[q] = zP[q * G::NINT + oidx];
          vr[q] = c[q * G::PS] - T(0.5) * zS[q * G::NINT + oidx];
        }
        if constexpr (CT) {
          ct_face_field(vl, vr, 2, bface(2, k + 1, orow, ocol));
          ctc.from_prims(cur + oidx, G::PS);
          ctc.fz_bx = zF[kBX * G::NINT + oidx];
          ctc.fz_by = zF[kBY * G::NINT + oidx];
          ctc.fz_rho = zF[kRHO * G::NINT + oidx];
        }
        if (k >= z0 - 1) {  // from k = z0-1 on, zP holds the face state of cell k
          glm_hlld_flux<2>(vl, vr, ch, half_chi, ph, F);
#pragma unroll
          for (int q = 0; q < kNV; ++q) {
            dUz[q] = mul_rn(F[q] - zF[q * G::NINT + oidx], dtdz);
            zF[q * G::NINT + oidx] = F[q];
          }
        }
#pragma unroll
        for (int q = 0; q < kNV; ++q)
          zP[q * G::NINT + oidx] = c[q * G::PS] + T(0.5) * zS[q * G::NINT + oidx];
      }
    }
    __syncthreads();

    // ---- D: right-hand side and RK combination (column owners) -------------
    if (main && owner) {
      const int gx = x0 + ocol, gy = y0 + orow;
      const bool valid = gx < nx && gy < ny;
      T unew[kNV];
#pragma unroll
      for (int q = 0; q < kNV; ++q) unew[q] = T(0);
      if (valid) {
        const long long off = (long long)k * p.sz + (long long)gy * p.sy + gx;
#pragma unroll
        for (int q = 0; q < kNV; ++q) {
          const T* fx = Fx + q * G::FXN + orow * (TX + 1) + ocol;
          // sums of products with their rounding fixed (mul_rn / fma_rn), so
          // every instantiation of this tile code gives the same bits
          T du = mul_rn(fx[1] - fx[0], dtdx);
          if constexpr (G::GY > 0) {
            const T* fy = Fy + q * G::FYN + orow * TX + ocol;
            du = fma_rn(fy[TX] - fy[0], dtdy, du);
          }
          if constexpr (ZACT) du += dUz[q];
          if (frozen) du = T(0);
          const T s1 = p.win[q * p.sv + off] - du;
          if constexpr (STAGE == 1) {
            unew[q] = s1;
          } else {
            unew[q] = fma_rn(p.a_n, p.un[q * p.sv + off], mul_rn(p.a_w, s1));
          }
        }
        if constexpr (CT) {
#pragma unroll
          for (int q = 0; q < kNV; ++q)
            if (q != kBX && q != kBY && q != kBZ) p.uout[q * p.sv + off] = q == kPSI ? T(0) : unew[q];
          ctc.write(p.ctf, p.sv, off, Fx + orow * (TX + 1) + ocol, G::FXN,
                    Fy + orow * TX + ocol, G::FYN, ch);
        } else {
          if constexpr (STAGE == 2) unew[kPSI] *= damp;
#pragma unroll
          for (int q = 0; q < kNV; ++q) p.uout[q * p.sv + off] = unew[q];
        }
      }
      if constexpr (STAGE == 2 && !CT) {  // every lane of the (whole) owner warps
        const int ndim = 1 + (G::GY > 0) + (ZACT ? 1 : 0);
        smax.update(unew, valid, ph, ndim, flags);
      }
    }
  }

  if constexpr (STAGE == 2 && !CT) {
    // block max of the wave speed -> one FP64-bit atomicMax per CTA
    double l = smax.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, l, o);
      l = nan_max(l, other);
    }
    __syncthreads();
    if ((tid & 31) == 0) wmax[tid >> 5] = l;
    __syncthreads();
    if (tid == 0) {
      double m = wmax[0];
      for (int w = 1; w < NW; ++w)
        m = nan_max(m, wmax[w]);
      SpeedMax<T>::publish(m, p.lam_bits, p.est_bits);
    }
  }
  __syncthreads();  // the CTA may start another tile on the same shared memory
}

template <class T, int TY, int NW, int STAGE, bool ZACT, bool CT, bool HALO = false>
__global__ void __launch_bounds__(NW * 32, 1) rk_stage_kernel(const StageParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double wmax[NW];
  const StepScalars sc = *p.sc;
  stage_tile<T, TY, NW, STAGE, ZACT, CT, HALO>(p, sc, blockIdx.x, blockIdx.y, blockIdx.z,
                                               smem_raw, wmax);
}

}  // namespace mhd
