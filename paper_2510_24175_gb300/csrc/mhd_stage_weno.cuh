// Fused Runge-Kutta stage kernel with WENO-Z reconstruction (the
// reconstruction of the paper's own runs, Section 4.2): WENO-Z weights of
// Borges, Carmona, Costa & Don (2008) with exponent 1 and the candidate
// stencils and smoothness indicators of Jiang & Shu (1996), applied to the
// primitive variables.  Same phases as the PLM kernel (mhd_stage.cuh):
//   A  load + cons->prim: interior of plane k+3 (5-plane ring) and the
//      (x, y) halo of plane k (three cells deep);
//   B  the two face values of each cell and direction, once: x for the 34
//      cells of each row, y for the TY+2 rows, z (column owners) for cell k+1;
//      a cell whose face density or pressure would be <= 0 keeps its flat
//      value;
//   C  face fluxes (GLM + HLLD), each face of the tile once; column owners also
//      the z face k+1/2;
//   D  flux divergence + Runge-Kutta combination (+ damping and the wave-speed
//      reduction in the last stage).
#pragma once

#include "mhd_stage.cuh"

namespace mhd {

// epsilon of the WENO-Z weights (FP32 uses a larger one so that tau / e_k
// below stays finite).  FP64's form below holds while |primitive| < ~1e25
// (the product of both faces' denominators, ~beta^6, stays finite).
template <class T> struct WenoEps;
template <> struct WenoEps<double> { static constexpr double v = 1e-40; };
template <> struct WenoEps<float> { static constexpr float v = 1e-18f; };

// WENO-Z values of one variable at the cell's faces i-1/2 (minus) and i+1/2
// (plus) from f[0..4] = cells i-2 .. i+2.  With the second differences
// d_k and the one-sided first-difference combinations g_k of the three
// candidate stencils, written as D_k = d_k/12 and G_k = g_k/4:
//   * every candidate value is the cell value plus D_k +- G_k (the plus face
//     takes D0+G0, D1-G1, D2-G2; the minus face, whose stencils are the
//     mirrored ones, D2+G2, D1+G1, D0-G0);
//   * the Jiang-Shu smoothness indicator is beta_k = 13/12 d_k^2 + 1/4 g_k^2
//     = 4 (39 D_k^2 + G_k^2); the weights are invariant under a common scale
//     of beta, tau and epsilon, so the code works with beta/4 and epsilon/4;
//   * the smoothness indicators are shared by both faces (the reversed
//     stencils' are the same three in reverse order), and so is tau;
//   * the normalised weights w_k = d_k (1 + tau / e_k) / sum_j (...),
//     e_k = beta_k + eps, ideal weights (1, 6, 3)/10 (plus face; reversed on
//     the minus face).
// FP64 multiplies the unnormalised weights by e0 e1 e2 (no reciprocal per
// stencil): P_k = e0 e1 e2 + tau prod_{j != k} e_j, and one reciprocal of the
// product of the two faces' denominators serves both faces.  In FP32 these
// products of epsilons underflow (a uniform variable has beta = 0), so FP32
// takes the reciprocals 1 / e_k and one per face.
template <class T>
__device__ __forceinline__ void wenoz_pair(const T f[5], T& minus, T& plus) {
  const T c12 = T(1.0 / 12.0), q4 = T(0.25), c39 = T(39);
  const T D0 = c12 * (f[0] + f[2] - T(2) * f[1]);
  const T D1 = c12 * (f[1] + f[3] - T(2) * f[2]);
  const T D2 = c12 * (f[2] + f[4] - T(2) * f[3]);
  const T G0 = q4 * (f[0] - T(4) * f[1] + T(3) * f[2]);
  const T G1 = q4 * (f[1] - f[3]);
  const T G2 = q4 * (T(3) * f[2] - T(4) * f[3] + f[4]);
  const T b0 = c39 * D0 * D0 + G0 * G0;
  const T b1 = c39 * D1 * D1 + G1 * G1;
  const T b2 = c39 * D2 * D2 + G2 * G2;
  const T eps = T(0.25) * WenoEps<T>::v;
  const T tau = tabs(b0 - b2);
  const T e0 = b0 + eps, e1 = b1 + eps, e2 = b2 + eps;
  T P0, P1, P2;
  if constexpr (sizeof(T) == 8) {
    const T E0 = e1 * e2, E2 = e0 * e1;
    const T pi = e0 * E0;
    P0 = pi + tau * E0, P1 = pi + tau * (e0 * e2), P2 = pi + tau * E2;
  } else {
    P0 = T(1) + tau * rcp(e0), P1 = T(1) + tau * rcp(e1), P2 = T(1) + tau * rcp(e2);
  }
  const T S1 = T(6) * P1, T0 = T(3) * P0, T2 = T(3) * P2;
  const T den_p = P0 + S1 + T2, den_m = P2 + S1 + T0;
  const T num_p = P0 * (D0 + G0) + S1 * (D1 - G1) + T2 * (D2 - G2);
  const T num_m = P2 * (D2 + G2) + S1 * (D1 + G1) + T0 * (D0 - G0);
  if constexpr (sizeof(T) == 8) {
    const T r = rcp(den_p * den_m);
    plus = f[2] + num_p * den_m * r;
    minus = f[2] + num_m * den_p * r;
  } else {
    plus = f[2] + num_p * rcp(den_p);
    minus = f[2] + num_m * rcp(den_m);
  }
}

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// FP32 WENO-Z of two variables at once (.x, .y), the steps of wenoz_pair<float>
// in packed FP32 with every operation written out; the reciprocals per lane.
__device__ __forceinline__ void wenoz_pair2(const float2 f[5], float2& minus, float2& plus) {
  const float2 C12 = pk1(1.0f / 12.0f), Q4 = pk1(0.25f), C39 = pk1(39.0f);
  const float2 M2 = pk1(-2.0f), M4 = pk1(-4.0f), T3 = pk1(3.0f);
  const float2 D0 = mul2(C12, fma2(M2, f[1], add2(f[0], f[2])));
  const float2 D1 = mul2(C12, fma2(M2, f[2], add2(f[1], f[3])));
  const float2 D2 = mul2(C12, fma2(M2, f[3], add2(f[2], f[4])));
  const float2 G0 = mul2(Q4, fma2(T3, f[2], fma2(M4, f[1], f[0])));
  const float2 G1 = mul2(Q4, sub2(f[1], f[3]));
  const float2 G2 = mul2(Q4, add2(fma2(M4, f[3], mul2(T3, f[2])), f[4]));
  const float2 b0 = fma2(G0, G0, mul2(mul2(C39, D0), D0));
  const float2 b1 = fma2(G1, G1, mul2(mul2(C39, D1), D1));
  const float2 b2 = fma2(G2, G2, mul2(mul2(C39, D2), D2));
  const float2 EPS = pk1(0.25f * WenoEps<float>::v);
  const float2 d02 = sub2(b0, b2);
  const float2 tau = pk(fabsf(d02.x), fabsf(d02.y));
  const float2 e0 = add2(b0, EPS), e1 = add2(b1, EPS), e2 = add2(b2, EPS);
  const float2 ONE = pk1(1.0f);
  const float2 P0 = fma2(tau, pk(rcp(e0.x), rcp(e0.y)), ONE);
  const float2 P1 = fma2(tau, pk(rcp(e1.x), rcp(e1.y)), ONE);
  const float2 P2 = fma2(tau, pk(rcp(e2.x), rcp(e2.y)), ONE);
  const float2 S1 = mul2(pk1(6.0f), P1), T0 = mul2(T3, P0), T2 = mul2(T3, P2);
  const float2 den_p = add2(add2(P0, S1), T2), den_m = add2(add2(P2, S1), T0);
  const float2 num_p = fma2(T2, sub2(D2, G2), fma2(S1, sub2(D1, G1), mul2(P0, add2(D0, G0))));
  const float2 num_m = fma2(T0, sub2(D0, G0), fma2(S1, add2(D1, G1), mul2(P2, add2(D2, G2))));
  plus = fma2(num_p, pk(rcp(den_p.x), rcp(den_p.y)), f[2]);
  minus = fma2(num_m, pk(rcp(den_m.x), rcp(den_m.y)), f[2]);
}
#endif

// Face values of all 9 primitives of one cell from five cells c[0..4]
// (variables stride[j] apart); flat fallback on non-positive face density
// or pressure.  FP32 on the device reconstructs the variables in pairs
// (0, 1) ... (6, 7) in packed instructions.
template <class T>
__device__ __forceinline__ void cell_weno(const T* const c[5], const int st[5], T M[kNV],
                                          T P[kNV]) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int k = 0; k + 1 < kNV; k += 2) {
      float2 f[5];
#pragma unroll
      for (int j = 0; j < 5; ++j) f[j] = pk(c[j][k * st[j]], c[j][(k + 1) * st[j]]);
      float2 m2, p2;
      wenoz_pair2(f, m2, p2);
      M[k] = m2.x;
      M[k + 1] = m2.y;
      P[k] = p2.x;
      P[k + 1] = p2.y;
    }
    {
      float2 f[5];
#pragma unroll
      for (int j = 0; j < 5; ++j) f[j] = pk1(c[j][(kNV - 1) * st[j]]);
      float2 m2, p2;
      wenoz_pair2(f, m2, p2);
      M[kNV - 1] = m2.x;
      P[kNV - 1] = p2.x;
    }
    const bool ok = M[kRHO] > T(0) && P[kRHO] > T(0) && M[kPRS] > T(0) && P[kPRS] > T(0);
    if (!ok) {
#pragma unroll
      for (int k = 0; k < kNV; ++k) M[k] = P[k] = c[2][k * st[2]];
    }
    return;
  }
#endif
#pragma unroll
  for (int k = 0; k < kNV; ++k) {
    T f[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) f[j] = c[j][k * st[j]];
    wenoz_pair(f, M[k], P[k]);
  }
  const bool ok = M[kRHO] > T(0) && P[kRHO] > T(0) && M[kPRS] > T(0) && P[kPRS] > T(0);
  if (!ok) {
#pragma unroll
    for (int k = 0; k < kNV; ++k) M[k] = P[k] = c[2][k * st[2]];
  }
}

template <int TY, bool ZACT>
struct WenoGeom {
  static constexpr int TX = 32;
  static constexpr int GY = TY > 1 ? 3 : 0;
  static constexpr int NINT = TY * TX;
  static constexpr int NXH = 6 * TY;               // x halo: columns -3..-1, 32..34
  static constexpr int NYH = GY ? 6 * TX : 0;      // y halo: rows -3..-1, TY..TY+2
  static constexpr int NRING = ZACT ? 5 : 1;
  static constexpr int RING_W = NRING * kNV * NINT;
  static constexpr int XH_W = kNV * NXH;
  static constexpr int YH_W = kNV * NYH;
  static constexpr int SXN = TY * (TX + 2);           // x face values, columns -1..32
  static constexpr int SYN = GY ? (TY + 2) * TX : 0;  // y face values, rows -1..TY
  static constexpr int FXN = TY * (TX + 1);
  static constexpr int FYN = GY ? (TY + 1) * TX : 0;
  static constexpr int Z_W = ZACT ? 4 * kNV * NINT : 0;  // zM, zPn, zP, zF per owner
  static constexpr int WORDS = RING_W + XH_W + YH_W + 2 * kNV * SXN + 2 * kNV * SYN +
                               kNV * FXN + kNV * FYN + Z_W;
  static constexpr int NLOAD = NINT + NXH + NYH;
  static constexpr int IT_X = TY * TX;
  static constexpr int IT_Y = FYN;
  static constexpr int IT_XE = TY;
  static constexpr int ITEMS = IT_X + IT_Y + IT_XE;
};

// CT: constrained transport, HALO: halo faces, as in stage_tile() (mhd_stage.cuh).
// 3-D FP32 with 8-warp CTAs: two CTAs per SM (128 registers at most);
// without the bound the packed reconstruction takes 132-150 registers and
// runs one CTA per SM, 25-30 % slower.  (Larger CTAs run one per SM.)
template <class T, int TY, int NW, int STAGE, bool ZACT, bool CT, bool HALO = false>
__global__ void __launch_bounds__(NW * 32, (sizeof(T) == 4 && ZACT && NW <= 8) ? 2 : 1)
    rk_stage_weno_kernel(const StageParams<T> p) {
  using G = WenoGeom<TY, ZACT>;
  constexpr int NT = NW * 32;
  constexpr int TX = G::TX;
  constexpr int ZT0 = NT - G::NINT;
  static_assert(ZT0 >= 0, "need one thread per tile column");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double wmax[NW];
  T* ring = reinterpret_cast<T*>(smem_raw);
  T* xh = ring + G::RING_W;
  T* yh = xh + G::XH_W;
  T* xM = yh + G::YH_W;
  T* xP = xM + kNV * G::SXN;
  T* yM = xP + kNV * G::SXN;
  T* yP = yM + kNV * G::SYN;
  T* Fx = yP + kNV * G::SYN;
  T* Fy = Fx + kNV * G::FXN;
  T* zM = Fy + kNV * G::FYN;   // per owner: minus-face value of cell k+1
  T* zPn = zM + kNV * G::NINT;  // per owner: plus-face value of cell k+1
  T* zP = zPn + kNV * G::NINT;  // per owner: plus-face value of cell k
  T* zF = zP + kNV * G::NINT;   // per owner: z flux at face k-1/2

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX;
  const int y0 = blockIdx.y * TY;
  const int z0 = p.zlo + blockIdx.z * p.tz;
  const int z1 = min(z0 + p.tz, p.zhi);
  const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
  const bool owner = tid >= ZT0;
  const int oidx = tid - ZT0;
  const int orow = oidx / TX, ocol = oidx - (oidx / TX) * TX;

  const StepScalars sc = *p.sc;
  const T ch = T(sc.ch);
  const T half_chi = T(0.5 / sc.ch);
  const T dtdx = T(sc.dtdx[0]), dtdy = T(sc.dtdx[1]), dtdz = T(sc.dtdx[2]);
  const T damp = T(sc.damp);
  const bool frozen = !(sc.dt != 0.0);
  const Phys<T> ph = p.ph;
  unsigned flags = 0;  // of the wave-speed conversions (not counted)

  auto slot = [](int zz) { return ZACT ? ((zz % 5) + 5) % 5 : 0; };
  auto ring_plane = [&](int zz) { return ring + slot(zz) * (kNV * G::NINT); };

  // floor activations: once per stage for each cell the tile updates, from
  // its own conversion (as in the PLM stage kernel)
  auto count_floors = [&](unsigned fl, int zz, int r, int c) {
    if (zz < z0 || zz >= z1 || x0 + c >= nx || (G::GY && y0 + r >= ny)) return;
    if (fl & kFloorRho) atomicAdd(&p.floor_cnt[0], 1ull);
    if (fl & kFloorP) atomicAdd(&p.floor_cnt[1], 1ull);
    if (fl & kPressF64) atomicAdd(&p.floor_cnt[2], 1ull);
  };
  auto load_cell = [&](int zz, int r, int c, T* dst, int dst_stride, bool own) {
    T u[kNV], v[kNV];
    if constexpr (HALO) {
      long long hs;
      const T* a = halo_cell<3>(p, x0 + c, y0 + r, zz, hs);
#pragma unroll
      for (int k = 0; k < kNV; ++k) u[k] = a[k * hs];
    } else {
      const int gz = ZACT ? remap3(zz, nz, p.bc_lo[2], p.bc_hi[2]) : 0;
      const int gx = remap3(x0 + c, nx, p.bc_lo[0], p.bc_hi[0]);
      const int gy = G::GY ? remap3(y0 + r, ny, p.bc_lo[1], p.bc_hi[1]) : 0;
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
  auto load_item = [&](int it, int zi, int zh) {
    if (it < G::NINT) {
      const int r = it / TX, c = it - (it / TX) * TX;
      load_cell(zi, r, c, ring_plane(zi) + it, G::NINT, true);
    } else if (it < G::NINT + G::NXH) {
      const int j = it - G::NINT;
      const int r = j / 6, q = j - (j / 6) * 6;
      const int c = q < 3 ? q - 3 : TX + q - 3;
      load_cell(zh, r, c, xh + j, G::NXH, false);
    } else {
      const int j = it - G::NINT - G::NXH;
      const int hr = j / TX, c = j - (j / TX) * TX;
      const int r = hr < 3 ? hr - 3 : TY + hr - 3;
      load_cell(zh, r, c, yh + j, G::NYH, false);
    }
  };
  auto cell_ptr = [&](const T* cur, int r, int c, int* st) -> const T* {
    if (c < 0 || c >= TX) {
      *st = G::NXH;
      return xh + r * 6 + (c < 0 ? c + 3 : c - TX + 3);
    }
    if (r < 0 || r >= TY) {
      *st = G::NYH;
      return yh + (r < 0 ? r + 3 : r - TY + 3) * TX + c;
    }
    *st = G::NINT;
    return cur + r * TX + c;
  };
  static_assert(!CT || ZACT, "constrained transport is 3-D only");
  static_assert(!HALO || (ZACT && !CT), "halo faces: 3-D GLM kernels only");
  // staggered normal field on the lower d-face of tile cell (r, c) of plane zz
  auto bface = [&](int d, int zz, int r, int c) -> T {
    const int gz = remap3(zz, nz, p.bc_lo[2], p.bc_hi[2]);
    const int gx = remap3(x0 + c, nx, p.bc_lo[0], p.bc_hi[0]);
    const int gy = remap3(y0 + r, ny, p.bc_lo[1], p.bc_hi[1]);
    return p.bw[d][(long long)gz * p.sz + (long long)gy * p.sy + gx];
  };
  CtCell<T> ctc;
  // face values of the owned column's cell in plane zc (planes zc-2..zc+2)
  auto z_cell = [&](int zc, T M[kNV], T P[kNV]) {
    const T* c[5];
    int st[5];
    for (int j = 0; j < 5; ++j) {
      c[j] = ring_plane(zc - 2 + j) + oidx;
      st[j] = G::NINT;
    }
    cell_weno(c, st, M, P);
  };

  // The z march: one loop body for every plane (see stage_tile in
  // mhd_stage.cuh), so a cell's result does not depend on where a z chunk,
  // block or launch range starts.  Warm-up: k = z0-6 .. z0-3 only load
  // planes z0-3 .. z0 into the ring, k = z0-2 computes the column owners'
  // face values of cell z0-1, k = z0-1 their flux through face z0-1/2; the
  // x, y work and the update start at k = z0.
  constexpr int NWARM = ZACT ? 6 : 0;
  SpeedMax<T> smax(ph);  // last stage: the new state's maximum wave speed
#pragma unroll 1
  for (int k = z0 - NWARM; k < z1; ++k) {
    const bool main = k >= z0;
    // ---- A: loads ---------------------------------------------------------
    const int nload = main ? G::NLOAD : G::NINT;
    for (int it = tid; it < nload; it += NT) {
      if (ZACT && it < G::NINT)
        load_item(it, k + 3, k);
      else
        load_item(it, k, k);
    }
    __syncthreads();
    if (ZACT && k < z0 - 2) continue;
    const T* cur = ring_plane(k);

    // ---- B: face values ---------------------------------------------------
    for (int it = tid; main && it < G::SXN + G::SYN; it += NT) {
      const T* c[5];
      int st[5];
      T M[kNV], P[kNV];
      T *dM, *dP;
      int ds;
      if (it < G::SXN) {
        const int r = it / (TX + 2), cc = it - r * (TX + 2) - 1;
        for (int j = 0; j < 5; ++j) c[j] = cell_ptr(cur, r, cc - 2 + j, &st[j]);
        dM = xM + it;
        dP = xP + it;
        ds = G::SXN;
      } else {
        const int j0 = it - G::SXN;
        const int rr = j0 / TX - 1, cc = j0 - (j0 / TX) * TX;
        for (int j = 0; j < 5; ++j) c[j] = cell_ptr(cur, rr - 2 + j, cc, &st[j]);
        dM = yM + j0;
        dP = yP + j0;
        ds = G::SYN;
      }
      cell_weno(c, st, M, P);
#pragma unroll
      for (int q = 0; q < kNV; ++q) {
        dM[q * ds] = M[q];
        dP[q * ds] = P[q];
      }
    }
    if (ZACT && owner) {
      T M[kNV], P[kNV];
      z_cell(k + 1, M, P);
#pragma unroll
      for (int q = 0; q < kNV; ++q) {
        zM[q * G::NINT + oidx] = M[q];
        zPn[q * G::NINT + oidx] = P[q];
      }
    }
    __syncthreads();

    // ---- C: fluxes --------------------------------------------------------
    for (int it = tid; main && it < G::ITEMS; it += NT) {
      T vl[kNV], vr[kNV], F[kNV];
      T* out;
      int os;
      const bool xdir = it < G::IT_X || it >= G::IT_X + G::IT_Y;
      if (xdir) {
        int r, fi;
        if (it < G::IT_X) {
          r = it / TX;
          fi = it - r * TX;
        } else {
          r = it - (G::IT_X + G::IT_Y);
          fi = TX;
        }
        const int ia = r * (TX + 2) + fi;  // cell fi-1; cell fi is ia + 1
#pragma unroll
        for (int q = 0; q < kNV; ++q) {
          vl[q] = xP[q * G::SXN + ia];
          vr[q] = xM[q * G::SXN + ia + 1];
        }
        if constexpr (CT) ct_face_field(vl, vr, 0, bface(0, k, r, fi));
        out = Fx + r * (TX + 1) + fi;
        os = G::FXN;
      } else {
        const int j = it - G::IT_X;
        const int fj = j / TX, c = j - (j / TX) * TX;
        const int ia = fj * TX + c;  // row fj-1; row fj is ia + TX
#pragma unroll
        for (int q = 0; q < kNV; ++q) {
          vl[q] = yP[q * G::SYN + ia];
          vr[q] = yM[q * G::SYN + ia + TX];
        }
        if constexpr (CT) ct_face_field(vl, vr, 1, bface(1, k, fj, c));
        out = Fy + j;
        os = G::FYN;
      }
      if (xdir)
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
#pragma unroll
        for (int q = 0; q < kNV; ++q) {
          vl[q] = zP[q * G::NINT + oidx];
          vr[q] = zM[q * G::NINT + oidx];
        }
        if constexpr (CT) {
          ct_face_field(vl, vr, 2, bface(2, k + 1, orow, ocol));
          ctc.from_prims(cur + oidx, G::NINT);
          ctc.fz_bx = zF[kBX * G::NINT + oidx];
          ctc.fz_by = zF[kBY * G::NINT + oidx];
          ctc.fz_rho = zF[kRHO * G::NINT + oidx];
        }
        if (k >= z0 - 1) {  // from k = z0-1 on, zP holds the plus value of cell k
          glm_hlld_flux<2>(vl, vr, ch, half_chi, ph, F);
#pragma unroll
          for (int q = 0; q < kNV; ++q) {
            dUz[q] = mul_rn(F[q] - zF[q * G::NINT + oidx], dtdz);
            zF[q * G::NINT + oidx] = F[q];
          }
        }
#pragma unroll
        for (int q = 0; q < kNV; ++q) zP[q * G::NINT + oidx] = zPn[q * G::NINT + oidx];
      }
    }
    __syncthreads();

    // ---- D: right-hand side and Runge-Kutta combination --------------------
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
    double l = smax.value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l = nan_max(l, __shfl_xor_sync(0xffffffffu, l, o));
    __syncthreads();
    if ((tid & 31) == 0) wmax[tid >> 5] = l;
    __syncthreads();
    if (tid == 0) {
      double m = wmax[0];
      for (int w = 1; w < NW; ++w) m = nan_max(m, wmax[w]);
      SpeedMax<T>::publish(m, p.lam_bits, p.est_bits);
    }
  }
}

}  // namespace mhd
