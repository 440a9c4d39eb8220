// Device-side pointwise physics of the GLM-MHD hot path, templated on the
// arithmetic type T (double for MHD_FP64, float for MHD_FP32).
//
// The stage structure is Section 3.2's (boundary calculation, cons->prim,
// reconstruction, Riemann solver, right-hand side); HLLD is named in
// Section 4.2 and divergence cleaning (GLM) in Section 4.2's strong-scaling
// paragraph.  The formulas are the published methods:
//   - HLLD: Miyoshi & Kusano (2005), J. Comput. Phys. 208: wave speeds
//     (Eq. 67), S_M and p_t* (Eqs. 38, 41), single-star states (Eqs. 43-48),
//     Alfven speeds S*_{L,R} (Eq. 51), double-star states (Eqs. 59-63),
//     fan-region fluxes (Eqs. 64-66).
//   - GLM interface values: Dedner et al. (2002), J. Comput. Phys. 175,
//     Eq. 41 (exact solution of the 2x2 (B_n, psi) Riemann problem).
//   - PLM slopes: minmod / monotonised-central limiters of van Leer (1977),
//     applied to primitive variables, with a zero-slope fallback for a cell
//     whose face density or pressure would be non-positive.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#define MHD_HD __host__ __device__ __forceinline__

namespace mhd {

enum { kRHO = 0, kVX = 1, kVY = 2, kVZ = 3, kBX = 4, kBY = 5, kBZ = 6, kPRS = 7, kPSI = 8,
       kNV = 9 };
enum { kLimFlat = 0, kLimMinmod = 1, kLimMC = 2, kLimWenoz = 3 };
// kBcHalo: the ghost cells of that side come from a caller-supplied halo buffer
// (a subdomain boundary of a decomposed grid)
enum { kBcPeriodic = 0, kBcOutflow = 1, kBcHalo = 2 };
// cons->prim flags: density floor, pressure floor, and (FP32 only) the
// pressure recomputed in FP64 because the FP32 value fell in the
// cancellation-dominated range
enum { kFloorRho = 1u, kFloorP = 2u, kPressF64 = 4u };

template <class T>
struct Phys {
  T gamma;      // adiabatic index
  T gm1;        // gamma - 1
  T gm1i;       // 1 / (gamma - 1)
  T rho_floor;
  T p_floor;
  double gamma_d, rho_floor_d, p_floor_d;  // FP64 copies for the floor branch
};

// Correctly rounded reciprocal (the host build, used only by host-side unit
// harnesses, divides).
MHD_HD double rcp(double x) {
#ifdef __CUDA_ARCH__
  return __drcp_rn(x);
#else
  return 1.0 / x;
#endif
}
// FP32 mode: hardware-approximate reciprocal and square root (a few ulp;
// the FP32 bulk path's error budget is ~1e-5 relative).
MHD_HD float rcp(float x) {
#ifdef __CUDA_ARCH__
  return __fdividef(1.0f, x);
#else
  return 1.0f / x;
#endif
}
// A product and a fused multiply-add whose rounding the source fixes.  In a
// sum of two products the compiler may fuse either product into the add, and
// copies of the same code inlined at different sites (or kernels that differ
// only elsewhere) may then round differently; the sums whose results must
// not depend on where the code runs are written with these (the same number
// of instructions as the contracted form).
MHD_HD double mul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
MHD_HD float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
MHD_HD double fma_rn(double a, double b, double c) { return fma(a, b, c); }
MHD_HD float fma_rn(float a, float b, float c) { return fmaf(a, b, c); }
// a0 b0 + a1 b1 + a2 b2, rounded as fma(a2, b2, fma(a1, b1, a0 b0))
template <class T>
MHD_HD T dot3_rn(T a0, T b0, T a1, T b1, T a2, T b2) {
  return fma_rn(a2, b2, fma_rn(a1, b1, mul_rn(a0, b0)));
}

MHD_HD double trsqrt(double x) { return rsqrt(x); }
MHD_HD float trsqrt(float x) { return rsqrtf(x); }
MHD_HD double tsqrt(double x) { return sqrt(x); }
MHD_HD float tsqrt(float x) {
#ifdef __CUDA_ARCH__
  return x > 0.0f ? x * rsqrtf(x) : 0.0f;
#else
  return sqrtf(x);
#endif
}
MHD_HD double tabs(double x) { return fabs(x); }
MHD_HD float tabs(float x) { return fabsf(x); }
MHD_HD double tmin(double a, double b) { return fmin(a, b); }
MHD_HD float tmin(float a, float b) { return fminf(a, b); }
MHD_HD double tmax(double a, double b) { return fmax(a, b); }
MHD_HD float tmax(float a, float b) { return fmaxf(a, b); }

// Bit-pattern helpers (the host build, used only by host-side harnesses,
// goes through memcpy).
MHD_HD long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long b;
  memcpy(&b, &x, sizeof(b));
  return b;
#endif
}
MHD_HD double bits2d(long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(b);
#else
  double x;
  memcpy(&x, &b, sizeof(x));
  return x;
#endif
}

// max that keeps a NaN once either operand has one (fmax drops NaNs).  Its
// operands are wave speeds or magnitudes: +0, positive, +inf or NaN.  For
// those, the unsigned order of the FP64 bit patterns is the numeric order
// with every NaN above +inf, so the device takes the FP64 max on the
// integer pipe (the FP64 pipe is the bound of the FP64 kernels).
MHD_HD double nan_max(double a, double b) {
#ifdef __CUDA_ARCH__
  const unsigned long long x = (unsigned long long)dbits(a), y = (unsigned long long)dbits(b);
  return bits2d((long long)(x > y ? x : y));
#else
  return (a != a || b > a || b != b) ? (a != a ? a : b) : a;
#endif
}
MHD_HD float nan_max(float a, float b) { return (a != a || b > a || b != b) ? (a != a ? a : b) : a; }
MHD_HD bool is_nan(double x) {
  return ((unsigned long long)dbits(x) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
}
MHD_HD bool is_nan(float x) { return x != x; }

// Sign tests and min / max with IEEE results (-0, subnormals, infinities and
// NaN included: a NaN compares false, and tmin2 / tmax2 return the other
// operand like fmin / fmax).  FP64 takes them on the integer pipe from the
// bit patterns: x > 0 exactly when the pattern lies in [1, +inf], x < 0 when
// it lies in [-0 + 1 ulp, -inf] (sign-magnitude order), and two doubles order
// like their patterns once the magnitude bits of negative ones are flipped.
MHD_HD bool gt0(double x) {
  return (unsigned long long)dbits(x) - 1ull < 0x7ff0000000000000ull;
}
MHD_HD bool lt0(double x) {
  return (unsigned long long)dbits(x) - 0x8000000000000001ull < 0x7ff0000000000000ull;
}
MHD_HD bool ge0(double x) {
  const unsigned long long b = (unsigned long long)dbits(x);
  return b <= 0x7ff0000000000000ull || b == 0x8000000000000000ull;
}
MHD_HD bool gt0(float x) { return x > 0.0f; }
MHD_HD bool lt0(float x) { return x < 0.0f; }
MHD_HD bool ge0(float x) { return x >= 0.0f; }
MHD_HD long long order_key(long long b) { return b ^ ((b >> 63) & 0x7fffffffffffffffll); }
MHD_HD double tmin2(double a, double b) {
  const long long x = dbits(a), y = dbits(b);
  const bool pick_a = is_nan(b) || (!is_nan(a) && order_key(x) <= order_key(y));
  return pick_a ? a : b;
}
MHD_HD double tmax2(double a, double b) {
  const long long x = dbits(a), y = dbits(b);
  const bool pick_a = is_nan(b) || (!is_nan(a) && order_key(x) >= order_key(y));
  return pick_a ? a : b;
}
MHD_HD float tmin2(float a, float b) { return fminf(a, b); }
MHD_HD float tmax2(float a, float b) { return fmaxf(a, b); }
// a < b with IEEE semantics (NaN unordered, -0 == +0): a double's pattern,
// with negative ones mapped to minus their magnitude, is a signed integer in
// the numeric order.
MHD_HD long long num_key(long long b) { return b < 0 ? -(b & 0x7fffffffffffffffll) : b; }
MHD_HD bool lt_ieee(double a, double b) {
  return !is_nan(a) && !is_nan(b) && num_key(dbits(a)) < num_key(dbits(b));
}
MHD_HD bool lt_ieee(float a, float b) { return a < b; }
// x != 0 (true for NaN, as the IEEE comparison)
MHD_HD bool nonzero(double x) { return (dbits(x) << 1) != 0; }
MHD_HD bool nonzero(float x) { return x != 0.0f; }
// |a| < t, IEEE (false when either is NaN)
MHD_HD bool abs_lt(double a, double t) {
  const long long x = dbits(a) & 0x7fffffffffffffffll, y = dbits(t);
  return x < y && y <= 0x7ff0000000000000ll;
}
MHD_HD bool abs_lt(float a, float t) { return fabsf(a) < t; }
// max(x, 0) for the square-root discriminant (fmax(NaN, 0) = 0 as well)
MHD_HD double pos_part(double x) { return gt0(x) ? x : 0.0; }
MHD_HD float pos_part(float x) { return fmaxf(x, 0.0f); }

// Exact 2x and x/2 of a non-negative double (or +inf / NaN, which are kept)
// from its bit pattern: a power-of-two scaling moves the exponent field; a
// subnormal doubles by a shift, and halving into the subnormal range
// shifts the significand right with the dropped bit rounded to nearest even
// (the IEEE results of x + x and 0.5 * x, overflow to +inf included).
MHD_HD long long twice_bits(long long b) {
  const long long e = b >> 52;
  if (e == 0) return b << 1;
  if (e < 2046) return b + (1ll << 52);
  return e == 2047 ? b : 0x7ff0000000000000ll;
}
MHD_HD long long half_bits(long long b) {
  const long long e = b >> 52;
  if (e >= 2) return e == 2047 ? b : b - (1ll << 52);
  return (b >> 1) + ((b & 1) & ((b >> 1) & 1));
}

// Pressure floor.  FP64: plain comparison.  FP32: when the FP32 pressure is
// within the cancellation-dominated range (internal energy below 1e-3 of the
// total, or below the floor) p is recomputed in FP64 from the promoted
// conservative inputs and the floor decision is taken in FP64.
MHD_HD double pressure_floor(double p, const double u[kNV], double rho,
                                                 const Phys<double>& ph, unsigned& flags) {
  if (lt_ieee(p, ph.p_floor)) {
    flags |= kFloorP;
    return ph.p_floor;
  }
  return p;
}
MHD_HD float pressure_floor(float p, const float u[kNV], float rho,
                                                const Phys<float>& ph, unsigned& flags) {
  if (p < ph.p_floor || p < 1e-3f * ph.gm1 * u[kPRS]) {
    flags |= kPressF64;
    double r = rho;
    double m2 = (double)u[kVX] * u[kVX] + (double)u[kVY] * u[kVY] + (double)u[kVZ] * u[kVZ];
    double b2 = (double)u[kBX] * u[kBX] + (double)u[kBY] * u[kBY] + (double)u[kBZ] * u[kBZ];
    double pd = (ph.gamma_d - 1.0) * ((double)u[kPRS] - 0.5 * m2 / r - 0.5 * b2);
    if (pd < ph.p_floor_d) {
      flags |= kFloorP;
      return ph.p_floor;
    }
    return (float)pd;
  }
  return p;
}

// Conservative -> primitive (step 2 of the stage).  Floors by replacement,
// density first, then pressure; activations are flagged.
template <class T>
MHD_HD void cons_to_prim(const T u[kNV], T v[kNV], const Phys<T>& ph,
                                             unsigned& flags) {
  T rho = u[kRHO];
  if (lt_ieee(rho, ph.rho_floor)) {
    rho = ph.rho_floor;
    flags |= kFloorRho;
  }
  const T ri = rcp(rho);
  const T vx = u[kVX] * ri, vy = u[kVY] * ri, vz = u[kVZ] * ri;
  const T kin = T(0.5) * dot3_rn(u[kVX], vx, u[kVY], vy, u[kVZ], vz);
  const T b2 = dot3_rn(u[kBX], u[kBX], u[kBY], u[kBY], u[kBZ], u[kBZ]);
  T p = ph.gm1 * (u[kPRS] - kin - T(0.5) * b2);
  p = pressure_floor(p, u, rho, ph, flags);
  v[kRHO] = rho;
  v[kVX] = vx;
  v[kVY] = vy;
  v[kVZ] = vz;
  v[kBX] = u[kBX];
  v[kBY] = u[kBY];
  v[kBZ] = u[kBZ];
  v[kPRS] = p;
  v[kPSI] = u[kPSI];
}

// Primitive -> conservative.
template <class T>
MHD_HD void prim_to_cons(const T v[kNV], T u[kNV], const Phys<T>& ph) {
  const T rho = v[kRHO];
  const T v2 = v[kVX] * v[kVX] + v[kVY] * v[kVY] + v[kVZ] * v[kVZ];
  const T b2 = v[kBX] * v[kBX] + v[kBY] * v[kBY] + v[kBZ] * v[kBZ];
  u[kRHO] = rho;
  u[kVX] = rho * v[kVX];
  u[kVY] = rho * v[kVY];
  u[kVZ] = rho * v[kVZ];
  u[kBX] = v[kBX];
  u[kBY] = v[kBY];
  u[kBZ] = v[kBZ];
  u[kPRS] = v[kPRS] * ph.gm1i + T(0.5) * rho * v2 + T(0.5) * b2;
  u[kPSI] = v[kPSI];
}

// -4x and x/2 with IEEE results; FP64 moves the exponent field on the
// integer pipe (twice_bits / half_bits, exact including subnormals and
// overflow).
MHD_HD double neg4(double x) {
  const long long b = dbits(x), sign = b & (long long)0x8000000000000000ull;
  return bits2d(twice_bits(twice_bits(b ^ sign)) | (sign ^ (long long)0x8000000000000000ull));
}
MHD_HD float neg4(float x) { return -4.0f * x; }
MHD_HD double half_of(double x) {
  const long long b = dbits(x), sign = b & (long long)0x8000000000000000ull;
  return bits2d(half_bits(b ^ sign) | sign);
}
MHD_HD float half_of(float x) { return 0.5f * x; }

// x * s for a sign factor s = +1 / -1 given by its sign bit (0, or the top
// bit of a 64-bit pattern): FP64 flips the sign bit of x on the integer pipe
// (the product by +-1 is exact, so the result is the same, NaN payloads
// aside); FP32 negates.
MHD_HD long long sign_bit_of(bool negative) {
  return negative ? (long long)0x8000000000000000ull : 0ll;
}
MHD_HD double sign_mul(double x, long long sbit) { return bits2d(dbits(x) ^ sbit); }
MHD_HD float sign_mul(float x, long long sbit) { return sbit ? -x : x; }

// Fast magnetosonic speed squared from 1/rho, gamma p, |B|^2 and B_n^2:
// with g = gamma p / rho, a = g + |B|^2 / rho and c_an^2 = B_n^2 / rho,
// c_f^2 = (a + sqrt(a^2 - 4 g c_an^2)) / 2.
template <class T>
MHD_HD T fast_speed2(T rho_i, T gp, T b2, T bn2) {
  const T g = mul_rn(gp, rho_i);
  const T a = fma_rn(b2, rho_i, g);
  const T disc = pos_part(fma_rn(a, a, neg4(g * (bn2 * rho_i))));
  return half_of(a + tsqrt(disc));
}

// Fast magnetosonic speed (see fast_speed2).
template <class T>
MHD_HD T fast_speed(T rho_i, T gp, T b2, T bn2) {
  return tsqrt(fast_speed2(rho_i, gp, b2, bn2));
}

// max over active directions of |v_d| + c_f,d for one conservative cell.
template <class T>
MHD_HD T cell_max_speed(const T u[kNV], const Phys<T>& ph, int ndim,
                                            unsigned& flags) {
  T v[kNV];
  cons_to_prim(u, v, ph, flags);
  const T ri = rcp(v[kRHO]);
  const T gp = ph.gamma * v[kPRS];
  const T b2 = dot3_rn(v[kBX], v[kBX], v[kBY], v[kBY], v[kBZ], v[kBZ]);
  T lam = tabs(v[kVX]) + fast_speed(ri, gp, b2, v[kBX] * v[kBX]);
  if (ndim > 1) lam = nan_max(lam, tabs(v[kVY]) + fast_speed(ri, gp, b2, v[kBY] * v[kBY]));
  if (ndim > 2) lam = nan_max(lam, tabs(v[kVZ]) + fast_speed(ri, gp, b2, v[kBZ] * v[kBZ]));
  // NaN anywhere in the cell (psi included) makes the speed NaN
  if (is_nan(v[kPSI]) || is_nan(lam)) lam = T(NAN);
  return lam;
}

#ifdef __CUDACC__
// ---------------------------------------------------------------------------
// Maximum wave speed of a state (cell_max_speed over all cells): the
// last-stage epilogue and the wave-speed kernels.  FP32 evaluates every cell.
// FP64 works in two passes.  Pass 1 (the epilogue, or a kernel over a state)
// takes an FP32 estimate of each cell's speed from FP32 images of its
// conservative variables (integer-pipe truncation, error < 2^-23 each)
// computed on the FP32 pipe, and the maximum M of the reliable estimates goes
// to one word (FP32 bits, atomicMax).  Reliable means: every input is 0 or
// within 2^-100 <= |x| < 2^100, rho and p are at least twice their floors (no
// floor acts), the internal energy is at least 1/50 of E and each
// direction's discriminant a^2 - 4 g c_an^2 at least 1e-4 a^2 (bounded
// cancellation: the FP32 errors of E - kin - |B|^2/2 and of the discriminant,
// a few 2^-24 of E and of a^2, are amplified at most 50-fold and, through the
// square root, to at most ~3e-5 of c_f^2); the estimate's relative error is
// then below 1e-4 (largest seen on 8 M random states pushed to the guard
// edges: 3.3e-6).  Pass 2
// (speed_exact_kernel) evaluates the FP64 speed of every cell whose estimate
// reaches 0.999 M or is not reliable.  The cell holding the exact maximum
// Lambda has an estimate >= Lambda (1 - 1e-4) when reliable, and
// M <= Lambda (1 + 1e-4), so it is always evaluated: the result is the exact
// FP64 maximum (floors and NaNs included, which are never screened out).
// Pass 2's FP64 evaluation sits behind a warp-uniform branch, so warps
// without a candidate issue no FP64 work for it.

// FP32 image of a double on the integer pipe: sign, rebiased exponent, top 23
// mantissa bits.  Clears ok unless x is 0 or 2^-100 <= |x| < 2^100.
__device__ __forceinline__ float f32_image(double x, bool& ok) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned mag = hi & 0x7fffffffu;
  const bool zero = (mag | lo) == 0u;
  ok = ok && (zero || ((mag >> 20) - 923u) < 200u);
  const unsigned fb = (hi & 0x80000000u) | (((mag - (896u << 20)) << 3) | (lo >> 29));
  return zero ? 0.0f : __uint_as_float(fb);
}

// FP32 estimate of cell_max_speed for an FP64 conservative cell (see above).
struct SpeedEstimator {
  float gm1, gamma, rho2, p2;  // FP32 images of the physics constants
  __device__ explicit SpeedEstimator(const Phys<double>& ph) {
    bool ok = true;
    gm1 = f32_image(ph.gm1, ok);
    gamma = f32_image(ph.gamma, ok);
    rho2 = 2.0f * f32_image(ph.rho_floor, ok);
    p2 = 2.0f * f32_image(ph.p_floor, ok);
    if (!ok) rho2 = __int_as_float(0x7f800000);  // never reliable
  }
  __device__ __forceinline__ float operator()(const double u[kNV], int ndim, bool& ok) const {
    float f[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) f[k] = f32_image(u[k], ok);
    const float r = f[kRHO];
    ok = ok && r >= rho2;
    const float ri = __frcp_rn(r);
    const float v[3] = {f[kVX] * ri, f[kVY] * ri, f[kVZ] * ri};
    const float kin = 0.5f * (f[kVX] * v[0] + f[kVY] * v[1] + f[kVZ] * v[2]);
    const float b2 = f[kBX] * f[kBX] + f[kBY] * f[kBY] + f[kBZ] * f[kBZ];
    const float eint = f[kPRS] - kin - 0.5f * b2;
    ok = ok && eint >= 0.02f * f[kPRS];
    const float pr = gm1 * eint;
    ok = ok && pr >= p2;
    const float g = gamma * pr * ri;
    const float a = b2 * ri + g;
    float lam = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d < ndim) {
        const float bd = f[kBX + d];
        const float disc = a * a - 4.0f * g * (bd * bd * ri);
        ok = ok && disc >= 1e-4f * a * a;
        lam = fmaxf(lam, fabsf(v[d]) + sqrtf(0.5f * (a + sqrtf(fmaxf(disc, 0.0f)))));
      }
    }
    return lam;
  }
};

// Per-thread accumulator of the epilogue and the wave-speed kernels: the
// exact FP32 maximum, or (FP64) the maximum of the reliable estimates.
template <class T>
struct SpeedMax;

template <>
struct SpeedMax<float> {
  float lam = 0.0f;
  __device__ explicit SpeedMax(const Phys<float>&) {}
  __device__ __forceinline__ void update(const float u[kNV], bool valid, const Phys<float>& ph,
                                         int ndim, unsigned& flags) {
    if (valid) lam = nan_max(lam, cell_max_speed(u, ph, ndim, flags));
  }
  __device__ __forceinline__ double value() const { return (double)lam; }
  // one thread per CTA: the CTA's maximum m into the state's wave-speed word
  __device__ __forceinline__ static void publish(double m, unsigned long long* lam_bits,
                                                 unsigned int*) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(m);
    if (is_nan(m)) bits = 0x7ff8000000000000ull;
    atomicMax(lam_bits, bits);
  }
};

template <>
struct SpeedMax<double> {
  float est = 0.0f;
  SpeedEstimator estimate;
  __device__ explicit SpeedMax(const Phys<double>& ph) : estimate(ph) {}
  __device__ __forceinline__ void update(const double u[kNV], bool valid, const Phys<double>&,
                                         int ndim, unsigned&) {
    bool ok = true;
    const float e = estimate(u, ndim, ok);
    if (valid && ok) est = fmaxf(est, e);
  }
  __device__ __forceinline__ double value() const { return (double)est; }
  // the CTA's maximum estimate (a non-negative FP32 value) into the estimate
  // word: non-negative floats order like their bit patterns
  __device__ __forceinline__ static void publish(double m, unsigned long long*,
                                                 unsigned int* est_bits) {
    atomicMax(est_bits, __float_as_uint((float)m));
  }
};
#endif

// Limited slope (van Leer 1977): 0 when the one-sided differences disagree in
// sign; minmod = smaller magnitude; MC = min(2|dm|, 2|dp|, |dm+dp|/2).
template <class T>
MHD_HD T limited_slope(T dm, T dp, int lim) {
  if (lim == kLimFlat || !(dm * dp > T(0))) return T(0);
  const T am = tabs(dm), ap = tabs(dp);
  T mag = tmin(am, ap);
  if (lim == kLimMC) mag = tmin(T(2) * mag, T(0.5) * tabs(dm + dp));
  return dm > T(0) ? mag : -mag;
}

// FP64 specialisation with the same result: the sign and zero tests, |.|,
// the magnitude comparisons (non-negative doubles order like their bit
// patterns), the doubling and halving of the MC limiter and the sign
// transfer run on the integer pipe; only |dm| + |dp| uses the (scarce) FP64
// pipe.  For equal signs |dm + dp| = |dm| + |dp| exactly, so the central
// slope is (|dm|+|dp|)/2.
template <>
MHD_HD double limited_slope<double>(double dm, double dp, int lim) {
  const long long a = dbits(dm), b = dbits(dp);
  const long long mask = 0x7fffffffffffffffll;
  const long long am = a & mask, bm = b & mask;
  if (lim == kLimFlat || (a ^ b) < 0 || am == 0 || bm == 0) return 0.0;
  long long mb = am < bm ? am : bm;
  if (lim == kLimMC) {
    const long long two = twice_bits(mb);
    const long long cen = half_bits(dbits(bits2d(am) + bits2d(bm)));
    mb = cen < two ? cen : two;
  }
  return bits2d(mb | (a & ~mask));
}

// PLM face states around one interface from four consecutive cells q0..q3
// (the interface lies between q1 and q2).  c[j] points at variable 0 of cell
// j; variables are vstride apart.  Writes the left state (from q1) and the
// right state (from q2).
template <class T>
MHD_HD void plm_face_pair(const T* c0, const T* c1, const T* c2,
                                              const T* c3, int vstride, int lim, T vl[kNV],
                                              T vr[kNV]) {
  T s1[kNV], s2[kNV];
#pragma unroll
  for (int k = 0; k < kNV; ++k) {
    const T q0 = c0[k * vstride], q1 = c1[k * vstride], q2 = c2[k * vstride],
            q3 = c3[k * vstride];
    s1[k] = limited_slope(q1 - q0, q2 - q1, lim);
    s2[k] = limited_slope(q2 - q1, q3 - q2, lim);
    vl[k] = q1;
    vr[k] = q2;
  }
  // zero-slope fallback per cell if a face density or pressure is <= 0
  const bool ok1 = gt0(vl[kRHO] - T(0.5) * tabs(s1[kRHO])) &&
                   gt0(vl[kPRS] - T(0.5) * tabs(s1[kPRS]));
  const bool ok2 = gt0(vr[kRHO] - T(0.5) * tabs(s2[kRHO])) &&
                   gt0(vr[kPRS] - T(0.5) * tabs(s2[kPRS]));
#pragma unroll
  for (int k = 0; k < kNV; ++k) {
    if (ok1) vl[k] = vl[k] + T(0.5) * s1[k];
    if (ok2) vr[k] = vr[k] - T(0.5) * s2[k];
  }
}

// Picks component (dir + j) % 3 of a 3-vector given as scalars (dir is a
// compile-time constant in the flux kernels, so this folds away).
template <class T>
MHD_HD T rot3(int dir, int j, T a, T b, T c) {
  const int m = (dir + j) % 3;
  return m == 0 ? a : (m == 1 ? b : c);
}

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// Packed FP32 (FFMA2 / FMUL2 / FADD2: two lanes per instruction, each lane
// rounded as the scalar instruction).  x - y is fma(y, -1, x): the product is
// exact, so it rounds once, as a subtraction does.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pk1(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }

// FP32 GLM + HLLD (the same steps as glm_hlld_flux) with the two sides'
// identical operations -- outer states, fast speeds, single-star states --
// and the two tangential components' ones -- double-star states, flux
// terms -- paired in packed instructions: .x the left state (or the first
// tangential component), .y the right one (or the second).  Every operation
// is written out (no contraction is left to the compiler), so the flux rounds
// the same in every kernel it is inlined into.
template <int dir>
__device__ __forceinline__ void glm_hlld_flux_f32x2(const float vl[kNV], const float vr[kNV],
                                                    float ch, float half_chi,
                                                    const Phys<float>& ph, float F[kNV]) {
  const float2 H = pk1(0.5f);
  const float2 u = pk(rot3(dir, 0, vl[kVX], vl[kVY], vl[kVZ]), rot3(dir, 0, vr[kVX], vr[kVY], vr[kVZ]));
  const float2 v = pk(rot3(dir, 1, vl[kVX], vl[kVY], vl[kVZ]), rot3(dir, 1, vr[kVX], vr[kVY], vr[kVZ]));
  const float2 w = pk(rot3(dir, 2, vl[kVX], vl[kVY], vl[kVZ]), rot3(dir, 2, vr[kVX], vr[kVY], vr[kVZ]));
  const float2 by = pk(rot3(dir, 1, vl[kBX], vl[kBY], vl[kBZ]), rot3(dir, 1, vr[kBX], vr[kBY], vr[kBZ]));
  const float2 bz = pk(rot3(dir, 2, vl[kBX], vl[kBY], vl[kBZ]), rot3(dir, 2, vr[kBX], vr[kBY], vr[kBZ]));
  const float bnL = rot3(dir, 0, vl[kBX], vl[kBY], vl[kBZ]);
  const float bnR = rot3(dir, 0, vr[kBX], vr[kBY], vr[kBZ]);
  const float2 r = pk(vl[kRHO], vr[kRHO]), p = pk(vl[kPRS], vr[kPRS]);

  // GLM: exact solution of the linear (B_n, psi) interface problem
  const float bx = fmaf(0.5f, __fadd_rn(bnL, bnR), -__fmul_rn(half_chi, __fsub_rn(vr[kPSI], vl[kPSI])));
  const float psis = fmaf(0.5f, __fadd_rn(vl[kPSI], vr[kPSI]),
                          -__fmul_rn(__fmul_rn(0.5f, ch), __fsub_rn(bnR, bnL)));
  const float bx2 = __fmul_rn(bx, bx);
  const float2 BX = pk1(bx), BX2 = pk1(bx2);

  // outer states
  const float2 b2 = fma2(bz, bz, fma2(by, by, BX2));
  const float2 pt = fma2(H, b2, p);
  const float2 vv = fma2(w, w, fma2(v, v, mul2(u, u)));
  const float2 e = fma2(H, b2, fma2(mul2(H, r), vv, mul2(p, pk1(ph.gm1i))));
  // 1/rho of both sides from one reciprocal; fast speeds squared
  const float qr = rcp(__fmul_rn(r.x, r.y));
  const float2 ri = mul2(swap2(r), pk1(qr));
  const float2 gp = mul2(pk1(ph.gamma), p);
  const float2 g = mul2(gp, ri);
  const float2 a = fma2(b2, ri, g);
  const float2 disc2 = fma2(a, a, mul2(pk1(-4.0f), mul2(g, mul2(BX2, ri))));
  const float dL = fmaxf(disc2.x, 0.0f), dR = fmaxf(disc2.y, 0.0f);
  const float2 dsc = pk(dL, dR);
  const float2 rq = pk(dL > 0.0f ? rsqrtf(dL) : 0.0f, dR > 0.0f ? rsqrtf(dR) : 0.0f);
  const float2 cf2 = mul2(H, fma2(dsc, rq, a));
  // wave-speed estimates, contact speed and total pressure
  const float c2m = fmaxf(cf2.x, cf2.y);
  const float cmax = c2m > 0.0f ? __fmul_rn(c2m, rsqrtf(c2m)) : 0.0f;
  const float2 S = add2(pk(fminf(u.x, u.y), fmaxf(u.x, u.y)), pk(-cmax, cmax));
  const float2 Su = sub2(S, u);
  const float2 d = mul2(Su, r);
  const float Di = rcp(__fsub_rn(d.y, d.x));
  const float SM =
      __fmul_rn(__fadd_rn(__fsub_rn(fmaf(d.y, u.y, -__fmul_rn(d.x, u.x)), pt.y), pt.x), Di);
  const float pts = __fmul_rn(fmaf(__fmul_rn(d.x, d.y), __fsub_rn(u.y, u.x),
                                   fmaf(d.y, pt.x, -__fmul_rn(d.x, pt.y))), Di);
  const float2 SMv = pk1(SM);

  // single-star states, degenerate when |rho (S-u)(S-S_M) - Bx^2| < 1e-8 p_t*;
  // paired reciprocals of S-S_M and of the two denominators
  const float2 sm = sub2(S, SMv);
  const float2 den = fma2(d, sm, pk1(-bx2));
  const float thr = __fmul_rn(1e-8f, pts);
  const bool degL = fabsf(den.x) < thr, degR = fabsf(den.y) < thr;
  const float2 dn = pk(degL ? 1.0f : den.x, degR ? 1.0f : den.y);
  const float ps = __fmul_rn(sm.x, sm.y), pd = __fmul_rn(dn.x, dn.y);
  const float q4 = rcp(__fmul_rn(ps, pd));
  const float qs = __fmul_rn(pd, q4), qd = __fmul_rn(ps, q4);
  const float2 smi = mul2(swap2(sm), pk1(qs));
  const float2 deni = mul2(swap2(dn), pk1(qd));
  const float2 rs = mul2(d, smi);
  const float2 fv = mul2(mul2(BX, sub2(SMv, u)), deni);
  const float2 fb = mul2(fma2(d, Su, pk1(-bx2)), deni);
  const float2 vs0 = fma2(pk(-by.x, -by.y), fv, v), ws0 = fma2(pk(-bz.x, -bz.y), fv, w);
  const float2 bys0 = mul2(by, fb), bzs0 = mul2(bz, fb);
  const float2 vs = pk(degL ? v.x : vs0.x, degR ? v.y : vs0.y);
  const float2 ws = pk(degL ? w.x : ws0.x, degR ? w.y : ws0.y);
  const float2 bys = pk(degL ? by.x : bys0.x, degR ? by.y : bys0.y);
  const float2 bzs = pk(degL ? bz.x : bzs0.x, degR ? bz.y : bzs0.y);
  const float2 vb = fma2(w, bz, fma2(v, by, mul2(u, BX)));
  const float2 vbs = fma2(ws, bzs, fma2(vs, bys, mul2(SMv, BX)));
  const float2 es = mul2(fma2(BX, sub2(vb, vbs),
                              fma2(pk1(pts), SMv, fma2(Su, e, pk(-__fmul_rn(pt.x, u.x),
                                                                 -__fmul_rn(pt.y, u.y))))),
                         smi);

  // fan region: side a = L if (S_L > 0) or (S_R >= 0 and S_M >= 0), else R
  const bool sup = S.x > 0.0f || S.y < 0.0f;
  const bool useL = S.x > 0.0f || (!(S.y < 0.0f) && SM >= 0.0f);
  const float ra = useL ? r.x : r.y, ua = useL ? u.x : u.y;
  const float2 vw = useL ? pk(v.x, w.x) : pk(v.y, w.y);
  const float2 bb = useL ? pk(by.x, bz.x) : pk(by.y, bz.y);
  const float ea = useL ? e.x : e.y, pta = useL ? pt.x : pt.y;
  const float rsa = useL ? rs.x : rs.y, esa = useL ? es.x : es.y;
  const float2 vws = useL ? pk(vs.x, ws.x) : pk(vs.y, ws.y);
  const float2 bbs = useL ? pk(bys.x, bzs.x) : pk(bys.y, bzs.y);
  const float vbsa = useL ? vbs.x : vbs.y, vba = useL ? vb.x : vb.y;
  const float c1 = sup ? 0.0f : (useL ? S.x : S.y);
  const float2 C1 = pk1(c1), UA = pk1(ua);
  // flux of the outer state plus the single-star jump
  const float ru = __fmul_rn(ra, ua);
  const float2 rvw = mul2(pk1(ra), vw);
  float f0 = fmaf(c1, __fsub_rn(rsa, ra), ru);
  float f1 = fmaf(c1, fmaf(rsa, SM, -ru), __fsub_rn(fmaf(ru, ua, pta), bx2));
  float2 f23 = fma2(C1, fma2(pk1(rsa), vws, pk(-rvw.x, -rvw.y)),
                    fma2(rvw, UA, pk(-__fmul_rn(bx, bb.x), -__fmul_rn(bx, bb.y))));
  float2 f45 = fma2(C1, sub2(bbs, bb), fma2(bb, UA, pk(-__fmul_rn(bx, vw.x), -__fmul_rn(bx, vw.y))));
  float f6 = fmaf(c1, __fsub_rn(esa, ea), fmaf(__fadd_rn(ea, pta), ua, -__fmul_rn(bx, vba)));

  // Alfven waves and double-star states; 1/sqrt(rho*) by rsqrt
  const float2 iq = pk(rsqrtf(rs.x), rsqrtf(rs.y));
  const float2 sq = mul2(rs, iq);
  const float abx = fabsf(bx);
  const float2 Ss = fma2(pk(-abx, abx), iq, SMv);  // (S_L*, S_R*)
  const float sg = bx >= 0.0f ? 1.0f : -1.0f;
  const float isum = rcp(__fadd_rn(sq.x, sq.y));
  const float sqLR = __fmul_rn(sq.x, sq.y);
  const float2 SG = pk1(sg), IS = pk1(isum), SQL = pk1(sq.x), SQR = pk1(sq.y);
  // (v**, w**) and (By**, Bz**)
  const float2 vwR = pk(vs.y, ws.y), vwL = pk(vs.x, ws.x);
  const float2 bbR = pk(bys.y, bzs.y), bbL = pk(bys.x, bzs.x);
  const float2 vwss = mul2(fma2(sub2(bbR, bbL), SG, fma2(SQR, vwR, mul2(SQL, vwL))), IS);
  const float2 bbss = mul2(fma2(pk1(sqLR), mul2(sub2(vwR, vwL), SG), fma2(SQR, bbL, mul2(SQL, bbR))), IS);
  const float vbss = fmaf(vwss.y, bbss.y, fmaf(vwss.x, bbss.x, __fmul_rn(SM, bx)));

  // inside the Alfven fan: c2 = S*_a
  const bool inner = !sup && (useL ? !(Ss.x > 0.0f) : !(Ss.y < 0.0f));
  const float sqa = useL ? -sq.x : sq.y;
  const float ess = fmaf(sqa, __fmul_rn(__fsub_rn(vbsa, vbss), sg), esa);
  const float c2 = inner ? (useL ? Ss.x : Ss.y) : 0.0f;
  const float c2rs = __fmul_rn(c2, rsa);
  f23 = fma2(pk1(c2rs), sub2(vwss, vws), f23);
  f45 = fma2(pk1(c2), sub2(bbss, bbs), f45);
  f6 = fmaf(c2, __fsub_rn(ess, esa), f6);

  F[kRHO] = f0;
  F[kPRS] = f6;
  F[kPSI] = __fmul_rn(__fmul_rn(ch, ch), bx);
  // un-rotate: component m gets rotated slot j = (m - dir) mod 3
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int j = (m - dir + 3) % 3;
    F[kVX + m] = j == 0 ? f1 : (j == 1 ? f23.x : f23.y);
    F[kBX + m] = j == 0 ? psis : (j == 1 ? f45.x : f45.y);
  }
}
#endif

// GLM interface step + HLLD along direction dir (0, 1, 2; template
// argument) for primitive face states vl, vr.  ch: cleaning speed;
// half_chi = 0.5 / ch.  F in conservative ordering.  Every sum of products
// is written with mul_rn / fma_rn / dot3_rn, so the flux rounds the same in
// every kernel and at every call site it is inlined into (the results of
// decomposed and undecomposed runs must agree bit for bit).
template <int dir, class T>
MHD_HD void glm_hlld_flux(const T vl[kNV], const T vr[kNV], T ch, T half_chi,
                          const Phys<T>& ph, T F[kNV]) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  if constexpr (sizeof(T) == 4) {  // FP32 on the device: the packed form
    glm_hlld_flux_f32x2<dir>(vl, vr, ch, half_chi, ph, F);
    return;
  }
#endif
  const T half = T(0.5);
  // rotate: u normal, (v, w) tangential in cyclic order; by, bz likewise
  const T uL = rot3(dir, 0, vl[kVX], vl[kVY], vl[kVZ]);
  const T vL = rot3(dir, 1, vl[kVX], vl[kVY], vl[kVZ]);
  const T wL = rot3(dir, 2, vl[kVX], vl[kVY], vl[kVZ]);
  const T bnL = rot3(dir, 0, vl[kBX], vl[kBY], vl[kBZ]);
  const T byL = rot3(dir, 1, vl[kBX], vl[kBY], vl[kBZ]);
  const T bzL = rot3(dir, 2, vl[kBX], vl[kBY], vl[kBZ]);
  const T uR = rot3(dir, 0, vr[kVX], vr[kVY], vr[kVZ]);
  const T vR = rot3(dir, 1, vr[kVX], vr[kVY], vr[kVZ]);
  const T wR = rot3(dir, 2, vr[kVX], vr[kVY], vr[kVZ]);
  const T bnR = rot3(dir, 0, vr[kBX], vr[kBY], vr[kBZ]);
  const T byR = rot3(dir, 1, vr[kBX], vr[kBY], vr[kBZ]);
  const T bzR = rot3(dir, 2, vr[kBX], vr[kBY], vr[kBZ]);
  const T rL = vl[kRHO], pL = vl[kPRS], rR = vr[kRHO], pR = vr[kPRS];

  // GLM: exact solution of the linear (B_n, psi) interface problem
  const T bx = fma_rn(half, bnL + bnR, -mul_rn(half_chi, vr[kPSI] - vl[kPSI]));
  const T psis = fma_rn(half, vl[kPSI] + vr[kPSI], -mul_rn(half * ch, bnR - bnL));
  const T bx2 = bx * bx;

  // outer states
  const T b2L = fma_rn(bzL, bzL, fma_rn(byL, byL, bx2));
  const T b2R = fma_rn(bzR, bzR, fma_rn(byR, byR, bx2));
  const T ptL = fma_rn(half, b2L, pL), ptR = fma_rn(half, b2R, pR);
  // (rho / 2 by half_of: an exponent move in FP64, the same value as 0.5 * rho)
  const T eL = fma_rn(half, b2L,
                      fma_rn(half_of(rL), dot3_rn(uL, uL, vL, vL, wL, wL), mul_rn(pL, ph.gm1i)));
  const T eR = fma_rn(half, b2R,
                      fma_rn(half_of(rR), dot3_rn(uR, uR, vR, vR, wR, wR), mul_rn(pR, ph.gm1i)));
  // 1/rho of both sides from one reciprocal; only max(c_fL, c_fR) is used,
  // so one square root of max(c_fL^2, c_fR^2) (sqrt is monotone and
  // correctly rounded: the same value)
  const T qr = rcp(rL * rR);
  const T cf2L = fast_speed2(rR * qr, ph.gamma * pL, b2L, bx2);
  const T cf2R = fast_speed2(rL * qr, ph.gamma * pR, b2R, bx2);

  // wave-speed estimates (MK05 Eq. 67), contact speed and total pressure
  const T cmax = tsqrt(tmax2(cf2L, cf2R));
  const T SL = tmin2(uL, uR) - cmax;
  const T SR = tmax2(uL, uR) + cmax;
  const T dL = (SL - uL) * rL, dR = (SR - uR) * rR;
  const T Di = rcp(dR - dL);
  const T SM = (fma_rn(dR, uR, -mul_rn(dL, uL)) - ptR + ptL) * Di;
  const T pts = fma_rn(mul_rn(dL, dR), uR - uL, fma_rn(dR, ptL, -mul_rn(dL, ptR))) * Di;

  // single-star states (MK05 Eqs. 43-48), degenerate when
  // |rho (S-u)(S-S_M) - Bx^2| < 1e-8 p_t*; paired reciprocals of S-S_M and
  // of the two denominators
  const T smL = SL - SM, smR = SR - SM;
  const T denL = fma_rn(dL, smL, -bx2), denR = fma_rn(dR, smR, -bx2);
  const bool degL = abs_lt(denL, T(1e-8) * pts);
  const bool degR = abs_lt(denR, T(1e-8) * pts);
  const T dnL = degL ? T(1) : denL, dnR = degR ? T(1) : denR;
  const T ps = smL * smR, pd = dnL * dnR;
  const T q4 = rcp(ps * pd);  // one reciprocal for the four divisors
  const T qs = pd * q4, qd = ps * q4;
  const T smiL = smR * qs, smiR = smL * qs;
  const T deniL = dnR * qd, deniR = dnL * qd;
  T rsL, vsL, wsL, bysL, bzsL, esL, vbsL, vbL;
  T rsR, vsR, wsR, bysR, bzsR, esR, vbsR, vbR;
  {
    rsL = dL * smiL;
    const T fv = bx * (SM - uL) * deniL;
    const T fb = fma_rn(dL, SL - uL, -bx2) * deniL;
    vsL = degL ? vL : fma_rn(-byL, fv, vL);
    wsL = degL ? wL : fma_rn(-bzL, fv, wL);
    bysL = degL ? byL : byL * fb;
    bzsL = degL ? bzL : bzL * fb;
    vbL = dot3_rn(uL, bx, vL, byL, wL, bzL);
    vbsL = dot3_rn(SM, bx, vsL, bysL, wsL, bzsL);
    esL = fma_rn(bx, vbL - vbsL,
                   fma_rn(pts, SM, fma_rn(SL - uL, eL, -mul_rn(ptL, uL)))) *
          smiL;
  }
  {
    rsR = dR * smiR;
    const T fv = bx * (SM - uR) * deniR;
    const T fb = fma_rn(dR, SR - uR, -bx2) * deniR;
    vsR = degR ? vR : fma_rn(-byR, fv, vR);
    wsR = degR ? wR : fma_rn(-bzR, fv, wR);
    bysR = degR ? byR : byR * fb;
    bzsR = degR ? bzR : bzR * fb;
    vbR = dot3_rn(uR, bx, vR, byR, wR, bzR);
    vbsR = dot3_rn(SM, bx, vsR, bysR, wsR, bzsR);
    esR = fma_rn(bx, vbR - vbsR,
                   fma_rn(pts, SM, fma_rn(SR - uR, eR, -mul_rn(ptR, uR)))) *
          smiR;
  }

  // Fan region: side a = L if (S_L > 0) or (S_R >= 0 and S_M >= 0), else R
  // (sign tests on the integer pipe in FP64: gt0 / lt0 / ge0).  The side's
  // outer and single-star values are picked here, before the double-star
  // states, so that the other side's outer state is no longer live there.
  const bool sup = gt0(SL) || lt0(SR);
  const bool useL = gt0(SL) || (!lt0(SR) && ge0(SM));
  const T r = useL ? rL : rR, u = useL ? uL : uR, v = useL ? vL : vR, w = useL ? wL : wR;
  const T by = useL ? byL : byR, bz = useL ? bzL : bzR, e = useL ? eL : eR;
  const T pt = useL ? ptL : ptR;
  const T rs = useL ? rsL : rsR, vs = useL ? vsL : vsR, ws = useL ? wsL : wsR;
  const T bys = useL ? bysL : bysR, bzs = useL ? bzsL : bzsR, es = useL ? esL : esR;
  const T vbs = useL ? vbsL : vbsR;
  const T vb = useL ? vbL : vbR;  // v . B of the side's outer state
  // the flux terms of the outer and single-star states (the Alfven-fan
  // terms are added below), so that the outer state dies here
  const T c1 = sup ? T(0) : (useL ? SL : SR);
  T f[7];
  {
    const T ru = mul_rn(r, u), rv = mul_rn(r, v), rw = mul_rn(r, w);
    f[0] = fma_rn(c1, rs - r, ru);
    f[1] = fma_rn(c1, fma_rn(rs, SM, -ru), fma_rn(ru, u, pt) - bx2);
    f[2] = fma_rn(c1, fma_rn(rs, vs, -rv), fma_rn(rv, u, -mul_rn(bx, by)));
    f[3] = fma_rn(c1, fma_rn(rs, ws, -rw), fma_rn(rw, u, -mul_rn(bx, bz)));
    f[4] = fma_rn(c1, bys - by, fma_rn(by, u, -mul_rn(bx, v)));
    f[5] = fma_rn(c1, bzs - bz, fma_rn(bz, u, -mul_rn(bx, w)));
    f[6] = fma_rn(c1, es - e, fma_rn(e + pt, u, -mul_rn(bx, vb)));
  }

  // Alfven waves (MK05 Eq. 51) and double-star states (Eqs. 59-63);
  // 1/sqrt(rho*) by rsqrt, sqrt(rho*) = rho* / sqrt(rho*)
  const T iqL = trsqrt(rsL), iqR = trsqrt(rsR);
  const T sqL = rsL * iqL, sqR = rsR * iqR;
  const T abx = tabs(bx);
  const T SLs = fma_rn(-abx, iqL, SM);
  const T SRs = fma_rn(abx, iqR, SM);
  // sign(B_x) applied as a sign flip (sign_mul), not a multiplication
  const long long sg = sign_bit_of(!ge0(bx));
  const T isum = rcp(sqL + sqR);
  const T sqLR = mul_rn(sqL, sqR);
  const T vss = (fma_rn(sqR, vsR, mul_rn(sqL, vsL)) + sign_mul(bysR - bysL, sg)) * isum;
  const T wss = (fma_rn(sqR, wsR, mul_rn(sqL, wsL)) + sign_mul(bzsR - bzsL, sg)) * isum;
  const T byss = fma_rn(sqLR, sign_mul(vsR - vsL, sg), fma_rn(sqR, bysL, mul_rn(sqL, bysR))) * isum;
  const T bzss = fma_rn(sqLR, sign_mul(wsR - wsL, sg), fma_rn(sqR, bzsL, mul_rn(sqL, bzsR))) * isum;
  const T vbss = dot3_rn(SM, bx, vss, byss, wss, bzss);

  // F = F_a + c1 (U*_a - U_a) + c2 (U**_a - U*_a) with c1 = S_a unless the
  // interface is supersonic, c2 = S*_a inside the Alfven fan.
  const bool inner = !sup && (useL ? !gt0(SLs) : !lt0(SRs));
  const T sq = useL ? -sqL : sqR;
  const T ess = fma_rn(sq, sign_mul(vbs - vbss, sg), es);
  const T c2 = inner ? (useL ? SLs : SRs) : T(0);
  const T c2rs = mul_rn(c2, rs);
  f[2] = fma_rn(c2rs, vss - vs, f[2]);
  f[3] = fma_rn(c2rs, wss - ws, f[3]);
  f[4] = fma_rn(c2, byss - bys, f[4]);
  f[5] = fma_rn(c2, bzss - bzs, f[5]);
  f[6] = fma_rn(c2, ess - es, f[6]);

  F[kRHO] = f[0];
  F[kPRS] = f[6];
  F[kPSI] = ch * ch * bx;
  // un-rotate: component m of a vector gets rotated slot j = (m - dir) mod 3
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int j = (m - dir + 3) % 3;
    F[kVX + m] = j == 0 ? f[1] : (j == 1 ? f[2] : f[3]);
    F[kBX + m] = j == 0 ? psis : (j == 1 ? f[4] : f[5]);
  }
}

}  // namespace mhd

namespace mhd {
// Runtime-direction entry (batched unit kernel): dispatches to the
// compile-time direction.
template <class T>
MHD_HD void glm_hlld_flux_dir(const T vl[kNV], const T vr[kNV], int dir, T ch, T half_chi,
                              const Phys<T>& ph, T F[kNV]) {
  if (dir == 0)
    glm_hlld_flux<0>(vl, vr, ch, half_chi, ph, F);
  else if (dir == 1)
    glm_hlld_flux<1>(vl, vr, ch, half_chi, ph, F);
  else
    glm_hlld_flux<2>(vl, vr, ch, half_chi, ph, F);
}
}  // namespace mhd
