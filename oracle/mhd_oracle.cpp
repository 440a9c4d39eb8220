// Test infrastructure -- NOT part of the product path.
//
// Plain, slow, obviously-correct CPU restatement (FP64) of one time step of
// the finite-volume ideal-MHD + GLM scheme whose five per-stage steps are
// listed in Section 3.2 ("Porting of gPLUTO"): boundary exchange/calculation,
// conservative->primitive map, reconstruction of interface values, Riemann
// solver, right-hand side; with the divergence of B controlled by divergence
// cleaning (Section 4.2, strong-scaling paragraph) and HLLD named as the
// Riemann solver (Section 4.2, weak-scaling paragraph).  The paper names the
// algorithms but does not print their equations, so every formula below is
// the published method it names:
//   * HLLD: Miyoshi & Kusano (2005), J. Comput. Phys. 208, 315 ("MK05"),
//     their Eqs. 38-63 and 66-67.
//   * GLM (mixed hyperbolic/parabolic divergence cleaning): Dedner et al.
//     (2002), J. Comput. Phys. 175, 645, Eq. 41 (the exact solution of the
//     2x2 (B_n, psi) interface problem), and the operator-split damping
//     psi <- psi exp(-alpha c_h dt / dh) of Mignone & Tzeferacos (2010),
//     J. Comput. Phys. 229, 2117, Eq. 27.
//   * PLM on primitive variables with the minmod or monotonised-central (MC)
//     limiter of van Leer (1977); or WENO-Z (Borges, Carmona, Costa & Don
//     2008, J. Comput. Phys. 227, 3191: their weights with exponent 1 and the
//     Jiang & Shu 1996 smoothness indicators), the reconstruction of the
//     paper's own runs (Section 4.2).
//   * RK2: two-stage, second-order (Heun / SSP) Runge-Kutta; or the
//     three-stage third-order SSP Runge-Kutta of Shu & Osher (1988), the
//     paper's RK3 (Section 4.2).
//   * CFL time step from the global maximum of |v_d| + c_f,d.
// Readings where the paper is silent are the ones stated next to each
// function.  Everything is templated on the scalar S so that S = Dual gives
// the exact directional derivative (JVP) of the same arithmetic.
//
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
// this library.  It shares no code with the CUDA path.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -shared -fPIC (oracle/__init__.py).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

namespace orc {

// ---------------------------------------------------------------- scalars --
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }

inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
inline double ssqrt(double a) { return std::sqrt(a); }
inline Dual ssqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, s > 0 ? 0.5 * a.d / s : 0.0);
}
inline double sabs(double a) { return std::fabs(a); }
inline Dual sabs(Dual a) { return a.v < 0 ? -a : a; }
template <class S> inline S smin(S a, S b) { return val(b) < val(a) ? b : a; }
template <class S> inline S smax(S a, S b) { return val(b) > val(a) ? b : a; }

// ------------------------------------------------------------- variables --
// Primitive V = (rho, vx, vy, vz, Bx, By, Bz, p, psi)
// Conservative U = (rho, mx, my, mz, Bx, By, Bz, E, psi)
enum { RHO = 0, VX = 1, VY = 2, VZ = 3, BX = 4, BY = 5, BZ = 6, PRS = 7, PSI = 8, NV = 9 };
enum { LIM_FLAT = 0, LIM_MINMOD = 1, LIM_MC = 2, LIM_WENOZ = 3 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1 };

struct Params {
  int n[3];
  double dx[3];
  double gamma;
  double glm_alpha;
  double rho_floor, p_floor;
  int limiter;
  int bc[6];
  int rk_order;  // 2 or 3
};

inline int ghost_width(const Params& P) { return P.limiter == LIM_WENOZ ? 3 : 2; }

struct Counters {
  long long rho_floor_hits;
  long long p_floor_hits;
};

// Total energy density E = p/(gamma-1) + rho |v|^2 / 2 + |B|^2 / 2
// (units with the 4 pi absorbed into B).
template <class S>
void prim_to_cons(const S V[NV], S U[NV], double gamma) {
  S v2 = V[VX] * V[VX] + V[VY] * V[VY] + V[VZ] * V[VZ];
  S b2 = V[BX] * V[BX] + V[BY] * V[BY] + V[BZ] * V[BZ];
  U[RHO] = V[RHO];
  U[VX] = V[RHO] * V[VX];
  U[VY] = V[RHO] * V[VY];
  U[VZ] = V[RHO] * V[VZ];
  U[BX] = V[BX];
  U[BY] = V[BY];
  U[BZ] = V[BZ];
  U[PRS] = V[PRS] / (gamma - 1.0) + 0.5 * V[RHO] * v2 + 0.5 * b2;
  U[PSI] = V[PSI];
}

// Step 2 of the stage (Section 3.2): conservative -> primitive.
// Reading: absolute floors rho_floor and p_floor, applied by replacement
// (rho first, then p), and counted.
template <class S>
void cons_to_prim(const S U[NV], S V[NV], const Params& P, Counters* c) {
  S rho = U[RHO];
  if (val(rho) < P.rho_floor) {
    rho = S(P.rho_floor);
    if (c) c->rho_floor_hits++;
  }
  S m2 = U[VX] * U[VX] + U[VY] * U[VY] + U[VZ] * U[VZ];
  S b2 = U[BX] * U[BX] + U[BY] * U[BY] + U[BZ] * U[BZ];
  S p = (P.gamma - 1.0) * (U[PRS] - 0.5 * m2 / rho - 0.5 * b2);
  if (val(p) < P.p_floor) {
    p = S(P.p_floor);
    if (c) c->p_floor_hits++;
  }
  V[RHO] = rho;
  V[VX] = U[VX] / rho;
  V[VY] = U[VY] / rho;
  V[VZ] = U[VZ] / rho;
  V[BX] = U[BX];
  V[BY] = U[BY];
  V[BZ] = U[BZ];
  V[PRS] = p;
  V[PSI] = U[PSI];
}

// Fast magnetosonic speed along direction d (0,1,2) with normal field bn:
// c_f^2 = ( (gp+|B|^2)/rho + sqrt( ((gp+|B|^2)/rho)^2 - 4 gp bn^2/rho^2 ) )/2,
// discriminant clamped at zero.
template <class S>
S fast_speed(const S V[NV], S bn, double gamma) {
  S gp = gamma * V[PRS];
  S b2 = V[BX] * V[BX] + V[BY] * V[BY] + V[BZ] * V[BZ];
  S a = (gp + b2) / V[RHO];
  S disc = a * a - 4.0 * gp * bn * bn / (V[RHO] * V[RHO]);
  if (val(disc) < 0.0) disc = S(0.0);
  return ssqrt(0.5 * (a + ssqrt(disc)));
}

// Slope limiters of van Leer (1977).
template <class S>
S limited_slope(S dm, S dp, int lim) {
  if (lim == LIM_FLAT) return S(0.0);
  if (val(dm) * val(dp) <= 0.0) return S(0.0);
  S am = sabs(dm), ap = sabs(dp);
  S mag;
  if (lim == LIM_MINMOD) {
    mag = smin(am, ap);
  } else {  // MC
    mag = smin(smin(2.0 * am, 2.0 * ap), 0.5 * sabs(dm + dp));
  }
  return val(dm) > 0.0 ? mag : -mag;
}

// WENO-Z value at the face x_{i+1/2}, biased towards cell i, from the five
// values f[0..4] at cells i-2 .. i+2 (Borges et al. 2008, exponent 1,
// epsilon 1e-40; candidate stencils and smoothness indicators of Jiang & Shu
// 1996).  The value at x_{i-1/2} biased towards cell i is the same function
// of the reversed stencil.
template <class S>
S wenoz_face(const S f[5]) {
  auto sq = [](S a) { return a * a; };
  S q0 = (2.0 * f[0] - 7.0 * f[1] + 11.0 * f[2]) / 6.0;
  S q1 = (-f[1] + 5.0 * f[2] + 2.0 * f[3]) / 6.0;
  S q2 = (2.0 * f[2] + 5.0 * f[3] - f[4]) / 6.0;
  S b0 = 13.0 / 12.0 * sq(f[0] - 2.0 * f[1] + f[2]) + 0.25 * sq(f[0] - 4.0 * f[1] + 3.0 * f[2]);
  S b1 = 13.0 / 12.0 * sq(f[1] - 2.0 * f[2] + f[3]) + 0.25 * sq(f[1] - f[3]);
  S b2 = 13.0 / 12.0 * sq(f[2] - 2.0 * f[3] + f[4]) + 0.25 * sq(3.0 * f[2] - 4.0 * f[3] + f[4]);
  S tau = sabs(b0 - b2);
  const double eps = 1e-40;
  S a0 = 0.1 * (1.0 + tau / (b0 + eps));
  S a1 = 0.6 * (1.0 + tau / (b1 + eps));
  S a2 = 0.3 * (1.0 + tau / (b2 + eps));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// Physical MHD flux along the rotated normal (index n = velocity component,
// bn = normal field), for the 7 HLLD components.  The entries for the normal
// field and psi are set by the GLM step, not here.
// Output in U ordering with the same rotation: F[RHO], F[mom n], F[mom t1],
// F[mom t2], F[B t1], F[B t2], F[E].
template <class S>
struct Rot {
  int n, t1, t2;  // velocity indices
  int bn, b1, b2;  // field indices
};
inline Rot<double> rot_for(int d) {
  Rot<double> r;
  r.n = VX + d;
  r.t1 = VX + (d + 1) % 3;
  r.t2 = VX + (d + 2) % 3;
  r.bn = BX + d;
  r.b1 = BX + (d + 1) % 3;
  r.b2 = BX + (d + 2) % 3;
  return r;
}

// 1-D state in rotated variables (MK05 notation: u normal, v,w tangential).
template <class S>
struct St {
  S rho, u, v, w, by, bz, p, pt, e;
};

// Fluxes of (rho, rho u, rho v, rho w, By, Bz, E) for given Bx (MK05 Eq. 3).
template <class S>
void flux7(const St<S>& q, S bx, S F[7]) {
  S vb = q.u * bx + q.v * q.by + q.w * q.bz;
  F[0] = q.rho * q.u;
  F[1] = q.rho * q.u * q.u + q.pt - bx * bx;
  F[2] = q.rho * q.v * q.u - bx * q.by;
  F[3] = q.rho * q.w * q.u - bx * q.bz;
  F[4] = q.by * q.u - bx * q.v;
  F[5] = q.bz * q.u - bx * q.w;
  F[6] = (q.e + q.pt) * q.u - bx * vb;
}

template <class S>
void cons7(const St<S>& q, S U[7]) {
  U[0] = q.rho;
  U[1] = q.rho * q.u;
  U[2] = q.rho * q.v;
  U[3] = q.rho * q.w;
  U[4] = q.by;
  U[5] = q.bz;
  U[6] = q.e;
}

// Step 4: the HLLD approximate Riemann solver (MK05), with the normal field
// bx already replaced by the GLM interface value.  Returns the 7 flux
// components in the order of flux7().
// Readings: wave-speed estimates S_L, S_R of MK05 Eq. 67; the intermediate
// states are taken as degenerate (v*, w*, By*, Bz* equal to the outer state)
// when |rho (S-u)(S-S_M) - Bx^2| < 1e-8 p_t* (MK05 Sect. 4.2 discusses the
// degeneracy without fixing the threshold); sign(0) = +1.
template <class S>
void hlld7(const St<S>& L, const St<S>& R, S bx, S cfL, S cfR, S F[7]) {
  S cmax = smax(cfL, cfR);
  S SL = smin(L.u, R.u) - cmax;  // MK05 Eq. 67
  S SR = smax(L.u, R.u) + cmax;

  S FL[7], FR[7];
  flux7(L, bx, FL);
  flux7(R, bx, FR);
  if (val(SL) > 0.0) {
    for (int k = 0; k < 7; ++k) F[k] = FL[k];
    return;
  }
  if (val(SR) < 0.0) {
    for (int k = 0; k < 7; ++k) F[k] = FR[k];
    return;
  }

  S dL = (SL - L.u) * L.rho;  // rho_L (S_L - u_L)
  S dR = (SR - R.u) * R.rho;
  S D = dR - dL;
  S SM = (dR * R.u - dL * L.u - R.pt + L.pt) / D;                   // MK05 Eq. 38
  S ptS = (dR * L.pt - dL * R.pt + dL * dR * (R.u - L.u)) / D;      // MK05 Eq. 41
  S bx2 = bx * bx;

  // Single-star states (MK05 Eqs. 43-48).
  St<S> sL, sR;
  const St<S>* outer[2] = {&L, &R};
  St<S>* star[2] = {&sL, &sR};
  S Sa[2] = {SL, SR};
  for (int s = 0; s < 2; ++s) {
    const St<S>& q = *outer[s];
    St<S>& t = *star[s];
    S da = (Sa[s] - q.u) * q.rho;
    t.rho = da / (Sa[s] - SM);                                   // Eq. 43
    t.u = SM;                                                     // Eq. 39
    t.pt = ptS;
    S den = da * (Sa[s] - SM) - bx2;
    if (val(sabs(den)) < 1e-8 * val(ptS)) {
      t.v = q.v;
      t.w = q.w;
      t.by = q.by;
      t.bz = q.bz;
    } else {
      S fac_v = bx * (SM - q.u) / den;
      t.v = q.v - q.by * fac_v;                                   // Eq. 44
      t.w = q.w - q.bz * fac_v;                                   // Eq. 46
      S fac_b = (da * (Sa[s] - q.u) - bx2) / den;
      t.by = q.by * fac_b;                                        // Eq. 45
      t.bz = q.bz * fac_b;                                        // Eq. 47
    }
    S vb = q.u * bx + q.v * q.by + q.w * q.bz;
    S vbs = t.u * bx + t.v * t.by + t.w * t.bz;
    t.e = ((Sa[s] - q.u) * q.e - q.pt * q.u + ptS * SM + bx * (vb - vbs)) /
          (Sa[s] - SM);                                           // Eq. 48
    t.p = S(0.0);
  }

  S rL = ssqrt(sL.rho), rR = ssqrt(sR.rho);
  S SLs = SM - sabs(bx) / rL;  // Eq. 51
  S SRs = SM + sabs(bx) / rR;

  S UL[7], UR[7], UsL[7], UsR[7];
  cons7(L, UL);
  cons7(R, UR);
  cons7(sL, UsL);
  cons7(sR, UsR);

  if (val(SLs) > 0.0) {  // S_L <= 0 < S*_L: F*_L = F_L + S_L (U*_L - U_L), Eq. 64
    for (int k = 0; k < 7; ++k) F[k] = FL[k] + SL * (UsL[k] - UL[k]);
    return;
  }
  if (val(SRs) < 0.0) {  // S*_R < 0 <= S_R: F*_R
    for (int k = 0; k < 7; ++k) F[k] = FR[k] + SR * (UsR[k] - UR[k]);
    return;
  }

  // Double-star states (MK05 Eqs. 59-63).
  S sgn = val(bx) >= 0.0 ? S(1.0) : S(-1.0);
  S isum = 1.0 / (rL + rR);
  St<S> ssL, ssR;
  S vss = (rL * sL.v + rR * sR.v + (sR.by - sL.by) * sgn) * isum;       // Eq. 59
  S wss = (rL * sL.w + rR * sR.w + (sR.bz - sL.bz) * sgn) * isum;       // Eq. 60
  S byss = (rL * sR.by + rR * sL.by + rL * rR * (sR.v - sL.v) * sgn) * isum;  // Eq. 61
  S bzss = (rL * sR.bz + rR * sL.bz + rL * rR * (sR.w - sL.w) * sgn) * isum;  // Eq. 62
  S vbss = SM * bx + vss * byss + wss * bzss;
  ssL = sL;
  ssR = sR;
  ssL.v = ssR.v = vss;
  ssL.w = ssR.w = wss;
  ssL.by = ssR.by = byss;
  ssL.bz = ssR.bz = bzss;
  S vbsL = sL.u * bx + sL.v * sL.by + sL.w * sL.bz;
  S vbsR = sR.u * bx + sR.v * sR.by + sR.w * sR.bz;
  ssL.e = sL.e - rL * (vbsL - vbss) * sgn;  // Eq. 63
  ssR.e = sR.e + rR * (vbsR - vbss) * sgn;

  S UssL[7], UssR[7];
  cons7(ssL, UssL);
  cons7(ssR, UssR);
  if (val(SM) >= 0.0) {  // S*_L <= 0 <= S_M: F**_L = F*_L + S*_L (U**_L - U*_L), Eq. 65
    for (int k = 0; k < 7; ++k)
      F[k] = FL[k] + SL * (UsL[k] - UL[k]) + SLs * (UssL[k] - UsL[k]);
  } else {  // S_M < 0 <= S*_R
    for (int k = 0; k < 7; ++k)
      F[k] = FR[k] + SR * (UsR[k] - UR[k]) + SRs * (UssR[k] - UsR[k]);
  }
}

// Full interface flux in direction d for primitive face states VL, VR:
// GLM interface step (Dedner et al. 2002, Eq. 41) then HLLD.
// F is in conservative ordering (rho, mx, my, mz, Bx, By, Bz, E, psi).
template <class S>
void interface_flux(const S VLin[NV], const S VRin[NV], int d, double ch, double gamma,
                    S F[NV]) {
  Rot<double> r = rot_for(d);
  S bnL = VLin[r.bn], bnR = VRin[r.bn];
  S psL = VLin[PSI], psR = VRin[PSI];
  S bn = 0.5 * (bnL + bnR) - (psR - psL) / (2.0 * ch);
  S ps = 0.5 * (psL + psR) - 0.5 * ch * (bnR - bnL);

  St<S> q[2];
  S cf[2];
  const S* Vin[2] = {VLin, VRin};
  for (int s = 0; s < 2; ++s) {
    S V[NV];
    for (int k = 0; k < NV; ++k) V[k] = Vin[s][k];
    V[r.bn] = bn;  // both sides carry the GLM normal field
    St<S>& t = q[s];
    t.rho = V[RHO];
    t.u = V[r.n];
    t.v = V[r.t1];
    t.w = V[r.t2];
    t.by = V[r.b1];
    t.bz = V[r.b2];
    t.p = V[PRS];
    S b2 = bn * bn + t.by * t.by + t.bz * t.bz;
    S v2 = t.u * t.u + t.v * t.v + t.w * t.w;
    t.pt = t.p + 0.5 * b2;
    t.e = t.p / (gamma - 1.0) + 0.5 * t.rho * v2 + 0.5 * b2;
    cf[s] = fast_speed(V, bn, gamma);
  }
  S F7[7];
  hlld7(q[0], q[1], bn, cf[0], cf[1], F7);
  F[RHO] = F7[0];
  F[r.n] = F7[1];
  F[r.t1] = F7[2];
  F[r.t2] = F7[3];
  F[r.bn] = ps;
  F[r.b1] = F7[4];
  F[r.b2] = F7[5];
  F[PRS] = F7[6];
  F[PSI] = ch * ch * bn;
}

// ------------------------------------------------------------------ grid --
// Padded SoA field: NV planes, each (n_z+2g_z) x (n_y+2g_y) x (n_x+2g_x),
// ghost width g_d = 2 in active dimensions (n_d > 1), 0 otherwise.
template <class S>
struct Field {
  int n[3], g[3], p[3];
  std::vector<S> a;
  explicit Field(const int nn[3], int gw = 2) {
    for (int d = 0; d < 3; ++d) {
      n[d] = nn[d];
      g[d] = nn[d] > 1 ? gw : 0;
      p[d] = n[d] + 2 * g[d];
    }
    a.assign((size_t)NV * p[0] * p[1] * p[2], S(0.0));
  }
  size_t idx(int v, int i, int j, int k) const {
    return (((size_t)v * p[2] + (k + g[2])) * p[1] + (j + g[1])) * p[0] + (i + g[0]);
  }
  S& at(int v, int i, int j, int k) { return a[idx(v, i, j, k)]; }
  const S& at(int v, int i, int j, int k) const { return a[idx(v, i, j, k)]; }
};

// Cell c of f is an interior cell (not a ghost).  Reading (the paper does not
// discuss floors): floor activations are counted once per stage for each
// interior cell, from its conversion of the stage input; the ghost copies'
// conversions and those of the time-step reduction are not counted.
template <class S>
bool interior(const Field<S>& f, const int c[3]) {
  for (int d = 0; d < 3; ++d)
    if (c[d] < 0 || c[d] >= f.n[d]) return false;
  return true;
}

// Step 1 of the stage (Section 3.2, "boundary exchange/calculation"): fill the
// ghost zones.  Periodic: ghost(i) = U(i mod N).  Outflow (zero gradient):
// ghost = nearest interior cell.  Dimension by dimension, each pass covering
// the ghosts already filled in the previous dimensions.
template <class S>
void fill_ghosts(Field<S>& f, const Params& P) {
  for (int d = 0; d < 3; ++d) {
    if (f.g[d] == 0) continue;
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      lo[e] = -f.g[e];
      hi[e] = f.n[e] + f.g[e];
    }
    lo[d] = 0;  // one pass per line along d
    hi[d] = 1;
    for (int side = 0; side < 2; ++side) {
      int bc = P.bc[2 * d + side];
      for (int gl = 0; gl < f.g[d]; ++gl) {
        int gi = side == 0 ? -1 - gl : f.n[d] + gl;  // ghost index along d
        int si;
        if (bc == BC_PERIODIC)
          si = ((gi % f.n[d]) + f.n[d]) % f.n[d];
        else
          si = side == 0 ? 0 : f.n[d] - 1;
        int c[3];
        for (int v = 0; v < NV; ++v)
          for (c[2] = lo[2]; c[2] < hi[2]; ++c[2])
            for (c[1] = lo[1]; c[1] < hi[1]; ++c[1])
              for (c[0] = lo[0]; c[0] < hi[0]; ++c[0]) {
                int a[3] = {c[0], c[1], c[2]}, b[3] = {c[0], c[1], c[2]};
                a[d] = gi;
                b[d] = si;
                f.at(v, a[0], a[1], a[2]) = f.at(v, b[0], b[1], b[2]);
              }
      }
    }
  }
}

// Step 3 of a stage (reconstruction): the left and right primitive states
// of the face f = c[d] along d, which separates cells f-1 (left) and f
// (right); the other two coordinates of c are the face's cell indices.
template <class S>
void face_states(const Params& P, const Field<S>& V, int d, const int c[3], S face[2][NV]) {
  for (int side = 0; side < 2; ++side) {
    const int cell = c[d] - 1 + side;  // f-1 (left), f (right)
    auto at = [&](int k, int off) {
      int a[3] = {c[0], c[1], c[2]};
      a[d] = cell + off;
      return V.at(k, a[0], a[1], a[2]);
    };
    S plus[NV], minus[NV];  // values at the cell's faces +1/2 and -1/2
    if (P.limiter == LIM_WENOZ) {
      for (int k = 0; k < NV; ++k) {
        S st[5], rv[5];
        for (int o = -2; o <= 2; ++o) st[o + 2] = at(k, o);
        for (int o = 0; o < 5; ++o) rv[o] = st[4 - o];
        plus[k] = wenoz_face(st);
        minus[k] = wenoz_face(rv);
      }
    } else {
      for (int k = 0; k < NV; ++k) {
        S sig = limited_slope(at(k, 0) - at(k, -1), at(k, 1) - at(k, 0), P.limiter);
        plus[k] = at(k, 0) + 0.5 * sig;
        minus[k] = at(k, 0) - 0.5 * sig;
      }
    }
    // Reading: if either face value of this cell has rho <= 0 or p <= 0, the
    // cell falls back to its own (flat) value.
    bool bad = val(plus[RHO]) <= 0.0 || val(minus[RHO]) <= 0.0 || val(plus[PRS]) <= 0.0 ||
               val(minus[PRS]) <= 0.0;
    for (int k = 0; k < NV; ++k) {
      const S v0 = at(k, 0);
      face[side][k] = bad ? v0 : (side == 0 ? plus[k] : minus[k]);
    }
  }
}

// One RK2 stage (Section 3.2, steps 1-5) on the input W.  Writes
//   stage 1:  out = W + dt L(W)
//   stage 2:  out = (Un + (W + dt L(W))) / 2
// on interior cells.  W's ghosts are (re)filled here.
// Runge-Kutta stage coefficients: out = a_n U^n + a_w (W + dt L(W)).
inline void rk_coeffs(int order, int stage, double* a_n, double* a_w) {
  if (stage == 1) {
    *a_n = 0.0;
    *a_w = 1.0;
  } else if (order == 2) {
    *a_n = 0.5;
    *a_w = 0.5;
  } else if (stage == 2) {
    *a_n = 0.75;
    *a_w = 0.25;
  } else {
    *a_n = 1.0 / 3.0;
    *a_w = 2.0 / 3.0;
  }
}

template <class S>
void rk_stage(const Params& P, Field<S>& W, const Field<S>* Un, double dt, double ch,
              int stage, Field<S>& out, Counters* cnt, bool fill = true) {
  if (fill) fill_ghosts(W, P);                                        // step 1

  Field<S> V(P.n, ghost_width(P));                                    // step 2
  {
    int c[3];
    for (c[2] = -W.g[2]; c[2] < W.n[2] + W.g[2]; ++c[2])
      for (c[1] = -W.g[1]; c[1] < W.n[1] + W.g[1]; ++c[1])
        for (c[0] = -W.g[0]; c[0] < W.n[0] + W.g[0]; ++c[0]) {
          S u[NV], v[NV];
          for (int k = 0; k < NV; ++k) u[k] = W.at(k, c[0], c[1], c[2]);
          cons_to_prim(u, v, P, interior(W, c) ? cnt : nullptr);
          for (int k = 0; k < NV; ++k) V.at(k, c[0], c[1], c[2]) = v[k];
        }
  }

  // L(W) on interior cells.
  const size_t ncell = (size_t)P.n[0] * P.n[1] * P.n[2];
  std::vector<S> L((size_t)NV * ncell, S(0.0));
  auto lidx = [&](int v, int i, int j, int k) {
    return (((size_t)v * P.n[2] + k) * P.n[1] + j) * P.n[0] + i;
  };

  for (int d = 0; d < 3; ++d) {
    if (P.n[d] <= 1) continue;
    // Faces f = 0..n_d along d; face f separates cells f-1 and f.
    int fn[3] = {P.n[0], P.n[1], P.n[2]};
    fn[d] += 1;
    std::vector<S> Fd((size_t)NV * fn[0] * fn[1] * fn[2]);
    auto fidx = [&](int v, int i, int j, int k) {
      return (((size_t)v * fn[2] + k) * fn[1] + j) * fn[0] + i;
    };
    int c[3];
    for (c[2] = 0; c[2] < fn[2]; ++c[2])
      for (c[1] = 0; c[1] < fn[1]; ++c[1])
        for (c[0] = 0; c[0] < fn[0]; ++c[0]) {
          // Step 3: reconstruction.
          S face[2][NV];
          face_states(P, V, d, c, face);
          // Step 4: GLM + HLLD.
          S F[NV];
          interface_flux(face[0], face[1], d, ch, P.gamma, F);
          for (int k = 0; k < NV; ++k) Fd[fidx(k, c[0], c[1], c[2])] = F[k];
        }
    // Step 5: right-hand side, -dF/dx_d accumulated per cell.
    for (c[2] = 0; c[2] < P.n[2]; ++c[2])
      for (c[1] = 0; c[1] < P.n[1]; ++c[1])
        for (c[0] = 0; c[0] < P.n[0]; ++c[0]) {
          int a[3] = {c[0], c[1], c[2]};
          a[d] += 1;
          for (int k = 0; k < NV; ++k) {
            S fp = Fd[fidx(k, a[0], a[1], a[2])];
            S fm = Fd[fidx(k, c[0], c[1], c[2])];
            L[lidx(k, c[0], c[1], c[2])] -= (fp - fm) / P.dx[d];
          }
        }
  }

  // Runge-Kutta combination.
  double a_n, a_w;
  rk_coeffs(P.rk_order, stage, &a_n, &a_w);
  int c[3];
  for (c[2] = 0; c[2] < P.n[2]; ++c[2])
    for (c[1] = 0; c[1] < P.n[1]; ++c[1])
      for (c[0] = 0; c[0] < P.n[0]; ++c[0])
        for (int k = 0; k < NV; ++k) {
          S w = W.at(k, c[0], c[1], c[2]);
          S s1 = w + dt * L[lidx(k, c[0], c[1], c[2])];
          if (stage == 1)
            out.at(k, c[0], c[1], c[2]) = s1;
          else
            out.at(k, c[0], c[1], c[2]) = a_n * Un->at(k, c[0], c[1], c[2]) + a_w * s1;
        }
}

// Global CFL time step (reading: the paper does not state it).
// lambda = max over interior cells and active d of |v_d| + c_f,d (normal field
// = the cell's own B_d); c_h = lambda; dt = cfl / (c_h * sum_active 1/dx_d).
template <class S>
double max_speed(const Params& P, const Field<S>& U, Counters* cnt) {
  double lam = 0.0;
  int c[3];
  for (c[2] = 0; c[2] < P.n[2]; ++c[2])
    for (c[1] = 0; c[1] < P.n[1]; ++c[1])
      for (c[0] = 0; c[0] < P.n[0]; ++c[0]) {
        S u[NV], v[NV];
        for (int k = 0; k < NV; ++k) u[k] = U.at(k, c[0], c[1], c[2]);
        cons_to_prim(u, v, P, cnt);
        for (int d = 0; d < 3; ++d) {
          if (P.n[d] <= 1) continue;
          double s = std::fabs(val(v[VX + d])) + val(fast_speed(v, v[BX + d], P.gamma));
          if (!(s <= lam)) lam = s;  // NaN propagates
        }
      }
  return lam;
}

// GLM damping of psi after a full step (Mignone & Tzeferacos 2010, Eq. 27).
inline double damping_factor(const Params& P, double dt, double ch) {
  double dh = 1e300;
  for (int d = 0; d < 3; ++d)
    if (P.n[d] > 1) dh = std::min(dh, P.dx[d]);
  return std::exp(-P.glm_alpha * ch * dt / dh);
}

// One full Runge-Kutta step (RK2, or SSP-RK3 when rk_order == 3) with frozen
// dt and c_h, followed by the GLM damping
// psi <- psi exp(-alpha c_h dt / dh_min) (Mignone & Tzeferacos 2010, Eq. 27).
template <class S>
void rk2_step(const Params& P, Field<S>& U, double dt, double ch, Counters* cnt) {
  const int gw = ghost_width(P);
  Field<S> U1(P.n, gw), Un1(P.n, gw);
  rk_stage(P, U, (const Field<S>*)nullptr, dt, ch, 1, U1, cnt);
  if (P.rk_order == 3) {
    Field<S> U2(P.n, gw);
    rk_stage(P, U1, &U, dt, ch, 2, U2, cnt);
    rk_stage(P, U2, &U, dt, ch, 3, Un1, cnt);
  } else {
    rk_stage(P, U1, &U, dt, ch, 2, Un1, cnt);
  }
  const double damp = damping_factor(P, dt, ch);
  int c[3];
  for (c[2] = 0; c[2] < P.n[2]; ++c[2])
    for (c[1] = 0; c[1] < P.n[1]; ++c[1])
      for (c[0] = 0; c[0] < P.n[0]; ++c[0]) {
        for (int k = 0; k < NV; ++k) U.at(k, c[0], c[1], c[2]) = Un1.at(k, c[0], c[1], c[2]);
        U.at(PSI, c[0], c[1], c[2]) = damp * Un1.at(PSI, c[0], c[1], c[2]);
      }
}

template <class S>
void load_interior(Field<S>& f, const double* src, const double* tan) {
  const int* n = f.n;
  size_t m = 0;
  for (int v = 0; v < NV; ++v)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i, ++m) {
          if constexpr (sizeof(S) == sizeof(double))
            f.at(v, i, j, k) = S(src[m]);
          else
            f.at(v, i, j, k) = S(src[m], tan ? tan[m] : 0.0);
        }
}

template <class S>
void store_interior(const Field<S>& f, double* dst, double* tan) {
  const int* n = f.n;
  size_t m = 0;
  for (int v = 0; v < NV; ++v)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i, ++m) {
          dst[m] = val(f.at(v, i, j, k));
          if constexpr (sizeof(S) != sizeof(double))
            if (tan) tan[m] = f.at(v, i, j, k).d;
        }
}


// ------------------------------------------------- constrained transport --
// The div-B control of the paper's weak-scaling runs (Section 4.2):
// constrained transport (Evans & Hawley 1988; Londrillo & Del Zanna 2004).
// The magnetic field is kept on cell faces, b_d on the faces normal to d, and
// advanced by Faraday's law in integral (Stokes) form, db/dt = -curl E with
// the electric field E = -v x B on cell edges, so the face divergence
// sum_d (b_d(+1/2) - b_d(-1/2)) / dx_d does not change.  Readings (the paper
// names the method only):
//   * three active dimensions, periodic boundaries;
//   * b_d stored at cell (i, j, k) is the one on the cell's lower d-face;
//     the cell-centred B of the conservative state is the mean of the cell's
//     two faces;
//   * each face's Riemann problem (the same reconstruction and HLLD as with
//     GLM) takes the staggered b_d as its normal field on both sides; psi is
//     identically zero (with equal normal fields and psi = 0 the GLM interface
//     step of interface_flux is the identity);
//   * the edge electric field is the upwind "CT-contact" average of Gardiner
//     & Stone (2005, J. Comput. Phys. 205, 509): the mean of the four face
//     values plus the difference of upwinded edge-to-cell derivatives, the
//     upwind side chosen by the sign of the face mass flux (their Eqs. 41,
//     45 and 50-51); a mass flux with |F_rho| <= 1e-12 c_h rho (rho of the
//     cell owning the face) counts as zero, so round-off cannot choose a side;
//   * the face field is combined across Runge-Kutta stages like the
//     conservative variables; there is no psi damping.
struct Faces {
  int n[3];
  std::vector<double> b[3];
  explicit Faces(const int nn[3]) {
    for (int d = 0; d < 3; ++d) n[d] = nn[d];
    for (int d = 0; d < 3; ++d) b[d].assign((size_t)n[0] * n[1] * n[2], 0.0);
  }
  // periodic wrap of any cell index
  size_t idx(int i, int j, int k) const {
    i = ((i % n[0]) + n[0]) % n[0];
    j = ((j % n[1]) + n[1]) % n[1];
    k = ((k % n[2]) + n[2]) % n[2];
    return ((size_t)k * n[1] + j) * n[0] + i;
  }
  double& at(int d, int i, int j, int k) { return b[d][idx(i, j, k)]; }
  double at(int d, int i, int j, int k) const { return b[d][idx(i, j, k)]; }
};

// A per-cell scalar array with periodic wrap (face, edge and cell-centred
// electric fields).
struct CellArray {
  int n[3];
  std::vector<double> a;
  explicit CellArray(const int nn[3]) {
    for (int d = 0; d < 3; ++d) n[d] = nn[d];
    a.assign((size_t)n[0] * n[1] * n[2], 0.0);
  }
  double& at(int i, int j, int k) {
    i = ((i % n[0]) + n[0]) % n[0];
    j = ((j % n[1]) + n[1]) % n[1];
    k = ((k % n[2]) + n[2]) % n[2];
    return a[((size_t)k * n[1] + j) * n[0] + i];
  }
};

// Upwind choice of Gardiner & Stone (2005): positive mass flux takes the
// candidate of the low side, negative that of the high side, zero their mean.
inline double ct_upwind(double F, double from_lo, double from_hi) {
  if (F > 0.0) return from_lo;
  if (F < 0.0) return from_hi;
  return 0.5 * (from_lo + from_hi);
}

// CT-contact electric field on an edge along e.  a and b are the two other
// directions.  The edge touches four faces and four cells:
//   Ea[0], Ea[1]: values on the a-faces on the low and high b side, with mass
//                 fluxes Fa[0], Fa[1];
//   Eb[0], Eb[1]: values on the b-faces on the low and high a side, with mass
//                 fluxes Fb[0], Fb[1];
//   Ec[ia][ib]:   cell-centred values, ia / ib = 0 (low) or 1 (high) side.
// Gardiner & Stone (2005), Eq. 41: E = (sum of the four faces)/4
//   + (db/8) (dE/db at the low quarter - dE/db at the high quarter)
//   + (da/8) (dE/da at the low quarter - dE/da at the high quarter),
// with each quarter derivative 2 (face - cell) / d (or 2 (cell - face) / d)
// taken from the cell upwind of the face whose mass flux it sits on
// (Eqs. 50-51); the d/8 and 2/d factors combine to 1/4.
double ct_contact_emf(const double Ea[2], const double Fa[2], const double Eb[2],
                      const double Fb[2], const double Ec[2][2]) {
  const double mean = 0.25 * (Ea[0] + Ea[1] + Eb[0] + Eb[1]);
  // dE/db on the low-b a-face and on the high-b a-face (upwind along a)
  const double db_lo = ct_upwind(Fa[0], Eb[0] - Ec[0][0], Eb[1] - Ec[1][0]);
  const double db_hi = ct_upwind(Fa[1], Ec[0][1] - Eb[0], Ec[1][1] - Eb[1]);
  // dE/da on the low-a b-face and on the high-a b-face (upwind along b)
  const double da_lo = ct_upwind(Fb[0], Ea[0] - Ec[0][0], Ea[1] - Ec[0][1]);
  const double da_hi = ct_upwind(Fb[1], Ec[1][0] - Ea[0], Ec[1][1] - Ea[1]);
  return mean + 0.25 * (db_lo - db_hi) + 0.25 * (da_lo - da_hi);
}

// Cell-centred B = mean of the cell's two faces, written into U.
inline void ct_cell_field(const Faces& b, Field<double>& U) {
  for (int k = 0; k < b.n[2]; ++k)
    for (int j = 0; j < b.n[1]; ++j)
      for (int i = 0; i < b.n[0]; ++i) {
        U.at(BX, i, j, k) = 0.5 * (b.at(0, i, j, k) + b.at(0, i + 1, j, k));
        U.at(BY, i, j, k) = 0.5 * (b.at(1, i, j, k) + b.at(1, i, j + 1, k));
        U.at(BZ, i, j, k) = 0.5 * (b.at(2, i, j, k) + b.at(2, i, j, k + 1));
      }
}

// One Runge-Kutta stage with constrained transport: out / bout =
// a_n (Un, bn) + a_w ((W, bw) + dt L(W, bw)) (stage 1: a_n = 0, a_w = 1).
void ct_stage(const Params& P, Field<double>& W, const Faces& bw, const Field<double>* Un,
              const Faces* bn, double dt, double ch, int stage, Field<double>& out,
              Faces& bout, Counters* cnt) {
  fill_ghosts(W, P);                                                  // step 1
  Field<double> V(P.n, ghost_width(P));                               // step 2
  {
    int c[3];
    for (c[2] = -W.g[2]; c[2] < W.n[2] + W.g[2]; ++c[2])
      for (c[1] = -W.g[1]; c[1] < W.n[1] + W.g[1]; ++c[1])
        for (c[0] = -W.g[0]; c[0] < W.n[0] + W.g[0]; ++c[0]) {
          double u[NV], v[NV];
          for (int k = 0; k < NV; ++k) u[k] = W.at(k, c[0], c[1], c[2]);
          cons_to_prim(u, v, P, interior(W, c) ? cnt : nullptr);
          for (int k = 0; k < NV; ++k) V.at(k, c[0], c[1], c[2]) = v[k];
        }
  }
  const int* n = P.n;
  const size_t ncell = (size_t)n[0] * n[1] * n[2];
  auto lidx = [&](int v, int i, int j, int k) {
    return (((size_t)v * n[2] + k) * n[1] + j) * n[0] + i;
  };
  std::vector<double> L((size_t)NV * ncell, 0.0);
  // Face electric fields (two per face: e1 along the first, e2 along the
  // second transverse axis in cyclic order) and mass fluxes, stored at the
  // cell owning the face.
  //   x-face: (Ey, Ez) = ( F[Bz], -F[By])
  //   y-face: (Ez, Ex) = ( F[Bx], -F[Bz])
  //   z-face: (Ex, Ey) = ( F[By], -F[Bx])
  // (F[B_t] = v_n B_t - v_t B_n and E = -v x B.)
  CellArray Ef[3][3] = {{CellArray(n), CellArray(n), CellArray(n)},
                        {CellArray(n), CellArray(n), CellArray(n)},
                        {CellArray(n), CellArray(n), CellArray(n)}};  // [face dir][E comp]
  CellArray Fm[3] = {CellArray(n), CellArray(n), CellArray(n)};

  for (int d = 0; d < 3; ++d) {
    int fn[3] = {n[0], n[1], n[2]};
    fn[d] += 1;
    std::vector<double> Fd((size_t)NV * fn[0] * fn[1] * fn[2]);
    auto fidx = [&](int v, int i, int j, int k) {
      return (((size_t)v * fn[2] + k) * fn[1] + j) * fn[0] + i;
    };
    const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
    int c[3];
    for (c[2] = 0; c[2] < fn[2]; ++c[2])
      for (c[1] = 0; c[1] < fn[1]; ++c[1])
        for (c[0] = 0; c[0] < fn[0]; ++c[0]) {
          double face[2][NV];
          face_states(P, V, d, c, face);                               // step 3
          const double bface = bw.at(d, c[0], c[1], c[2]);
          for (int s = 0; s < 2; ++s) {
            face[s][BX + d] = bface;
            face[s][PSI] = 0.0;
          }
          double F[NV];
          interface_flux(face[0], face[1], d, ch, P.gamma, F);         // step 4
          for (int k = 0; k < NV; ++k) Fd[fidx(k, c[0], c[1], c[2])] = F[k];
          if (c[d] < n[d]) {
            // E_e1 = -(v x B)_e1 = F[B_e2]; E_e2 = -F[B_e1]
            Ef[d][e1].at(c[0], c[1], c[2]) = F[BX + e2];
            Ef[d][e2].at(c[0], c[1], c[2]) = -F[BX + e1];
            const double thr = 1e-12 * ch * V.at(RHO, c[0], c[1], c[2]);
            Fm[d].at(c[0], c[1], c[2]) = std::fabs(F[RHO]) > thr ? F[RHO] : 0.0;
          }
        }
    for (c[2] = 0; c[2] < n[2]; ++c[2])                               // step 5
      for (c[1] = 0; c[1] < n[1]; ++c[1])
        for (c[0] = 0; c[0] < n[0]; ++c[0]) {
          int a[3] = {c[0], c[1], c[2]};
          a[d] += 1;
          for (int k : {RHO, VX, VY, VZ, PRS}) {
            const double fp = Fd[fidx(k, a[0], a[1], a[2])];
            const double fm = Fd[fidx(k, c[0], c[1], c[2])];
            L[lidx(k, c[0], c[1], c[2])] -= (fp - fm) / P.dx[d];
          }
        }
  }

  // Cell-centred electric field E = -v x B.
  CellArray Ec[3] = {CellArray(n), CellArray(n), CellArray(n)};
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        const double vx = V.at(VX, i, j, k), vy = V.at(VY, i, j, k), vz = V.at(VZ, i, j, k);
        const double Bx = V.at(BX, i, j, k), By = V.at(BY, i, j, k), Bz = V.at(BZ, i, j, k);
        Ec[0].at(i, j, k) = vz * By - vy * Bz;
        Ec[1].at(i, j, k) = vx * Bz - vz * Bx;
        Ec[2].at(i, j, k) = vy * Bx - vx * By;
      }

  // Edge electric fields.  E_e at cell (i, j, k) lives on the cell's edge
  // along e at the low corner of the other two directions.
  CellArray Ee[3] = {CellArray(n), CellArray(n), CellArray(n)};
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3, b = (e + 2) % 3;
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          // cell (i, j, k) shifted by -1 along a and/or b
          auto sh = [&](int da, int db, int out[3]) {
            out[0] = i;
            out[1] = j;
            out[2] = k;
            out[a] -= da;
            out[b] -= db;
          };
          int q[3];
          double Ea[2], Fa[2], Eb[2], Fb[2], Ecell[2][2];
          // a-faces of the cells on the low-b (shifted along b) and high-b side
          for (int s = 0; s < 2; ++s) {
            sh(0, 1 - s, q);
            Ea[s] = Ef[a][e].at(q[0], q[1], q[2]);
            Fa[s] = Fm[a].at(q[0], q[1], q[2]);
            sh(1 - s, 0, q);
            Eb[s] = Ef[b][e].at(q[0], q[1], q[2]);
            Fb[s] = Fm[b].at(q[0], q[1], q[2]);
          }
          for (int ia = 0; ia < 2; ++ia)
            for (int ib = 0; ib < 2; ++ib) {
              sh(1 - ia, 1 - ib, q);
              Ecell[ia][ib] = Ec[e].at(q[0], q[1], q[2]);
            }
          Ee[e].at(i, j, k) = ct_contact_emf(Ea, Fa, Eb, Fb, Ecell);
        }
  }

  // Faraday's law on the faces: db_d/dt = -(curl E)_d, with
  // (curl E)_d = dE_b/da - dE_a/db for (d, a, b) cyclic.
  double a_n, a_w;
  rk_coeffs(P.rk_order, stage, &a_n, &a_w);
  for (int d = 0; d < 3; ++d) {
    const int a = (d + 1) % 3, b = (d + 2) % 3;
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          int pa[3] = {i, j, k}, pb[3] = {i, j, k};
          pa[a] += 1;
          pb[b] += 1;
          const double curl = (Ee[b].at(pa[0], pa[1], pa[2]) - Ee[b].at(i, j, k)) / P.dx[a] -
                              (Ee[a].at(pb[0], pb[1], pb[2]) - Ee[a].at(i, j, k)) / P.dx[b];
          const double s1 = bw.at(d, i, j, k) - dt * curl;
          bout.at(d, i, j, k) = stage == 1 ? s1 : a_n * bn->at(d, i, j, k) + a_w * s1;
        }
  }

  // Conservative variables: rho, m, E by the flux divergence; B from the faces.
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        for (int q : {RHO, VX, VY, VZ, PRS}) {
          const double s1 = W.at(q, i, j, k) + dt * L[lidx(q, i, j, k)];
          out.at(q, i, j, k) = stage == 1 ? s1 : a_n * Un->at(q, i, j, k) + a_w * s1;
        }
        out.at(PSI, i, j, k) = 0.0;
      }
  ct_cell_field(bout, out);
}

// One full constrained-transport step (RK2 or SSP-RK3, frozen dt, c_h).
void ct_step(const Params& P, Field<double>& U, Faces& b, double dt, double ch,
             Counters* cnt) {
  const int gw = ghost_width(P);
  Field<double> U1(P.n, gw), Un1(P.n, gw);
  Faces b1(P.n), bn1(P.n);
  ct_stage(P, U, b, nullptr, nullptr, dt, ch, 1, U1, b1, cnt);
  if (P.rk_order == 3) {
    Field<double> U2(P.n, gw);
    Faces b2(P.n);
    ct_stage(P, U1, b1, &U, &b, dt, ch, 2, U2, b2, cnt);
    ct_stage(P, U2, b2, &U, &b, dt, ch, 3, Un1, bn1, cnt);
  } else {
    ct_stage(P, U1, b1, &U, &b, dt, ch, 2, Un1, bn1, cnt);
  }
  for (int k = 0; k < P.n[2]; ++k)
    for (int j = 0; j < P.n[1]; ++j)
      for (int i = 0; i < P.n[0]; ++i)
        for (int q = 0; q < NV; ++q) U.at(q, i, j, k) = Un1.at(q, i, j, k);
  b = bn1;
}

inline void load_faces(Faces& f, const double* src) {
  const size_t m = (size_t)f.n[0] * f.n[1] * f.n[2];
  for (int d = 0; d < 3; ++d) std::memcpy(f.b[d].data(), src + d * m, m * sizeof(double));
}
inline void store_faces(const Faces& f, double* dst) {
  const size_t m = (size_t)f.n[0] * f.n[1] * f.n[2];
  for (int d = 0; d < 3; ++d) std::memcpy(dst + d * m, f.b[d].data(), m * sizeof(double));
}

}  // namespace orc

// ------------------------------------------------------------- C exports --
using namespace orc;

extern "C" {

// Layout of every array argument: interior-only SoA, [9][nz][ny][nx] doubles.
struct orc_params {
  int n[3];
  double dx[3];
  double gamma, glm_alpha, rho_floor, p_floor;
  int limiter;
  int bc[6];
  int rk_order;
};

static Params to_params(const orc_params* p) {
  Params P;
  for (int d = 0; d < 3; ++d) {
    P.n[d] = p->n[d];
    P.dx[d] = p->dx[d];
  }
  P.gamma = p->gamma;
  P.glm_alpha = p->glm_alpha;
  P.rho_floor = p->rho_floor;
  P.p_floor = p->p_floor;
  P.limiter = p->limiter;
  for (int s = 0; s < 6; ++s) P.bc[s] = p->bc[s];
  P.rk_order = p->rk_order == 3 ? 3 : 2;
  return P;
}

// Pointwise maps over ncell cells; arrays are [9][ncell].
void orc_prim_to_cons(const double* V, double* U, long ncell, double gamma) {
  for (long c = 0; c < ncell; ++c) {
    double v[NV], u[NV];
    for (int k = 0; k < NV; ++k) v[k] = V[k * ncell + c];
    prim_to_cons(v, u, gamma);
    for (int k = 0; k < NV; ++k) U[k * ncell + c] = u[k];
  }
}

void orc_cons_to_prim(const orc_params* p, const double* U, double* V, long ncell,
                      long long counters[2]) {
  Params P = to_params(p);
  Counters cnt = {0, 0};
  for (long c = 0; c < ncell; ++c) {
    double u[NV], v[NV];
    for (int k = 0; k < NV; ++k) u[k] = U[k * ncell + c];
    cons_to_prim(u, v, P, &cnt);
    for (int k = 0; k < NV; ++k) V[k * ncell + c] = v[k];
  }
  if (counters) {
    counters[0] = cnt.rho_floor_hits;
    counters[1] = cnt.p_floor_hits;
  }
}

// Fast magnetosonic speed of each cell along d with the cell's own B_d.
void orc_fast_speed(const double* V, double* cf, long ncell, int d, double gamma) {
  for (long c = 0; c < ncell; ++c) {
    double v[NV];
    for (int k = 0; k < NV; ++k) v[k] = V[k * ncell + c];
    cf[c] = fast_speed(v, v[BX + d], gamma);
  }
}

// Interface fluxes for nface primitive face-state pairs, arrays [9][nface].
void orc_interface_flux(const double* VL, const double* VR, double* F, long nface, int d,
                        double ch, double gamma) {
  for (long f = 0; f < nface; ++f) {
    double l[NV], r[NV], out[NV];
    for (int k = 0; k < NV; ++k) {
      l[k] = VL[k * nface + f];
      r[k] = VR[k * nface + f];
    }
    interface_flux(l, r, d, ch, gamma, out);
    for (int k = 0; k < NV; ++k) F[k * nface + f] = out[k];
  }
}

// Limited slope sigma(dm, dp) elementwise.
void orc_limited_slope(const double* dm, const double* dp, double* out, long n, int lim) {
  for (long i = 0; i < n; ++i) out[i] = limited_slope(dm[i], dp[i], lim);
}

// WENO-Z face values: f is [5][n] (cells i-2..i+2), out[n] = value at
// x_{i+1/2} biased towards cell i.
void orc_wenoz_face(const double* f, double* out, long n) {
  for (long i = 0; i < n; ++i) {
    double st[5];
    for (int o = 0; o < 5; ++o) st[o] = f[o * n + i];
    out[i] = wenoz_face(st);
  }
}

// Ghost fill on an interior-only array, returning the padded array
// ([9][nz+2gz][ny+2gy][nx+2gx]).
void orc_fill_ghosts(const orc_params* p, const double* U, double* padded) {
  Params P = to_params(p);
  Field<double> f(P.n, ghost_width(P));
  load_interior(f, U, nullptr);
  fill_ghosts(f, P);
  std::memcpy(padded, f.a.data(), f.a.size() * sizeof(double));
}

// lambda = max |v_d| + c_f,d (see max_speed).
double orc_max_speed(const orc_params* p, const double* U, long long counters[2]) {
  Params P = to_params(p);
  Field<double> f(P.n, ghost_width(P));
  load_interior(f, U, nullptr);
  Counters cnt = {0, 0};
  double lam = max_speed(P, f, &cnt);
  if (counters) {
    counters[0] = cnt.rho_floor_hits;
    counters[1] = cnt.p_floor_hits;
  }
  return lam;
}

// One RK2 stage; Un may be null for stage 1.
void orc_stage(const orc_params* p, const double* W, const double* Un, double dt, double ch,
               int stage, double* out, long long counters[2]) {
  Params P = to_params(p);
  Field<double> w(P.n, ghost_width(P)), un(P.n, ghost_width(P)), o(P.n, ghost_width(P));
  load_interior(w, W, nullptr);
  if (Un) load_interior(un, Un, nullptr);
  Counters cnt = {0, 0};
  rk_stage(P, w, Un ? &un : nullptr, dt, ch, stage, o, &cnt);
  store_interior(o, out, nullptr);
  if (counters) {
    counters[0] = cnt.rho_floor_hits;
    counters[1] = cnt.p_floor_hits;
  }
}

// One RK2 stage on a caller-filled padded array (ghost zones supplied by the
// caller, e.g. exchanged between subdomains): Wp is
// [9][nz+2gz][ny+2gy][nx+2gx]; Un and out are interior-only.  With damp != 0
// (stage 2 only) psi of the result is multiplied by the step's GLM damping
// factor, completing the step.
void orc_stage_padded(const orc_params* p, const double* Wp, const double* Un, double dt,
                      double ch, int stage, int damp, double* out) {
  Params P = to_params(p);
  Field<double> w(P.n, ghost_width(P)), un(P.n, ghost_width(P)), o(P.n, ghost_width(P));
  std::memcpy(w.a.data(), Wp, w.a.size() * sizeof(double));
  if (Un) load_interior(un, Un, nullptr);
  rk_stage(P, w, Un ? &un : nullptr, dt, ch, stage, o, (Counters*)nullptr, false);
  if (damp) {
    const double f = damping_factor(P, dt, ch);
    for (int k = 0; k < P.n[2]; ++k)
      for (int j = 0; j < P.n[1]; ++j)
        for (int i = 0; i < P.n[0]; ++i) o.at(PSI, i, j, k) = f * o.at(PSI, i, j, k);
  }
  store_interior(o, out, nullptr);
}

// nsteps full RK2 steps in place.  If dts/chs are non-null and dts[s] > 0 the
// step uses the given dt/c_h; otherwise it computes c_h = lambda(U) and
// dt = cfl / (c_h sum 1/dx_d), clamped to t_end - t when t_end > 0.  The dt and
// c_h used are written back into dts/chs when those are non-null.
// Returns the time reached.
double orc_run(const orc_params* p, double* U, int nsteps, double cfl, double t0, double t_end,
               double* dts, double* chs, long long counters[2]) {
  Params P = to_params(p);
  Field<double> f(P.n, ghost_width(P));
  load_interior(f, U, nullptr);
  Counters cnt = {0, 0};
  double t = t0;
  double inv_sum = 0.0;
  for (int d = 0; d < 3; ++d)
    if (P.n[d] > 1) inv_sum += 1.0 / P.dx[d];
  for (int s = 0; s < nsteps; ++s) {
    if (t_end > 0.0 && t >= t_end) break;
    double dt, ch;
    if (dts && dts[s] > 0.0) {
      dt = dts[s];
      ch = chs[s];
    } else {
      ch = max_speed(P, f, (Counters*)nullptr);
      dt = cfl / (ch * inv_sum);
      if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
      if (dts) {
        dts[s] = dt;
        chs[s] = ch;
      }
    }
    rk2_step(P, f, dt, ch, &cnt);
    t += dt;
  }
  store_interior(f, U, nullptr);
  if (counters) {
    counters[0] = cnt.rho_floor_hits;
    counters[1] = cnt.p_floor_hits;
  }
  return t;
}

// Forward-mode derivative of nsteps RK2 steps with the recorded (frozen)
// dt/c_h sequence: (U, dU) -> (U_N, dU_N), in place.
void orc_run_jvp(const orc_params* p, double* U, double* dU, int nsteps, const double* dts,
                 const double* chs) {
  Params P = to_params(p);
  Field<Dual> f(P.n, ghost_width(P));
  load_interior(f, U, dU);
  for (int s = 0; s < nsteps; ++s) rk2_step(P, f, dts[s], chs[s], (Counters*)nullptr);
  store_interior(f, U, dU);
}

// Conservation sums: for v in (rho, mx, my, mz, E, Bx, By, Bz), sum_cells U_v
// times the cell volume (product of dx_d over active dims), with Kahan
// compensation.
void orc_conserved_sums(const orc_params* p, const double* U, double out[8]) {
  Params P = to_params(p);
  long ncell = (long)P.n[0] * P.n[1] * P.n[2];
  double vol = 1.0;
  for (int d = 0; d < 3; ++d)
    if (P.n[d] > 1) vol *= P.dx[d];
  const int vars[8] = {RHO, VX, VY, VZ, PRS, BX, BY, BZ};
  for (int q = 0; q < 8; ++q) {
    double s = 0.0, comp = 0.0;
    for (long c = 0; c < ncell; ++c) {
      double y = U[vars[q] * ncell + c] * vol - comp;
      double t = s + y;
      comp = (t - s) - y;
      s = t;
    }
    out[q] = s;
  }
}


// ---- constrained transport (face field arrays are [3][nz][ny][nx]: b_d on
// ---- the lower d-face of each cell)

// nsteps CT steps in place on (U, b); dt rule and dts/chs as orc_run.
double orc_ct_run(const orc_params* p, double* U, double* b, int nsteps, double cfl, double t0,
                  double t_end, double* dts, double* chs, long long counters[2]) {
  Params P = to_params(p);
  Field<double> f(P.n, ghost_width(P));
  load_interior(f, U, nullptr);
  Faces fb(P.n);
  load_faces(fb, b);
  Counters cnt = {0, 0};
  double t = t0;
  double inv_sum = 0.0;
  for (int d = 0; d < 3; ++d) inv_sum += 1.0 / P.dx[d];
  for (int s = 0; s < nsteps; ++s) {
    if (t_end > 0.0 && t >= t_end) break;
    double dt, ch;
    if (dts && dts[s] > 0.0) {
      dt = dts[s];
      ch = chs[s];
    } else {
      ch = max_speed(P, f, (Counters*)nullptr);
      dt = cfl / (ch * inv_sum);
      if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
      if (dts) {
        dts[s] = dt;
        chs[s] = ch;
      }
    }
    ct_step(P, f, fb, dt, ch, &cnt);
    t += dt;
  }
  store_interior(f, U, nullptr);
  store_faces(fb, b);
  if (counters) {
    counters[0] = cnt.rho_floor_hits;
    counters[1] = cnt.p_floor_hits;
  }
  return t;
}

// One first Runge-Kutta stage with constrained transport and the given dt,
// c_h: (W, bw) -> (out, bout) = (W, bw) + dt L(W, bw).
void orc_ct_stage1(const orc_params* p, const double* W, const double* bw, double dt, double ch,
                   double* out, double* bout) {
  Params P = to_params(p);
  Field<double> w(P.n, ghost_width(P)), o(P.n, ghost_width(P));
  load_interior(w, W, nullptr);
  Faces fb(P.n), fo(P.n);
  load_faces(fb, bw);
  ct_stage(P, w, fb, nullptr, nullptr, dt, ch, 1, o, fo, (Counters*)nullptr);
  store_interior(o, out, nullptr);
  store_faces(fo, bout);
}

// Face divergence of b per cell: sum_d (b_d(+1/2) - b_d(-1/2)) / dx_d.
void orc_ct_divb(const orc_params* p, const double* b, double* out) {
  Params P = to_params(p);
  Faces fb(P.n);
  load_faces(fb, b);
  size_t m = 0;
  for (int k = 0; k < P.n[2]; ++k)
    for (int j = 0; j < P.n[1]; ++j)
      for (int i = 0; i < P.n[0]; ++i, ++m)
        out[m] = (fb.at(0, i + 1, j, k) - fb.at(0, i, j, k)) / P.dx[0] +
                 (fb.at(1, i, j + 1, k) - fb.at(1, i, j, k)) / P.dx[1] +
                 (fb.at(2, i, j, k + 1) - fb.at(2, i, j, k)) / P.dx[2];
}

// CT-contact edge electric field for n edges; in is [12][n]:
// Ea0, Ea1, Fa0, Fa1, Eb0, Eb1, Fb0, Fb1, Ec00, Ec01, Ec10, Ec11.
void orc_ct_edge_emf(const double* in, double* out, long n) {
  for (long e = 0; e < n; ++e) {
    auto g = [&](int r) { return in[(long)r * n + e]; };
    const double Ea[2] = {g(0), g(1)}, Fa[2] = {g(2), g(3)};
    const double Eb[2] = {g(4), g(5)}, Fb[2] = {g(6), g(7)};
    const double Ec[2][2] = {{g(8), g(9)}, {g(10), g(11)}};
    out[e] = ct_contact_emf(Ea, Fa, Eb, Fb, Ec);
  }
}

}  // extern "C"
