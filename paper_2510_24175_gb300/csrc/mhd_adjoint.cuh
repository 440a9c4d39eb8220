// Reverse-mode derivatives (vector-Jacobian products) of the pointwise
// pieces of the stage: the GLM + HLLD interface flux, the limited PLM slope
// and the conservative->primitive map.  Written by hand, statement by
// statement in reverse order of the forward code in mhd_physics.cuh, with
// the same branch decisions (HLLD fan region, degenerate star state, limiter
// selection, positivity fallback), which are piecewise constant and carry no
// derivative.  dt and c_h are frozen constants.
#pragma once

#include "mhd_physics.cuh"

namespace mhd {

// Forward intermediates of one side of the HLLD fan.
template <class T>
struct Side {
  // outer state
  T r, u, v, w, by, bz, p, b2, pt, e, ri, gp, a, disc, sd, cf;
  T isd, icf;  // 1 / sd, 1 / cf (from reciprocal square roots)
  // single-star state
  T S, d, sm, smi, rs, den, deni, fv, fb, vs, ws, bys, bzs, vb, vbs, es, sq;
  bool deg, clamp;
};

// Adjoints of one side.
template <class T>
struct SideBar {
  T r, u, v, w, by, bz, p, b2, pt, e, ri, gp, a, disc, sd, cf;
  T S, d, sm, smi, rs, den, deni, fv, fb, vs, ws, bys, bzs, vb, vbs, es, sq;
};

template <class T>
MHD_HD void zero_bar(SideBar<T>& b) {
  b.r = b.u = b.v = b.w = b.by = b.bz = b.p = b.b2 = b.pt = b.e = T(0);
  b.ri = b.gp = b.a = b.disc = b.sd = b.cf = T(0);
  b.S = b.d = b.sm = b.smi = b.rs = b.den = b.deni = b.fv = b.fb = T(0);
  b.vs = b.ws = b.bys = b.bzs = b.vb = b.vbs = b.es = b.sq = T(0);
}

// Outer-state forward: total field, total pressure, energy and gamma p.  The
// reciprocal of rho is formed for both sides at once by the caller (one
// reciprocal of rho_L rho_R, as glm_hlld_flux does).
template <class T>
MHD_HD void side_outer(Side<T>& s, T bx2, const Phys<T>& ph) {
  const T half = T(0.5);
  s.b2 = bx2 + s.by * s.by + s.bz * s.bz;
  s.pt = s.p + half * s.b2;
  s.e = s.p * ph.gm1i + half * s.r * (s.u * s.u + s.v * s.v + s.w * s.w) + half * s.b2;
  s.gp = ph.gamma * s.p;
}

// Square of the fast speed, (a + sqrt(a^2 - 4 gp bx2 / rho^2)) / 2, with the
// reciprocal square root of the discriminant the reverse needs (sd = disc /
// sqrt(disc)); a clamped discriminant gives sd = 0.  Needs s.ri.  The root of
// the square itself is taken only for the faster side, the one c_max uses.
template <class T>
MHD_HD T side_c2(Side<T>& s, T bx2) {
  s.a = (s.gp + s.b2) * s.ri;
  const T disc = s.a * s.a - T(4) * s.gp * bx2 * (s.ri * s.ri);
  s.clamp = !gt0(disc);
  s.disc = s.clamp ? T(0) : disc;
  s.isd = trsqrt(s.disc);
  s.sd = s.clamp ? T(0) : s.disc * s.isd;
  return T(0.5) * (s.a + s.sd);
}

// Single-star state, first part: S - S_M, the denominator and the
// degeneracy test.  The caller forms 1 / (S - S_M) and 1 / den of both sides
// from one reciprocal (as glm_hlld_flux does) and sets s.smi, s.deni.
template <class T>
MHD_HD void side_star_den(Side<T>& s, T bx2, T SM, T pts) {
  s.sm = s.S - SM;
  s.den = s.d * s.sm - bx2;
  s.deg = abs_lt(s.den, T(1e-8) * pts);
}

template <class T>
MHD_HD void side_star(Side<T>& s, T bx, T bx2, T SM, T pts) {
  s.rs = s.d * s.smi;
  s.fv = bx * (SM - s.u) * s.deni;
  s.fb = (s.d * (s.S - s.u) - bx2) * s.deni;
  s.vs = s.deg ? s.v : s.v - s.by * s.fv;
  s.ws = s.deg ? s.w : s.w - s.bz * s.fv;
  s.bys = s.deg ? s.by : s.by * s.fb;
  s.bzs = s.deg ? s.bz : s.bz * s.fb;
  s.vb = s.u * bx + s.v * s.by + s.w * s.bz;
  s.vbs = SM * bx + s.vs * s.bys + s.ws * s.bzs;
  s.es = ((s.S - s.u) * s.e - s.pt * s.u + pts * SM + bx * (s.vb - s.vbs)) * s.smi;
}

// Reverse of side_star.  Accumulates into sb and the shared adjoints.
template <class T>
MHD_HD void side_star_bar(const Side<T>& s, SideBar<T>& sb, T bx, T bx2, T SM, T pts,
                          T& bxb, T& bx2b, T& SMb, T& ptsb) {
  // es = Ne * smi
  const T Ne = (s.S - s.u) * s.e - s.pt * s.u + pts * SM + bx * (s.vb - s.vbs);
  const T Neb = sb.es * s.smi;
  sb.smi += sb.es * Ne;
  sb.S += Neb * s.e;
  sb.u -= Neb * s.e;
  sb.e += Neb * (s.S - s.u);
  sb.pt -= Neb * s.u;
  sb.u -= Neb * s.pt;
  ptsb += Neb * SM;
  SMb += Neb * pts;
  bxb += Neb * (s.vb - s.vbs);
  sb.vb += Neb * bx;
  sb.vbs -= Neb * bx;
  // vbs = SM bx + vs bys + ws bzs
  SMb += sb.vbs * bx;
  bxb += sb.vbs * SM;
  sb.vs += sb.vbs * s.bys;
  sb.bys += sb.vbs * s.vs;
  sb.ws += sb.vbs * s.bzs;
  sb.bzs += sb.vbs * s.ws;
  // vb = u bx + v by + w bz
  sb.u += sb.vb * bx;
  bxb += sb.vb * s.u;
  sb.v += sb.vb * s.by;
  sb.by += sb.vb * s.v;
  sb.w += sb.vb * s.bz;
  sb.bz += sb.vb * s.w;
  if (s.deg) {
    sb.v += sb.vs;
    sb.w += sb.ws;
    sb.by += sb.bys;
    sb.bz += sb.bzs;
  } else {
    sb.v += sb.vs;
    sb.by -= sb.vs * s.fv;
    sb.fv -= sb.vs * s.by;
    sb.w += sb.ws;
    sb.bz -= sb.ws * s.fv;
    sb.fv -= sb.ws * s.bz;
    sb.by += sb.bys * s.fb;
    sb.fb += sb.bys * s.by;
    sb.bz += sb.bzs * s.fb;
    sb.fb += sb.bzs * s.bz;
    // fb = (d (S - u) - bx2) deni
    sb.d += sb.fb * (s.S - s.u) * s.deni;
    sb.S += sb.fb * s.d * s.deni;
    sb.u -= sb.fb * s.d * s.deni;
    bx2b -= sb.fb * s.deni;
    sb.deni += sb.fb * (s.d * (s.S - s.u) - bx2);
    // fv = bx (SM - u) deni
    bxb += sb.fv * (SM - s.u) * s.deni;
    SMb += sb.fv * bx * s.deni;
    sb.u -= sb.fv * bx * s.deni;
    sb.deni += sb.fv * bx * (SM - s.u);
    // deni = 1 / den; den = d sm - bx2
    sb.den -= sb.deni * s.deni * s.deni;
    sb.d += sb.den * s.sm;
    sb.sm += sb.den * s.d;
    bx2b -= sb.den;
  }
  // rs = d smi; smi = 1 / sm; sm = S - SM
  sb.d += sb.rs * s.smi;
  sb.smi += sb.rs * s.d;
  sb.sm -= sb.smi * s.smi * s.smi;
  sb.S += sb.sm;
  SMb -= sb.sm;
}

// Reverse of side_outer.
template <class T>
MHD_HD void side_outer_bar(const Side<T>& s, SideBar<T>& sb, T bx2, const Phys<T>& ph,
                           T& bx2b) {
  const T half = T(0.5);
  // cf = sqrt(half (a + sd))
  const T cf2b = sb.cf * half * s.icf;
  sb.a += half * cf2b;
  sb.sd += half * cf2b;
  // sd = sqrt(disc) (disc clamped at 0: no derivative through the clamp)
  if (!s.clamp && gt0(s.sd)) sb.disc += sb.sd * half * s.isd;
  // disc = a^2 - 4 gp bx2 ri^2
  sb.a += sb.disc * T(2) * s.a;
  sb.gp -= sb.disc * T(4) * bx2 * s.ri * s.ri;
  bx2b -= sb.disc * T(4) * s.gp * s.ri * s.ri;
  sb.ri -= sb.disc * T(8) * s.gp * bx2 * s.ri;
  // a = (gp + b2) ri
  sb.gp += sb.a * s.ri;
  sb.b2 += sb.a * s.ri;
  sb.ri += sb.a * (s.gp + s.b2);
  // gp = gamma p; ri = 1 / r
  sb.p += ph.gamma * sb.gp;
  sb.r -= sb.ri * s.ri * s.ri;
  // e = p gm1i + r (u^2+v^2+w^2)/2 + b2/2
  sb.p += sb.e * ph.gm1i;
  sb.r += sb.e * half * (s.u * s.u + s.v * s.v + s.w * s.w);
  sb.u += sb.e * s.r * s.u;
  sb.v += sb.e * s.r * s.v;
  sb.w += sb.e * s.r * s.w;
  sb.b2 += half * sb.e;
  // pt = p + b2/2
  sb.p += sb.pt;
  sb.b2 += half * sb.pt;
  // b2 = bx2 + by^2 + bz^2
  bx2b += sb.b2;
  sb.by += T(2) * s.by * sb.b2;
  sb.bz += T(2) * s.bz * sb.b2;
}

// Vector-Jacobian product of glm_hlld_flux: given the flux adjoint Fb (9,
// conservative ordering) returns the adjoints of the primitive face states
// vlb, vrb (9 each, overwritten).
template <class T>
MHD_HD void glm_hlld_flux_vjp(const T vl[kNV], const T vr[kNV], int dir, T ch, T half_chi,
                              const Phys<T>& ph, const T Fb[kNV], T vlb[kNV], T vrb[kNV]) {
  const T half = T(0.5);
  Side<T> L, R;
  L.r = vl[kRHO];
  L.p = vl[kPRS];
  L.u = rot3(dir, 0, vl[kVX], vl[kVY], vl[kVZ]);
  L.v = rot3(dir, 1, vl[kVX], vl[kVY], vl[kVZ]);
  L.w = rot3(dir, 2, vl[kVX], vl[kVY], vl[kVZ]);
  L.by = rot3(dir, 1, vl[kBX], vl[kBY], vl[kBZ]);
  L.bz = rot3(dir, 2, vl[kBX], vl[kBY], vl[kBZ]);
  R.r = vr[kRHO];
  R.p = vr[kPRS];
  R.u = rot3(dir, 0, vr[kVX], vr[kVY], vr[kVZ]);
  R.v = rot3(dir, 1, vr[kVX], vr[kVY], vr[kVZ]);
  R.w = rot3(dir, 2, vr[kVX], vr[kVY], vr[kVZ]);
  R.by = rot3(dir, 1, vr[kBX], vr[kBY], vr[kBZ]);
  R.bz = rot3(dir, 2, vr[kBX], vr[kBY], vr[kBZ]);
  const T bnL = rot3(dir, 0, vl[kBX], vl[kBY], vl[kBZ]);
  const T bnR = rot3(dir, 0, vr[kBX], vr[kBY], vr[kBZ]);

  // ---------------------------------------------------------- forward --
  const T bx = half * (bnL + bnR) - half_chi * (vr[kPSI] - vl[kPSI]);
  const T bx2 = bx * bx;
  side_outer(L, bx2, ph);
  side_outer(R, bx2, ph);
  // 1/rho of both sides from one reciprocal
  const T qr = rcp(L.r * R.r);
  L.ri = R.r * qr;
  R.ri = L.r * qr;
  const T c2L = side_c2(L, bx2), c2R = side_c2(R, bx2);
  // (comparisons on the integer pipe in FP64: lt_ieee, gt0, lt0, ge0)
  const bool cfL_max = !lt_ieee(c2L, c2R);  // cmax = cfL on ties (sqrt is monotone)
  // c_max = sqrt(max(c2L, c2R)); only that side's fast speed has an adjoint,
  // the other side's 1/cf is zero
  const T icf = trsqrt(cfL_max ? c2L : c2R);
  const T cmax = (cfL_max ? c2L : c2R) * icf;
  L.cf = cfL_max ? cmax : T(0);
  L.icf = cfL_max ? icf : T(0);
  R.cf = cfL_max ? T(0) : cmax;
  R.icf = cfL_max ? T(0) : icf;
  const bool uL_min = !lt_ieee(R.u, L.u);     // min(uL, uR) picks uL on ties
  const bool uL_max = !lt_ieee(L.u, R.u);     // max(uL, uR) picks uL on ties
  L.S = (uL_min ? L.u : R.u) - cmax;
  R.S = (uL_max ? L.u : R.u) + cmax;
  L.d = (L.S - L.u) * L.r;
  R.d = (R.S - R.u) * R.r;
  const T Di = rcp(R.d - L.d);
  const T Ns = R.d * R.u - L.d * L.u - R.pt + L.pt;
  const T SM = Ns * Di;
  const T Np = R.d * L.pt - L.d * R.pt + L.d * R.d * (R.u - L.u);
  const T pts = Np * Di;
  // 1/(S - S_M) and 1/den of both sides from one reciprocal
  side_star_den(L, bx2, SM, pts);
  side_star_den(R, bx2, SM, pts);
  {
    const T dnL = L.deg ? T(1) : L.den, dnR = R.deg ? T(1) : R.den;
    const T ps = L.sm * R.sm, pd = dnL * dnR;
    const T q4 = rcp(ps * pd);
    const T qs = pd * q4, qd = ps * q4;
    L.smi = R.sm * qs;
    R.smi = L.sm * qs;
    L.deni = dnR * qd;
    R.deni = dnL * qd;
  }
  side_star(L, bx, bx2, SM, pts);
  side_star(R, bx, bx2, SM, pts);
  const T abx = tabs(bx);
  const T sg = ge0(bx) ? T(1) : T(-1);
  const bool sup = gt0(L.S) || lt0(R.S);
  const bool useL = gt0(L.S) || (!lt0(R.S) && ge0(SM));
  // inside the Alfven fan: decided by the selected side's Alfven speed
  const T iqa = trsqrt(useL ? L.rs : R.rs);
  const bool inner = !sup && (useL ? !gt0(SM - abx * iqa) : !lt0(SM + abx * iqa));
  // The double-star states enter only inside the fan (c2 != 0).  Where no
  // lane of the warp is inside, they and their reverse are skipped: their
  // adjoints would all be zero.
#ifdef __CUDA_ARCH__
  const bool fan = __any_sync(__activemask(), inner);
#else
  const bool fan = inner;
#endif
  T iqL = T(0), iqR = T(0), SLs = T(0), SRs = T(0), isum = T(0);
  T Nv = T(0), Nw = T(0), Nby = T(0), Nbz = T(0);
  T vss = T(0), wss = T(0), byss = T(0), bzss = T(0), vbss = T(0);
  L.sq = R.sq = T(0);
  if (fan) {
    const T iqo = trsqrt(useL ? R.rs : L.rs);
    iqL = useL ? iqa : iqo;
    iqR = useL ? iqo : iqa;
    L.sq = L.rs * iqL;
    R.sq = R.rs * iqR;
    SLs = SM - abx * iqL;
    SRs = SM + abx * iqR;
    isum = rcp(L.sq + R.sq);
    Nv = L.sq * L.vs + R.sq * R.vs + (R.bys - L.bys) * sg;
    Nw = L.sq * L.ws + R.sq * R.ws + (R.bzs - L.bzs) * sg;
    Nby = L.sq * R.bys + R.sq * L.bys + L.sq * R.sq * (R.vs - L.vs) * sg;
    Nbz = L.sq * R.bzs + R.sq * L.bzs + L.sq * R.sq * (R.ws - L.ws) * sg;
    vss = Nv * isum;
    wss = Nw * isum;
    byss = Nby * isum;
    bzss = Nbz * isum;
    vbss = SM * bx + vss * byss + wss * bzss;
  }
  // selected side a
  const T r = useL ? L.r : R.r, u = useL ? L.u : R.u, v = useL ? L.v : R.v;
  const T w = useL ? L.w : R.w, by = useL ? L.by : R.by, bz = useL ? L.bz : R.bz;
  const T e = useL ? L.e : R.e, pt = useL ? L.pt : R.pt;
  const T rs = useL ? L.rs : R.rs, vs = useL ? L.vs : R.vs, ws = useL ? L.ws : R.ws;
  const T bys = useL ? L.bys : R.bys, bzs = useL ? L.bzs : R.bzs, es = useL ? L.es : R.es;
  const T sq = useL ? -L.sq : R.sq;
  const T vbs = useL ? L.vbs : R.vbs;
  const T ess = es + sq * (vbs - vbss) * sg;
  const T c1 = sup ? T(0) : (useL ? L.S : R.S);
  const T c2 = inner ? (useL ? SLs : SRs) : T(0);
  const T vb = u * bx + v * by + w * bz;

  // ---------------------------------------------------------- reverse --
  // un-rotate the flux adjoint into the 7 HLLD components
  T fb[7];
  fb[0] = Fb[kRHO];
  fb[6] = Fb[kPRS];
  T psisb = T(0);
  // rotated slot j of a vector is component (dir + j) mod 3
  fb[1] = rot3(dir, 0, Fb[kVX], Fb[kVY], Fb[kVZ]);
  fb[2] = rot3(dir, 1, Fb[kVX], Fb[kVY], Fb[kVZ]);
  fb[3] = rot3(dir, 2, Fb[kVX], Fb[kVY], Fb[kVZ]);
  psisb = rot3(dir, 0, Fb[kBX], Fb[kBY], Fb[kBZ]);
  fb[4] = rot3(dir, 1, Fb[kBX], Fb[kBY], Fb[kBZ]);
  fb[5] = rot3(dir, 2, Fb[kBX], Fb[kBY], Fb[kBZ]);
  T bxb = ch * ch * Fb[kPSI];
  T bx2b = T(0), SMb = T(0), ptsb = T(0);
  // adjoints of the selected-side quantities
  T rb = 0, ub = 0, vb_ = 0, wb = 0, byb = 0, bzb = 0, eb = 0, ptb = 0;
  T rsb = 0, vsb = 0, wsb = 0, bysb = 0, bzsb = 0, esb = 0, vbsb = 0, sqb = 0;
  T vssb = 0, wssb = 0, byssb = 0, bzssb = 0, vbssb = 0, essb = 0, c1b = 0, c2b = 0, vbb = 0;
  // f0 = r u + c1 (rs - r)
  rb += fb[0] * (u - c1);
  ub += fb[0] * r;
  c1b += fb[0] * (rs - r);
  rsb += fb[0] * c1;
  // f1 = r u u + pt - bx2 + c1 (rs SM - r u)
  rb += fb[1] * (u * u - c1 * u);
  ub += fb[1] * (T(2) * r * u - c1 * r);
  ptb += fb[1];
  bx2b -= fb[1];
  c1b += fb[1] * (rs * SM - r * u);
  rsb += fb[1] * c1 * SM;
  SMb += fb[1] * c1 * rs;
  // f2 = r v u - bx by + c1 (rs vs - r v) + c2 rs (vss - vs)
  rb += fb[2] * (v * u - c1 * v);
  vb_ += fb[2] * (r * u - c1 * r);
  ub += fb[2] * r * v;
  bxb -= fb[2] * by;
  byb -= fb[2] * bx;
  c1b += fb[2] * (rs * vs - r * v);
  rsb += fb[2] * (c1 * vs + c2 * (vss - vs));
  vsb += fb[2] * (c1 * rs - c2 * rs);
  c2b += fb[2] * rs * (vss - vs);
  vssb += fb[2] * c2 * rs;
  // f3 = r w u - bx bz + c1 (rs ws - r w) + c2 rs (wss - ws)
  rb += fb[3] * (w * u - c1 * w);
  wb += fb[3] * (r * u - c1 * r);
  ub += fb[3] * r * w;
  bxb -= fb[3] * bz;
  bzb -= fb[3] * bx;
  c1b += fb[3] * (rs * ws - r * w);
  rsb += fb[3] * (c1 * ws + c2 * (wss - ws));
  wsb += fb[3] * (c1 * rs - c2 * rs);
  c2b += fb[3] * rs * (wss - ws);
  wssb += fb[3] * c2 * rs;
  // f4 = by u - bx v + c1 (bys - by) + c2 (byss - bys)
  byb += fb[4] * (u - c1);
  ub += fb[4] * by;
  bxb -= fb[4] * v;
  vb_ -= fb[4] * bx;
  c1b += fb[4] * (bys - by);
  bysb += fb[4] * (c1 - c2);
  c2b += fb[4] * (byss - bys);
  byssb += fb[4] * c2;
  // f5 = bz u - bx w + c1 (bzs - bz) + c2 (bzss - bzs)
  bzb += fb[5] * (u - c1);
  ub += fb[5] * bz;
  bxb -= fb[5] * w;
  wb -= fb[5] * bx;
  c1b += fb[5] * (bzs - bz);
  bzsb += fb[5] * (c1 - c2);
  c2b += fb[5] * (bzss - bzs);
  bzssb += fb[5] * c2;
  // f6 = (e + pt) u - bx vb + c1 (es - e) + c2 (ess - es)
  eb += fb[6] * (u - c1);
  ptb += fb[6] * u;
  ub += fb[6] * (e + pt);
  bxb -= fb[6] * vb;
  vbb -= fb[6] * bx;
  c1b += fb[6] * (es - e);
  esb += fb[6] * (c1 - c2);
  c2b += fb[6] * (ess - es);
  essb += fb[6] * c2;
  // vb = u bx + v by + w bz (selected outer side)
  ub += vbb * bx;
  bxb += vbb * u;
  vb_ += vbb * by;
  byb += vbb * v;
  wb += vbb * bz;
  bzb += vbb * w;
  // ess = es + sq (vbs - vbss) sg
  esb += essb;
  sqb += essb * (vbs - vbss) * sg;
  vbsb += essb * sq * sg;
  vbssb -= essb * sq * sg;
  // c1, c2
  T SLb = 0, SRb = 0, SLsb = 0, SRsb = 0;
  if (!sup) {
    if (useL) SLb += c1b; else SRb += c1b;
  }
  if (inner) {
    if (useL) SLsb += c2b; else SRsb += c2b;
  }
  // route the selected-side adjoints to L or R
  SideBar<T> Lb, Rb;
  zero_bar(Lb);
  zero_bar(Rb);
#define MHD_ROUTE(field, val) \
  if (useL) Lb.field += (val);   \
  else Rb.field += (val)
  MHD_ROUTE(r, rb);
  MHD_ROUTE(u, ub);
  MHD_ROUTE(v, vb_);
  MHD_ROUTE(w, wb);
  MHD_ROUTE(by, byb);
  MHD_ROUTE(bz, bzb);
  MHD_ROUTE(e, eb);
  MHD_ROUTE(pt, ptb);
  MHD_ROUTE(rs, rsb);
  MHD_ROUTE(vs, vsb);
  MHD_ROUTE(ws, wsb);
  MHD_ROUTE(bys, bysb);
  MHD_ROUTE(bzs, bzsb);
  MHD_ROUTE(es, esb);
  MHD_ROUTE(vbs, vbsb);
#undef MHD_ROUTE
  if (useL) Lb.sq -= sqb; else Rb.sq += sqb;
  Lb.S += SLb;
  Rb.S += SRb;
  if (fan) {  // the double-star states (all their adjoints are zero otherwise)
    // vbss = SM bx + vss byss + wss bzss
    SMb += vbssb * bx;
    bxb += vbssb * SM;
    vssb += vbssb * byss;
    byssb += vbssb * vss;
    wssb += vbssb * bzss;
    bzssb += vbssb * wss;
    // byss = Nby isum, Nby = sqL bysR + sqR bysL + sqL sqR (vsR - vsL) sg
    T isumb = 0;
    {
      const T nb = byssb * isum;
      isumb += byssb * Nby;
      Lb.sq += nb * (R.bys + R.sq * (R.vs - L.vs) * sg);
      Rb.sq += nb * (L.bys + L.sq * (R.vs - L.vs) * sg);
      Rb.bys += nb * L.sq;
      Lb.bys += nb * R.sq;
      Rb.vs += nb * L.sq * R.sq * sg;
      Lb.vs -= nb * L.sq * R.sq * sg;
    }
    {
      const T nb = bzssb * isum;
      isumb += bzssb * Nbz;
      Lb.sq += nb * (R.bzs + R.sq * (R.ws - L.ws) * sg);
      Rb.sq += nb * (L.bzs + L.sq * (R.ws - L.ws) * sg);
      Rb.bzs += nb * L.sq;
      Lb.bzs += nb * R.sq;
      Rb.ws += nb * L.sq * R.sq * sg;
      Lb.ws -= nb * L.sq * R.sq * sg;
    }
    // vss = Nv isum, Nv = sqL vsL + sqR vsR + (bysR - bysL) sg
    {
      const T nb = vssb * isum;
      isumb += vssb * Nv;
      Lb.sq += nb * L.vs;
      Lb.vs += nb * L.sq;
      Rb.sq += nb * R.vs;
      Rb.vs += nb * R.sq;
      Rb.bys += nb * sg;
      Lb.bys -= nb * sg;
    }
    {
      const T nb = wssb * isum;
      isumb += wssb * Nw;
      Lb.sq += nb * L.ws;
      Lb.ws += nb * L.sq;
      Rb.sq += nb * R.ws;
      Rb.ws += nb * R.sq;
      Rb.bzs += nb * sg;
      Lb.bzs -= nb * sg;
    }
    // isum = 1 / (sqL + sqR)
    Lb.sq -= isumb * isum * isum;
    Rb.sq -= isumb * isum * isum;
    // SLs = SM - abx iqL; SRs = SM + abx iqR; iq = 1 / sq
    T abxb = 0;
    SMb += SLsb + SRsb;
    abxb -= SLsb * iqL;
    abxb += SRsb * iqR;
    Lb.sq += SLsb * abx * iqL * iqL;
    Rb.sq -= SRsb * abx * iqR * iqR;
    // abx = |bx| (derivative sign(bx), +1 at 0)
    bxb += abxb * sg;
    // sq = sqrt(rs)
    Lb.rs += Lb.sq * half * iqL;
    Rb.rs += Rb.sq * half * iqR;
  }
  // single-star states
  side_star_bar(L, Lb, bx, bx2, SM, pts, bxb, bx2b, SMb, ptsb);
  side_star_bar(R, Rb, bx, bx2, SM, pts, bxb, bx2b, SMb, ptsb);
  // pts = Np Di; SM = Ns Di; Di = 1 / (dR - dL)
  T Dib = 0;
  {
    const T nb = ptsb * Di;
    Dib += ptsb * Np;
    Rb.d += nb * (L.pt + L.d * (R.u - L.u));
    Lb.pt += nb * R.d;
    Lb.d += nb * (-R.pt + R.d * (R.u - L.u));
    Rb.pt -= nb * L.d;
    Rb.u += nb * L.d * R.d;
    Lb.u -= nb * L.d * R.d;
  }
  {
    const T nb = SMb * Di;
    Dib += SMb * Ns;
    Rb.d += nb * R.u;
    Rb.u += nb * R.d;
    Lb.d -= nb * L.u;
    Lb.u -= nb * L.d;
    Rb.pt -= nb;
    Lb.pt += nb;
  }
  {
    const T Db = -Dib * Di * Di;
    Rb.d += Db;
    Lb.d -= Db;
  }
  // d = (S - u) r
  Lb.S += Lb.d * L.r;
  Lb.u -= Lb.d * L.r;
  Lb.r += Lb.d * (L.S - L.u);
  Rb.S += Rb.d * R.r;
  Rb.u -= Rb.d * R.r;
  Rb.r += Rb.d * (R.S - R.u);
  // SL = min(uL, uR) - cmax; SR = max(uL, uR) + cmax
  T cmaxb = -Lb.S + Rb.S;
  if (uL_min) Lb.u += Lb.S; else Rb.u += Lb.S;
  if (uL_max) Lb.u += Rb.S; else Rb.u += Rb.S;
  if (cfL_max) Lb.cf += cmaxb; else Rb.cf += cmaxb;
  // outer states
  side_outer_bar(L, Lb, bx2, ph, bx2b);
  side_outer_bar(R, Rb, bx2, ph, bx2b);
  // bx2 = bx^2
  bxb += T(2) * bx * bx2b;
  // bx = (bnL + bnR)/2 - half_chi (psR - psL); psis = (psL + psR)/2 - ch (bnR - bnL)/2
  T bnLb = half * bxb + half * ch * psisb;
  T bnRb = half * bxb - half * ch * psisb;
  vlb[kPSI] = half_chi * bxb + half * psisb;
  vrb[kPSI] = -half_chi * bxb + half * psisb;
  vlb[kRHO] = Lb.r;
  vrb[kRHO] = Rb.r;
  vlb[kPRS] = Lb.p;
  vrb[kPRS] = Rb.p;
  // un-rotate velocity and field adjoints: component m gets rotated slot (m - dir) mod 3
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int j = (m - dir + 3) % 3;
    vlb[kVX + m] = j == 0 ? Lb.u : (j == 1 ? Lb.v : Lb.w);
    vrb[kVX + m] = j == 0 ? Rb.u : (j == 1 ? Rb.v : Rb.w);
    vlb[kBX + m] = j == 0 ? bnLb : (j == 1 ? Lb.by : Lb.bz);
    vrb[kBX + m] = j == 0 ? bnRb : (j == 1 ? Rb.by : Rb.bz);
  }
}

// Limited slope and its (piecewise constant) partial derivatives with
// respect to the one-sided differences dm, dp.
template <class T>
MHD_HD T limited_slope_d(T dm, T dp, int lim, T& ddm, T& ddp) {
  ddm = T(0);
  ddp = T(0);
  // the zero branch is decided exactly as in the forward limiter
  const T s = limited_slope(dm, dp, lim);
  if (s == T(0)) return s;
  const T am = tabs(dm), ap = tabs(dp);
  // minmod: the smaller magnitude (dm on ties, as min(a, b) picks a)
  const bool m_is_dm = !(ap < am);
  T gdm = m_is_dm ? T(1) : T(0), gdp = m_is_dm ? T(0) : T(1);
  if (lim == kLimMC) {
    const T two = T(2) * (m_is_dm ? am : ap);
    const T cen = T(0.5) * (am + ap);  // = |dm + dp| / 2 for equal signs
    if (cen < two) {  // central slope selected
      gdm = T(0.5);
      gdp = T(0.5);
    } else {
      gdm *= T(2);
      gdp *= T(2);
    }
  }
  // sign(s) = sign(dm) = sign(dp), so d s / d dm = gdm (signs cancel)
  ddm = gdm;
  ddp = gdp;
  return s;
}

// Derivative code of a limited slope, which is piecewise linear in the
// one-sided differences dm, dp: bits 0-1 the piece -- 0 zero slope, 1 the
// smaller-magnitude difference (minmod), 2 twice it (MC), 3 the central slope
// (dm + dp) / 2 (MC) -- and bit 2 set when the one-sided difference is dm.
// Three bits instead of two doubles keep the 18 derivatives of a face's two
// slopes in one register pair through the flux reverse.
MHD_HD void slope_code_d(unsigned code, double& ddm, double& ddp) {
  const unsigned piece = code & 3u;
  const bool m = (code >> 2) & 1u;
  const double f = piece == 1u ? 1.0 : 2.0;
  ddm = piece == 0u ? 0.0 : (piece == 3u ? 0.5 : (m ? f : 0.0));
  ddp = piece == 0u ? 0.0 : (piece == 3u ? 0.5 : (m ? 0.0 : f));
}

// FP64: the limited slope from the bit patterns, as limited_slope<double>,
// with its derivative code: the zero test, the minmod choice, the MC doubling
// / halving and the MC decision on the integer pipe; |dm| + |dp| is the only
// FP64 operation.
MHD_HD double limited_slope_c(double dm, double dp, int lim, unsigned& code) {
  code = 0u;
  const long long a = dbits(dm), b = dbits(dp);
  const long long mask = 0x7fffffffffffffffll;
  const long long am = a & mask, bm = b & mask;
  if (lim == kLimFlat || (a ^ b) < 0 || am == 0 || bm == 0) return 0.0;
  const bool m_is_dm = !(bm < am);  // the smaller magnitude; dm on ties
  long long mb = m_is_dm ? am : bm;
  unsigned piece = 1u;
  if (lim == kLimMC) {
    const long long two = twice_bits(mb);
    const long long cen = half_bits(dbits(bits2d(am) + bits2d(bm)));
    if (cen < two) {  // central slope selected
      mb = cen;
      piece = 3u;
    } else {
      mb = two;
      piece = 2u;
    }
  }
  code = piece | (m_is_dm ? 4u : 0u);
  return bits2d(mb | (a & ~mask));
}

template <>
MHD_HD double limited_slope_d<double>(double dm, double dp, int lim, double& ddm, double& ddp) {
  unsigned code;
  const double s = limited_slope_c(dm, dp, lim, code);
  slope_code_d(code, ddm, ddp);
  return s;
}

// Reverse of cons_to_prim (floors inactive: a floored value has zero
// derivative).  vb: adjoint of the primitives; ub: adjoint of the
// conservatives (overwritten).
template <class T>
MHD_HD void cons_to_prim_vjp(const T u[kNV], const T vb[kNV], const Phys<T>& ph,
                             T ub[kNV]) {
  const T rho = u[kRHO];
  const T ri = rcp(rho);
  const T vx = u[kVX] * ri, vy = u[kVY] * ri, vz = u[kVZ] * ri;
  const T kin = T(0.5) * (u[kVX] * vx + u[kVY] * vy + u[kVZ] * vz);
  const T b2 = u[kBX] * u[kBX] + u[kBY] * u[kBY] + u[kBZ] * u[kBZ];
  const T p = ph.gm1 * (u[kPRS] - kin - T(0.5) * b2);
  const bool rfl = lt_ieee(rho, ph.rho_floor);
  const bool pfl = lt_ieee(p, ph.p_floor);
  const T pb = pfl ? T(0) : vb[kPRS];
  // p = gm1 (E - |m|^2/(2 rho) - |B|^2/2)
  T rhob = rfl ? T(0) : vb[kRHO];
  rhob += pb * ph.gm1 * (vx * vx + vy * vy + vz * vz) * T(0.5);
  // v_k = m_k / rho
  rhob -= (vb[kVX] * vx + vb[kVY] * vy + vb[kVZ] * vz) * ri;
  ub[kRHO] = rfl ? T(0) : rhob;
  ub[kVX] = vb[kVX] * ri - pb * ph.gm1 * vx;
  ub[kVY] = vb[kVY] * ri - pb * ph.gm1 * vy;
  ub[kVZ] = vb[kVZ] * ri - pb * ph.gm1 * vz;
  ub[kBX] = vb[kBX] - pb * ph.gm1 * u[kBX];
  ub[kBY] = vb[kBY] - pb * ph.gm1 * u[kBY];
  ub[kBZ] = vb[kBZ] - pb * ph.gm1 * u[kBZ];
  ub[kPRS] = pb * ph.gm1;
  ub[kPSI] = vb[kPSI];
}

}  // namespace mhd
