// Discrete adjoint of one RK2 step (reverse-mode derivative of mhd_step with
// dt and c_h frozen).  With L the spatial operator of a stage (Section 3.2's
// five steps), the forward step is
//   U1 = U + dt L(U),  U' = (U + U1 + dt L(U1)) / 2,  U'' = D U'
// (D: the GLM damping of psi).  Its adjoint, for lam = dJ/dU'':
//   h  = D lam / 2
//   a1 = h + dt J_L(U1)^T h
//   dJ/dU = h + a1 + dt J_L(U)^T a1.
// J_L(W)^T x is evaluated per face: the face-flux adjoint
// g_f = (x_right - x_left) / dx_d, the GLM + HLLD vector-Jacobian product,
// the PLM slope derivatives (scattered with FP64 atomics onto the four cells
// of the face's stencil, through the same boundary remap as the forward),
// then per cell the cons->prim vector-Jacobian product.
#include <cstdio>
#include <cmath>

#include "mhd_adjoint.cuh"
#include "mhd_internal.h"

namespace mhd {

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct FaceArgs {
  int n[3];
  long long sy, sz, sv;
  int bc_lo[3], bc_hi[3];
  int limiter;
  double inv_dx;   // 1 / dx_d
  double ch, half_chi;
  Phys<double> ph;
};

// Primitives of every cell of W (the face kernels' stencils read them instead
// of converting each of their four cells again).
__global__ void adj_prims_kernel(const double* __restrict__ W, double* __restrict__ V,
                                 long long ncell, Phys<double> ph) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double u[kNV], v[kNV];
    unsigned flags = 0;
#pragma unroll
    for (int k = 0; k < kNV; ++k) u[k] = W[k * ncell + c];
    cons_to_prim(u, v, ph, flags);
#pragma unroll
    for (int k = 0; k < kNV; ++k) V[k * ncell + c] = v[k];
  }
}

// One thread per face of direction DIR; faces f = 0..n_d along d (face f
// separates cells f-1 and f).  Wp: the primitives of the stage input.
template <int DIR>
__global__ void __launch_bounds__(128) adj_faces_kernel(const double* __restrict__ Wp,
                                                        const double* __restrict__ x,
                                                        double* __restrict__ gV,
                                                        const FaceArgs a) {
  const int nd = a.n[DIR];
  const long long nfx = DIR == 0 ? (long long)(a.n[0] + 1) : a.n[0];
  const long long nfy = DIR == 1 ? (long long)(a.n[1] + 1) : a.n[1];
  const long long nfz = DIR == 2 ? (long long)(a.n[2] + 1) : a.n[2];
  const long long total = nfx * nfy * nfz;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int c[3];
    c[0] = (int)(id % nfx);
    c[1] = (int)((id / nfx) % nfy);
    c[2] = (int)(id / (nfx * nfy));
    const int f = c[DIR];
    // the four virtual cells f-2 .. f+1 along DIR, remapped into the grid
    long long off[4];
    for (int q = 0; q < 4; ++q) {
      int cc[3] = {c[0], c[1], c[2]};
      cc[DIR] = remap(f - 2 + q, nd, a.bc_lo[DIR], a.bc_hi[DIR]);
      off[q] = (long long)cc[2] * a.sz + (long long)cc[1] * a.sy + cc[0];
    }
    double V[4][kNV];
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int k = 0; k < kNV; ++k) V[q][k] = Wp[k * a.sv + off[q]];
    }
    // slopes of cells f-1 (a) and f (b) with their derivative codes (bits
    // 6k..6k+2: cell a, 6k+3..6k+5: cell b of variable k)
    double sa[kNV], sb[kNV];
    unsigned long long codes = 0ull;
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
      unsigned ca, cb;
      sa[k] = limited_slope_c(V[1][k] - V[0][k], V[2][k] - V[1][k], a.limiter, ca);
      sb[k] = limited_slope_c(V[2][k] - V[1][k], V[3][k] - V[2][k], a.limiter, cb);
      codes |= (unsigned long long)(ca | (cb << 3)) << (6 * k);
    }
    const bool oka = gt0(V[1][kRHO] - 0.5 * fabs(sa[kRHO])) &&
                     gt0(V[1][kPRS] - 0.5 * fabs(sa[kPRS]));
    const bool okb = gt0(V[2][kRHO] - 0.5 * fabs(sb[kRHO])) &&
                     gt0(V[2][kPRS] - 0.5 * fabs(sb[kPRS]));
    double vl[kNV], vr[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
      vl[k] = oka ? V[1][k] + 0.5 * sa[k] : V[1][k];
      vr[k] = okb ? V[2][k] - 0.5 * sb[k] : V[2][k];
    }
    // face-flux adjoint: L_{f-1} -= F_f / dx, L_f += F_f / dx
    double Fb[kNV];
    {
      int cr[3] = {c[0], c[1], c[2]}, cl[3] = {c[0], c[1], c[2]};
      cl[DIR] = f - 1;
      const bool has_r = f < nd, has_l = f >= 1;
      const long long orr = (long long)cr[2] * a.sz + (long long)cr[1] * a.sy + cr[0];
      const long long orl = (long long)cl[2] * a.sz + (long long)cl[1] * a.sy + cl[0];
#pragma unroll
      for (int k = 0; k < kNV; ++k) {
        const double xr = has_r ? x[k * a.sv + orr] : 0.0;
        const double xl = has_l ? x[k * a.sv + orl] : 0.0;
        Fb[k] = (xr - xl) * a.inv_dx;
      }
    }
    double vlb[kNV], vrb[kNV];
    glm_hlld_flux_vjp(vl, vr, DIR, a.ch, a.half_chi, a.ph, Fb, vlb, vrb);
    // PLM: vl = V_a + s_a/2, vr = V_b - s_b/2, s = lim(V_c - V_{c-1}, V_{c+1} - V_c)
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
      const unsigned ck = (unsigned)(codes >> (6 * k));
      double dma, dpa, dmb, dpb;
      slope_code_d(ck & 7u, dma, dpa);
      slope_code_d((ck >> 3) & 7u, dmb, dpb);
      const double ga = oka ? 0.5 * vlb[k] : 0.0;   // dJ/ds_a
      const double gb = okb ? -0.5 * vrb[k] : 0.0;  // dJ/ds_b
      const double g0 = -dma * ga;
      const double g1 = vlb[k] + (dma - dpa) * ga - dmb * gb;
      const double g2 = dpa * ga + vrb[k] + (dmb - dpb) * gb;
      const double g3 = dpb * gb;
      // (zero tests on the integer pipe)
      if (nonzero(g0)) atomicAdd(&gV[k * a.sv + off[0]], g0);
      if (nonzero(g1)) atomicAdd(&gV[k * a.sv + off[1]], g1);
      if (nonzero(g2)) atomicAdd(&gV[k * a.sv + off[2]], g2);
      if (nonzero(g3)) atomicAdd(&gV[k * a.sv + off[3]], g3);
    }
  }
}

// h = D lam / 2 (D scales psi by the damping factor).
__global__ void adj_init_kernel(const double* __restrict__ lam, double* __restrict__ h,
                                long long ncell, double damp) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
      const double s = k == kPSI ? 0.5 * damp : 0.5;
      h[k * ncell + c] = s * lam[k * ncell + c];
    }
  }
}

// out = b1 (+ b2) + dt * (dV/dW)^T gV  per cell.
__global__ void adj_cells_kernel(const double* __restrict__ W, const double* __restrict__ gV,
                                 const double* __restrict__ b1, const double* __restrict__ b2,
                                 double* __restrict__ out, long long ncell, double dt,
                                 Phys<double> ph) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double u[kNV], vb[kNV], ub[kNV];
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
      u[k] = W[k * ncell + c];
      vb[k] = gV[k * ncell + c];
    }
    cons_to_prim_vjp(u, vb, ph, ub);
#pragma unroll
    for (int k = 0; k < kNV; ++k) {
      double o = b1[k * ncell + c] + dt * ub[k];
      if (b2) o += b2[k * ncell + c];
      out[k * ncell + c] = o;
    }
  }
}

unsigned blocks_for(long long n, int threads, int nsm) {
  long long b = (n + threads - 1) / threads;
  const long long cap = (long long)nsm * 32;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

// Wp = prim(W); gV = 0; gV += J_V^T-scatter of every face;
// out = b1 (+ b2) + dt (dV/dW)^T gV
cudaError_t vjp_L(const Grid& g, const FaceArgs& fa0, const double* W, double* Wp,
                  const double* x, double* gV, const double* b1, const double* b2, double* out,
                  double dt, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(gV, 0, (size_t)9 * g.ncell * sizeof(double), s);
  if (e != cudaSuccess) return e;
  adj_prims_kernel<<<blocks_for(g.ncell, 256, g.nsm), 256, 0, s>>>(W, Wp, g.ncell,
                                                                     make_phys<double>(g));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int d = 0; d < 3; ++d) {
    if (g.n[d] <= 1) continue;
    FaceArgs fa = fa0;
    fa.inv_dx = 1.0 / g.dx[d];
    long long nf = g.ncell / g.n[d] * (g.n[d] + 1);
    const unsigned nb = blocks_for(nf, 128, g.nsm);
    if (d == 0) adj_faces_kernel<0><<<nb, 128, 0, s>>>(Wp, x, gV, fa);
    if (d == 1) adj_faces_kernel<1><<<nb, 128, 0, s>>>(Wp, x, gV, fa);
    if (d == 2) adj_faces_kernel<2><<<nb, 128, 0, s>>>(Wp, x, gV, fa);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  adj_cells_kernel<<<blocks_for(g.ncell, 256, g.nsm), 256, 0, s>>>(W, gV, b1, b2, out, g.ncell,
                                                                     dt, make_phys<double>(g));
  return cudaGetLastError();
}

}  // namespace

// Scratch: U1, h, a1, gV and the primitives of a stage input (9 ncell
// doubles each), the step scalars of the stage-1 recomputation and its
// (unused) reduction words.
size_t adjoint_scratch_bytes(const Grid& g) {
  const size_t state = a256((size_t)9 * g.ncell * sizeof(double));
  return 5 * state + a256(sizeof(StepScalars)) + 256;
}

int adjoint_step(const Grid& g, double dt, double ch, double glm_alpha, double dh_min,
                 const double* U_n, const double* U1_in, const double* lam_np1, double* lam_n,
                 void* scratch, size_t scratch_bytes, cudaStream_t s, char* err,
                 size_t errlen) {
  if (scratch_bytes < adjoint_scratch_bytes(g)) {
    snprintf(err, errlen, "adjoint scratch too small");
    return -2;
  }
  const size_t state = a256((size_t)9 * g.ncell * sizeof(double));
  char* p = static_cast<char*>(scratch);
  double* U1s = reinterpret_cast<double*>(p);
  double* h = reinterpret_cast<double*>(p + state);
  double* a1 = reinterpret_cast<double*>(p + 2 * state);
  double* gV = reinterpret_cast<double*>(p + 3 * state);
  double* Vp = reinterpret_cast<double*>(p + 4 * state);
  StepScalars* sc = reinterpret_cast<StepScalars*>(p + 5 * state);
  unsigned long long* words =
      reinterpret_cast<unsigned long long*>(p + 5 * state + a256(sizeof(StepScalars)));

  StepScalars hs{};
  hs.dt = dt;
  hs.ch = ch;
  for (int d = 0; d < 3; ++d) hs.dtdx[d] = g.n[d] > 1 ? dt / g.dx[d] : 0.0;
  hs.damp = std::exp(-glm_alpha * ch * dt / dh_min);
  cudaError_t e = cudaMemcpyAsync(sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(words, 0, 256, s);
  // forward stage 1: recomputed from U_n unless the caller kept it (U1_in)
  const double* U1 = U1_in ? U1_in : U1s;
  if (e == cudaSuccess && !U1_in)
    e = launch_stage<double>(g, 1, U_n, nullptr, U1s, sc, words, words + 1, s);
  if (e == cudaSuccess)
    adj_init_kernel<<<blocks_for(g.ncell, 256, g.nsm), 256, 0, s>>>(lam_np1, h, g.ncell,
                                                                    hs.damp);
  if (e == cudaSuccess) e = cudaGetLastError();
  FaceArgs fa{};
  for (int d = 0; d < 3; ++d) {
    fa.n[d] = g.n[d];
    fa.bc_lo[d] = g.bc_lo[d];
    fa.bc_hi[d] = g.bc_hi[d];
  }
  fa.sy = g.n[0];
  fa.sz = (long long)g.n[0] * g.n[1];
  fa.sv = g.ncell;
  fa.limiter = g.limiter;
  fa.ch = ch;
  fa.half_chi = 0.5 / ch;
  fa.ph = make_phys<double>(g);
  // a1 = h + dt J_L(U1)^T h
  if (e == cudaSuccess) e = vjp_L(g, fa, U1, Vp, h, gV, h, nullptr, a1, dt, s);
  // lam_n = h + a1 + dt J_L(U_n)^T a1
  if (e == cudaSuccess) e = vjp_L(g, fa, U_n, Vp, a1, gV, h, a1, lam_n, dt, s);
  if (e != cudaSuccess) {
    snprintf(err, errlen, "adjoint launch failed: %s", cudaGetErrorString(e));
    return -3;
  }
  return 0;
}

}  // namespace mhd
