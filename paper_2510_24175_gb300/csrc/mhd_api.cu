// C ABI of the GLM-MHD hot path (declared in include/mhd.h).  Host code only:
// validates arguments, carves the caller's workspace, and enqueues the
// kernels of mhd_aux.cu / mhd_stage_*.cu / mhd_adjoint.cu on the context's
// stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <functional>
#include <new>
#include <queue>
#include <vector>

#include "mhd_ctx.h"

using mhd::Scalars;
using mhd::align256;
using mhd::kSumBlocks;

static cudaEvent_t prof_event(mhd_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Brackets one launch with events when profiling is on.
struct ProfScope {
  mhd_ctx* c;
  cudaEvent_t a = nullptr, b = nullptr;
  int kind;
  ProfScope(mhd_ctx* ctx, int k) : c(ctx), kind(k) {
    if (!c->prof_on) return;
    a = prof_event(c);
    b = prof_event(c);
    if (a) cudaEventRecord(a, c->stream);
  }
  ~ProfScope() {
    if (!c->prof_on || !a || !b) return;
    cudaEventRecord(b, c->stream);
    c->prof_recs.push_back({a, b, kind});
  }
};

static int fail(mhd_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CK(ctx, call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail((ctx), MHD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

namespace mhd {
static thread_local char g_free_err[256] = "no error";

int free_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_free_err, sizeof(g_free_err), fmt, ap);
  va_end(ap);
  return code;
}
}  // namespace mhd

static int validate(const mhd_config* c, char* msg, size_t len) {
  if (!c) {
    snprintf(msg, len, "null config");
    return MHD_ERR_INVALID;
  }
  for (int d = 0; d < 3; ++d) {
    if (c->n[d] < 1) {
      snprintf(msg, len, "n[%d] = %d < 1", d, c->n[d]);
      return MHD_ERR_INVALID;
    }
    if (!(c->xmax[d] > c->xmin[d])) {
      snprintf(msg, len, "empty domain in dimension %d", d);
      return MHD_ERR_INVALID;
    }
    if (!(c->dx[d] >= 0.0) || !(c->dx[d] < INFINITY)) {
      snprintf(msg, len, "bad cell size dx[%d] (0: derived from the domain, else > 0)", d);
      return MHD_ERR_INVALID;
    }
  }
  if (c->n[0] < 2) {
    snprintf(msg, len, "x must be active (nx >= 2)");
    return MHD_ERR_INVALID;
  }
  if (c->n[2] > 1 && c->n[1] < 2) {
    snprintf(msg, len, "inactive dimensions must be trailing (ny = 1 needs nz = 1)");
    return MHD_ERR_INVALID;
  }
  if ((long long)c->n[0] * c->n[1] * c->n[2] > (1ll << 34)) {
    snprintf(msg, len, "grid too large");
    return MHD_ERR_INVALID;
  }
  if (!(c->gamma > 1.0) || !(c->cfl > 0.0 && c->cfl <= 1.0) || !(c->glm_alpha >= 0.0) ||
      !(c->rho_floor >= 0.0) || !(c->p_floor >= 0.0) || !(c->t_end >= 0.0)) {
    snprintf(msg, len, "bad physics constant (gamma > 1, 0 < cfl <= 1, alpha/floors >= 0)");
    return MHD_ERR_INVALID;
  }
  if (c->limiter < MHD_LIM_FLAT || c->limiter > MHD_LIM_WENOZ) {
    snprintf(msg, len, "bad limiter %d", c->limiter);
    return MHD_ERR_INVALID;
  }
  if (c->limiter == MHD_LIM_WENOZ)
    for (int d = 0; d < 3; ++d)
      if (c->n[d] == 2) {
        snprintf(msg, len, "WENO-Z needs active dimensions of at least 3 cells");
        return MHD_ERR_INVALID;
      }
  bool halo = false;
  for (int d = 0; d < 3; ++d) {
    const int lo = c->bc[2 * d], hi = c->bc[2 * d + 1];
    auto ok = [](int b) { return b == MHD_BC_PERIODIC || b == MHD_BC_OUTFLOW || b == MHD_BC_HALO; };
    if (!ok(lo) || !ok(hi) || ((lo == MHD_BC_PERIODIC) != (hi == MHD_BC_PERIODIC))) {
      snprintf(msg, len, "bad boundary conditions in dimension %d", d);
      return MHD_ERR_INVALID;
    }
    halo = halo || lo == MHD_BC_HALO || hi == MHD_BC_HALO;
  }
  if (halo) {
    const int gw = c->limiter == MHD_LIM_WENOZ ? 3 : 2;
    for (int d = 0; d < 3; ++d)
      if (c->n[d] < gw) {
        snprintf(msg, len, "halo faces need three active dimensions of at least %d cells", gw);
        return MHD_ERR_INVALID;
      }
    if (c->divb != MHD_DIVB_GLM || (c->flags & MHD_FLAG_ADJOINT)) {
      snprintf(msg, len, "halo faces are for GLM contexts without the adjoint");
      return MHD_ERR_INVALID;
    }
  }
  if (c->precision != MHD_FP64 && c->precision != MHD_FP32) {
    snprintf(msg, len, "bad precision %d", c->precision);
    return MHD_ERR_INVALID;
  }
  if (c->rk_order != 2 && c->rk_order != 3) {
    snprintf(msg, len, "rk_order must be 2 or 3");
    return MHD_ERR_INVALID;
  }
  if ((c->flags & MHD_FLAG_ADJOINT) &&
      (c->precision != MHD_FP64 || c->rk_order != 2 || c->limiter == MHD_LIM_WENOZ ||
       c->divb != MHD_DIVB_GLM)) {
    snprintf(msg, len, "the adjoint needs MHD_FP64, RK2, a PLM limiter and GLM");
    return MHD_ERR_INVALID;
  }
  if (c->divb != MHD_DIVB_GLM && c->divb != MHD_DIVB_CT) {
    snprintf(msg, len, "bad divb %d", c->divb);
    return MHD_ERR_INVALID;
  }
  if (c->divb == MHD_DIVB_CT) {
    for (int d = 0; d < 3; ++d)
      if (c->n[d] < 2 || c->bc[2 * d] != MHD_BC_PERIODIC) {
        snprintf(msg, len, "constrained transport needs three active periodic dimensions");
        return MHD_ERR_INVALID;
      }
  }
  return MHD_OK;
}

// Adjoint scratch bytes (mhd_adjoint.cu).
namespace mhd {
size_t adjoint_scratch_bytes(const Grid& g);
int adjoint_step(const Grid& g, double dt, double ch, double glm_alpha, double dh_min,
                 const double* U_n, const double* U1_in, const double* lam_np1, double* lam_n,
                 void* scratch, size_t scratch_bytes, cudaStream_t stream, char* err,
                 size_t errlen);
}  // namespace mhd

static void fill_grid(const mhd_config* c, mhd::Grid* g) {
  memset(g, 0, sizeof(*g));
  g->ndim = 0;
  g->ncell = 1;
  for (int d = 0; d < 3; ++d) {
    g->n[d] = c->n[d];
    g->ncell *= c->n[d];
    g->dx[d] = c->dx[d] > 0.0 ? c->dx[d] : (c->xmax[d] - c->xmin[d]) / c->n[d];
    g->bc_lo[d] = c->bc[2 * d];
    g->bc_hi[d] = c->bc[2 * d + 1];
    if (c->n[d] > 1) g->ndim++;
  }
  g->limiter = c->limiter;
  g->gamma = c->gamma;
  g->rho_floor = c->rho_floor;
  g->p_floor = c->p_floor;
}

// Duration, in plane iterations, of one stage launch of `cols` column tiles
// over nz planes in z chunks of tz planes, on `slots` CTA slots: the CTAs
// start in launch order (the full chunks of every column tile, then the
// last, possibly shorter, chunk of every column tile), each on the slot that
// frees first, and a CTA takes its planes plus one for its warm-up planes.
static double launch_span(long long cols, int nz, int tz, long long slots) {
  const long long chunks = (nz + tz - 1) / tz;
  const double a = tz + 1.0, b = (double)(nz - (chunks - 1) * tz) + 1.0;
  const long long n1 = cols * (chunks - 1);
  const long long q = n1 / slots, r = n1 % slots;  // full chunks per slot
  std::priority_queue<double, std::vector<double>, std::greater<double>> freed;
  double span = 0.0;
  for (long long s = 0; s < slots; ++s) {
    const double t = (s < r ? q + 1 : q) * a;
    freed.push(t);
    span = std::max(span, t);
  }
  for (long long c = 0; c < cols; ++c) {
    const double t = freed.top() + b;
    freed.pop();
    freed.push(t);
    span = std::max(span, t);
  }
  return span;
}

// z planes per CTA: the candidate depth with the shortest launch_span, the
// deeper one on a tie (fewer warm-ups).  (A depth that leaves a shorter last
// chunk can win: those short CTAs run last and fill the slots that the last
// wave of full chunks leaves idle.)
static int plan_tz(long long cols, int nz, long long slots, double* span_out) {
  int best = nz;
  double best_span = 1e300;
  const int cands[] = {256, 192, 128, 96, 80, 64, 56, 48, 40, 32, 24, 20, 16, 12, 8, 4};
  for (int tz : cands) {
    if (tz > nz && tz != 4) continue;
    const double span = launch_span(cols, nz, tz, slots);
    if (span < best_span) {
      best_span = span;
      best = tz;
    }
  }
  if (span_out) *span_out = best_span;
  return best;
}

static int choose_tz(const mhd::Grid& g, int ctas_per_sm, int ty) {
  if (g.ndim < 3) return 1;
  const long long cols = (long long)((g.n[0] + 31) / 32) * ((g.n[1] + ty - 1) / ty);
  return plan_tz(cols, g.n[2], (long long)g.nsm * ctas_per_sm, nullptr);
}

int mhd_plan_z_chunks(const int n[3], int ty, int nsm, int ctas_per_sm, int* tz,
                      double* span) {
  if (!n || !tz || n[0] < 1 || n[1] < 1 || n[2] < 1 || ty < 1 || nsm < 1 || ctas_per_sm < 1)
    return mhd::free_fail(MHD_ERR_INVALID, "mhd_plan_z_chunks: bad argument");
  const long long cols = (long long)((n[0] + 31) / 32) * ((n[1] + ty - 1) / ty);
  const long long slots = (long long)nsm * ctas_per_sm;
  if (n[0] <= 1 || n[1] <= 1 || n[2] <= 1) {  // not 3-D: one plane per CTA
    *tz = 1;
    if (span) *span = launch_span(cols, 1, 1, slots);
    return MHD_OK;
  }
  *tz = plan_tz(cols, n[2], slots, span);
  return MHD_OK;
}

// The face field that belongs to state buffer U (constrained transport).
static void* faces_of(mhd_ctx* c, void* U) {
  if (U == c->Ua) return c->fa;
  if (U == c->Ub) return c->fb;
  if (U == c->Uc) return c->fc;
  return nullptr;
}

// One constrained-transport stage: the fused stage kernel (rho, m, E and the
// face / cell electric fields), then edge fields, the face update with the
// Runge-Kutta combination, and the cell-centred B (+ the wave-speed
// reduction after the last stage).
template <class T>
static int ct_stage(mhd_ctx* c, int kind, int cls, void* win, void* un, void* out, double an,
                    double aw) {
  const T* bw[3];
  const T* fw = static_cast<const T*>(faces_of(c, win));
  for (int d = 0; d < 3; ++d) bw[d] = fw + (size_t)d * c->grid.ncell;
  const T* fn = un ? static_cast<const T*>(faces_of(c, un)) : nullptr;
  T* fo = static_cast<T*>(faces_of(c, out));
  T* ctf = static_cast<T*>(c->ctf);
  T* edge = static_cast<T*>(c->edge);
  {
    ProfScope ps(c, cls);
    CK(c, mhd::launch_stage<T>(c->grid, kind, static_cast<const T*>(win),
                               static_cast<const T*>(un), static_cast<T*>(out), &c->scal->sc,
                               &c->scal->lam_bits, c->scal->floor_cnt, c->stream, an, aw, bw,
                               ctf));
  }
  ProfScope ps(c, 5);
  CK(c, mhd::launch_ct_edges<T>(c->grid, ctf, edge, c->stream));
  CK(c, mhd::launch_ct_faces<T>(c->grid, kind == 1, edge, fw, fn, fo, &c->scal->sc, an, aw,
                                c->stream));
  CK(c, mhd::launch_ct_cells<T>(c->grid, kind == 2, fo, static_cast<T*>(out),
                                &c->scal->lam_bits, c->stream));
  return MHD_OK;
}

extern "C" {

int mhd_config_default(mhd_config* cfg) {
  if (!cfg) return MHD_ERR_INVALID;
  memset(cfg, 0, sizeof(*cfg));
  for (int d = 0; d < 3; ++d) {
    cfg->n[d] = 1;
    cfg->xmin[d] = 0.0;
    cfg->xmax[d] = 1.0;
  }
  cfg->gamma = 5.0 / 3.0;
  cfg->cfl = 0.8;
  cfg->glm_alpha = 0.1;
  cfg->rho_floor = 1e-12;
  cfg->p_floor = 1e-12;
  cfg->t_end = 0.0;
  cfg->limiter = MHD_LIM_MC;
  for (int s = 0; s < 6; ++s) cfg->bc[s] = MHD_BC_PERIODIC;
  cfg->precision = MHD_FP64;
  cfg->flags = 0;
  cfg->rk_order = 2;
  cfg->divb = MHD_DIVB_GLM;
  return MHD_OK;
}

int mhd_workspace_bytes(const mhd_config* cfg, size_t* bytes) {
  char msg[256];
  int rc = validate(cfg, msg, sizeof(msg));
  if (rc != MHD_OK) return mhd::free_fail(rc, "invalid config: %s", msg);
  if (!bytes) return mhd::free_fail(MHD_ERR_INVALID, "mhd_workspace_bytes: null bytes");
  mhd::Grid g;
  fill_grid(cfg, &g);
  const size_t es = cfg->precision == MHD_FP64 ? 8 : 4;
  const size_t state = align256((size_t)9 * g.ncell * es);
  const int nstate = cfg->rk_order == 3 ? 3 : 2;
  size_t total = nstate * state + align256(sizeof(Scalars)) +
                 align256(kSumBlocks * 8 * sizeof(double));
  if (cfg->divb == MHD_DIVB_CT)
    total += nstate * align256((size_t)3 * g.ncell * es) +
             align256((size_t)mhd::kCtPlanes * g.ncell * es) + align256((size_t)3 * g.ncell * es);
  if (cfg->flags & MHD_FLAG_ADJOINT) total += align256(mhd::adjoint_scratch_bytes(g));
  *bytes = total;
  return MHD_OK;
}

int mhd_create(const mhd_config* cfg, void* d_workspace, size_t bytes, void* stream,
               mhd_ctx** out) {
  if (!out) return mhd::free_fail(MHD_ERR_INVALID, "mhd_create: null out");
  *out = nullptr;
  char msg[256] = "";
  int rc = validate(cfg, msg, sizeof(msg));
  if (rc != MHD_OK) return mhd::free_fail(rc, "mhd_create: invalid config: %s", msg);
  size_t need = 0;
  mhd_workspace_bytes(cfg, &need);
  if (!d_workspace || bytes < need || ((uintptr_t)d_workspace & 255))
    return mhd::free_fail(MHD_ERR_NOMEM,
                          "mhd_create: workspace %p of %zu bytes (need %zu, 256-byte aligned)",
                          d_workspace, bytes, need);
  mhd_ctx* c = new (std::nothrow) mhd_ctx();
  if (!c) return mhd::free_fail(MHD_ERR_NOMEM, "mhd_create: host allocation failed");
  c->cfg = *cfg;
  fill_grid(cfg, &c->grid);
  int dev = 0;
  cudaGetDevice(&dev);
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      nsm <= 0) {
    delete c;
    return mhd::free_fail(MHD_ERR_CUDA, "mhd_create: no usable CUDA device");
  }
  c->grid.nsm = nsm;
  c->esize = cfg->precision == MHD_FP64 ? 8 : 4;
  c->state_bytes = (size_t)9 * c->grid.ncell * c->esize;
  c->ws = static_cast<char*>(d_workspace);
  c->ws_bytes = bytes;
  size_t off = 0;
  c->Ua = c->ws + off;
  off += align256(c->state_bytes);
  c->Ub = c->ws + off;
  off += align256(c->state_bytes);
  c->Uc = nullptr;
  if (cfg->rk_order == 3) {
    c->Uc = c->ws + off;
    off += align256(c->state_bytes);
  }
  c->scal = reinterpret_cast<Scalars*>(c->ws + off);
  off += align256(sizeof(Scalars));
  c->partials = reinterpret_cast<double*>(c->ws + off);
  off += align256(kSumBlocks * 8 * sizeof(double));
  c->fa = c->fb = c->fc = c->ctf = c->edge = nullptr;
  c->faces_set = false;
  if (cfg->divb == MHD_DIVB_CT) {
    const size_t fbytes = align256((size_t)3 * c->grid.ncell * c->esize);
    c->fa = c->ws + off;
    off += fbytes;
    c->fb = c->ws + off;
    off += fbytes;
    if (cfg->rk_order == 3) {
      c->fc = c->ws + off;
      off += fbytes;
    }
    c->ctf = c->ws + off;
    off += align256((size_t)mhd::kCtPlanes * c->grid.ncell * c->esize);
    c->edge = c->ws + off;
    off += fbytes;
  }
  c->adj = nullptr;
  c->adj_bytes = 0;
  if (cfg->flags & MHD_FLAG_ADJOINT) {
    c->adj = c->ws + off;
    c->adj_bytes = mhd::adjoint_scratch_bytes(c->grid);
    off += align256(c->adj_bytes);
  }
  c->stream = static_cast<cudaStream_t>(stream);
  c->inv_dx_sum = 0.0;
  c->dh_min = 1e300;
  for (int d = 0; d < 3; ++d)
    if (c->grid.n[d] > 1) {
      c->inv_dx_sum += 1.0 / c->grid.dx[d];
      c->dh_min = fmin(c->dh_min, c->grid.dx[d]);
    }
  size_t smem;
  int threads, ty;
  if (c->esize == 8)
    mhd::stage_shape<double>(c->grid, &smem, &threads, &ty);
  else
    mhd::stage_shape<float>(c->grid, &smem, &threads, &ty);
  const int per_sm = (int)(228 * 1024 / (smem + 1024));
  c->grid.tz = choose_tz(c->grid, per_sm < 1 ? 1 : per_sm, ty);
  {
    mhd::Grid gh = c->grid;  // the half-depth grid of mhd_step_host's last stage
    gh.n[2] = (gh.n[2] + 1) / 2;
    c->tz_half = choose_tz(gh, per_sm < 1 ? 1 : per_sm, ty);
  }
  {
    // kernel attributes now, so that no later launch (a captured one in
    // particular) needs the driver call
    const bool ct = cfg->divb == MHD_DIVB_CT;
    c->has_halo = false;
    for (int s = 0; s < 6; ++s) c->has_halo = c->has_halo || cfg->bc[s] == MHD_BC_HALO;
    cudaError_t pe = c->esize == 8 ? mhd::prepare_stage_kernels<double>(c->grid, ct)
                                   : mhd::prepare_stage_kernels<float>(c->grid, ct);
    if (pe == cudaSuccess && c->has_halo)
      pe = c->esize == 8 ? mhd::prepare_stage_kernels_halo<double>(c->grid)
                         : mhd::prepare_stage_kernels_halo<float>(c->grid);
    if (pe != cudaSuccess) {
      delete c;
      return mhd::free_fail(MHD_ERR_CUDA, "mhd_create: kernel attributes: %s",
                            cudaGetErrorString(pe));
    }
  }
  c->xfer_ready = false;
  c->xfer = nullptr;
  c->cap = nullptr;
  c->gexec = nullptr;
  c->graph_steps = 0;
  c->stage1_valid = false;
  c->have_state = false;
  c->lam_valid = false;
  c->step_open = false;
  c->stage_next = 0;
  snprintf(c->err, sizeof(c->err), "no error");
  cudaError_t e = cudaMemsetAsync(c->scal, 0, sizeof(Scalars), c->stream);
  if (e != cudaSuccess) {
    delete c;
    return mhd::free_fail(MHD_ERR_CUDA, "mhd_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return MHD_OK;
}

int mhd_set_stream(mhd_ctx* c, void* stream) {
  if (!c) return MHD_ERR_INVALID;
  c->stream = static_cast<cudaStream_t>(stream);
  return MHD_OK;
}

int mhd_set_state(mhd_ctx* c, const double* U, int where, int kind) {
  if (!c) return MHD_ERR_INVALID;
  if (!U || (where != MHD_HOST && where != MHD_DEVICE) ||
      (kind != MHD_CONS && kind != MHD_PRIM))
    return fail(c, MHD_ERR_INVALID, "mhd_set_state: bad argument");
  const long long n = 9 * c->grid.ncell;
  const cudaMemcpyKind mk = where == MHD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (c->esize == 8) {
    double* A = static_cast<double*>(c->Ua);
    if (kind == MHD_CONS) {
      CK(c, cudaMemcpyAsync(A, U, n * 8, mk, c->stream));
    } else {
      const double* src = U;
      if (where == MHD_HOST) {
        CK(c, cudaMemcpyAsync(c->Ub, U, n * 8, mk, c->stream));
        src = static_cast<const double*>(c->Ub);
      }
      CK(c, mhd::launch_prim_to_cons<double>(c->grid, src, A, c->stream));
    }
  } else {
    float* A = static_cast<float*>(c->Ua);
    if (where == MHD_DEVICE) {
      if (kind == MHD_CONS)
        CK(c, mhd::launch_f64_to_f32(U, A, n, c->stream));
      else
        CK(c, mhd::launch_prim_to_cons<float>(c->grid, U, A, c->stream));
    } else {
      // stage FP64 host data through Ub (half the FP64 bytes) in chunks
      const long long chunk = (long long)(c->state_bytes / 8);
      double* B = static_cast<double*>(c->Ub);
      for (long long o = 0; o < n; o += chunk) {
        const long long m = n - o < chunk ? n - o : chunk;
        CK(c, cudaMemcpyAsync(B, U + o, m * 8, cudaMemcpyHostToDevice, c->stream));
        CK(c, mhd::launch_f64_to_f32(B, A + o, m, c->stream));
      }
      if (kind == MHD_PRIM) CK(c, mhd::launch_prim_to_cons_inplace<float>(c->grid, A, c->stream));
    }
  }
  CK(c, cudaMemsetAsync(c->scal, 0, sizeof(Scalars), c->stream));
  c->have_state = true;
  c->lam_valid = false;
  c->faces_set = false;
  c->stage1_valid = false;
  c->step_open = false;
  return MHD_OK;
}

int mhd_set_face_field(mhd_ctx* c, const double* b, int where) {
  if (!c) return MHD_ERR_INVALID;
  if (c->cfg.divb != MHD_DIVB_CT)
    return fail(c, MHD_ERR_STATE, "mhd_set_face_field needs MHD_DIVB_CT");
  if (!b || (where != MHD_HOST && where != MHD_DEVICE))
    return fail(c, MHD_ERR_INVALID, "mhd_set_face_field: bad argument");
  if (!c->have_state) return fail(c, MHD_ERR_STATE, "mhd_set_face_field before mhd_set_state");
  c->stage1_valid = false;
  const long long n = 3 * c->grid.ncell;
  const cudaMemcpyKind mk = where == MHD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (c->esize == 8) {
    CK(c, cudaMemcpyAsync(c->fa, b, n * 8, mk, c->stream));
    CK(c, mhd::launch_ct_set_cells<double>(c->grid, static_cast<const double*>(c->fa),
                                           static_cast<double*>(c->Ua), c->stream));
  } else {
    const double* src = b;
    if (where == MHD_HOST) {  // Ub holds 9 FP32 planes = 4.5 FP64 planes >= 3
      CK(c, cudaMemcpyAsync(c->Ub, b, n * 8, mk, c->stream));
      src = static_cast<const double*>(c->Ub);
    }
    CK(c, mhd::launch_f64_to_f32(src, static_cast<float*>(c->fa), n, c->stream));
    CK(c, mhd::launch_ct_set_cells<float>(c->grid, static_cast<const float*>(c->fa),
                                          static_cast<float*>(c->Ua), c->stream));
  }
  c->faces_set = true;
  c->lam_valid = false;
  return MHD_OK;
}

int mhd_get_face_field(mhd_ctx* c, double* b, int where) {
  if (!c) return MHD_ERR_INVALID;
  if (c->cfg.divb != MHD_DIVB_CT)
    return fail(c, MHD_ERR_STATE, "mhd_get_face_field needs MHD_DIVB_CT");
  if (!b || (where != MHD_HOST && where != MHD_DEVICE))
    return fail(c, MHD_ERR_INVALID, "mhd_get_face_field: bad argument");
  if (!c->faces_set) return fail(c, MHD_ERR_STATE, "no face field set");
  const long long n = 3 * c->grid.ncell;
  if (c->esize == 8) {
    CK(c, cudaMemcpyAsync(b, c->fa, n * 8,
                          where == MHD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          c->stream));
  } else if (where == MHD_DEVICE) {
    CK(c, mhd::launch_f32_to_f64(static_cast<const float*>(c->fa), b, n, c->stream));
  } else {
    double* B = static_cast<double*>(c->Ub);
    CK(c, mhd::launch_f32_to_f64(static_cast<const float*>(c->fa), B, n, c->stream));
    CK(c, cudaMemcpyAsync(b, B, n * 8, cudaMemcpyDeviceToHost, c->stream));
  }
  if (where == MHD_HOST) CK(c, cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

int mhd_divb_max(mhd_ctx* c, double* out) {
  if (!c || !out) return MHD_ERR_INVALID;
  if (c->cfg.divb != MHD_DIVB_CT) return fail(c, MHD_ERR_STATE, "mhd_divb_max needs MHD_DIVB_CT");
  if (!c->faces_set) return fail(c, MHD_ERR_STATE, "no face field set");
  CK(c, cudaMemsetAsync(&c->scal->aux_bits, 0, sizeof(unsigned long long), c->stream));
  if (c->esize == 8)
    CK(c, mhd::launch_ct_divb<double>(c->grid, static_cast<const double*>(c->fa),
                                      &c->scal->aux_bits, c->stream));
  else
    CK(c, mhd::launch_ct_divb<float>(c->grid, static_cast<const float*>(c->fa),
                                     &c->scal->aux_bits, c->stream));
  unsigned long long bits = 0;
  CK(c, cudaMemcpyAsync(&bits, &c->scal->aux_bits, sizeof(bits), cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  memcpy(out, &bits, sizeof(*out));
  return MHD_OK;
}

int mhd_get_state(mhd_ctx* c, double* U, int where, int kind) {
  if (!c) return MHD_ERR_INVALID;
  if (!U || (where != MHD_HOST && where != MHD_DEVICE) ||
      (kind != MHD_CONS && kind != MHD_PRIM) || (kind == MHD_PRIM && where != MHD_DEVICE))
    return fail(c, MHD_ERR_INVALID, "mhd_get_state: bad argument");
  if (!c->have_state) return fail(c, MHD_ERR_STATE, "mhd_get_state before mhd_set_state");
  const long long n = 9 * c->grid.ncell;
  if (kind == MHD_PRIM) {
    if (c->esize == 8)
      CK(c, mhd::launch_cons_to_prim<double>(c->grid, static_cast<const double*>(c->Ua), U,
                                             c->stream));
    else
      CK(c, mhd::launch_cons_to_prim<float>(c->grid, static_cast<const float*>(c->Ua), U,
                                            c->stream));
    return MHD_OK;
  }
  if (c->esize == 8) {
    CK(c, cudaMemcpyAsync(U, c->Ua, n * 8,
                          where == MHD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          c->stream));
  } else if (where == MHD_DEVICE) {
    CK(c, mhd::launch_f32_to_f64(static_cast<const float*>(c->Ua), U, n, c->stream));
  } else {
    const long long chunk = (long long)(c->state_bytes / 8);
    double* B = static_cast<double*>(c->Ub);
    const float* A = static_cast<const float*>(c->Ua);
    for (long long o = 0; o < n; o += chunk) {
      const long long m = n - o < chunk ? n - o : chunk;
      CK(c, mhd::launch_f32_to_f64(A + o, B, m, c->stream));
      CK(c, cudaMemcpyAsync(U + o, B, m * 8, cudaMemcpyDeviceToHost, c->stream));
    }
  }
  if (where == MHD_HOST) CK(c, cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

static int ensure_lambda(mhd_ctx* c) {
  if (c->lam_valid) return MHD_OK;
  ProfScope ps(c, 3);
  if (c->esize == 8)
    CK(c, mhd::launch_max_speed<double>(c->grid, static_cast<const double*>(c->Ua),
                                        &c->scal->lam_bits, &c->scal->est_bits, c->stream));
  else
    CK(c, mhd::launch_max_speed<float>(c->grid, static_cast<const float*>(c->Ua),
                                       &c->scal->lam_bits, nullptr, c->stream));
  c->lam_valid = true;
  return MHD_OK;
}

int mhd_dt(mhd_ctx* c, double* dt, double* ch) {
  if (!c) return MHD_ERR_INVALID;
  if (!c->have_state) return fail(c, MHD_ERR_STATE, "mhd_dt before mhd_set_state");
  int rc = ensure_lambda(c);
  if (rc != MHD_OK) return rc;
  unsigned long long bits = 0;
  CK(c, cudaMemcpyAsync(&bits, &c->scal->lam_bits, sizeof(bits), cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  double lam;
  memcpy(&lam, &bits, sizeof(lam));
  if (!(lam > 0.0) || !std::isfinite(lam))
    return fail(c, MHD_ERR_NONFINITE, "max wave speed is %g", lam);
  if (ch) *ch = lam;
  if (dt) *dt = c->cfg.cfl / (lam * c->inv_dx_sum);
  return MHD_OK;
}

// Host output of mhd_step_host: the last stage runs as two launches over the
// z planes [0, zh) and [zh, nz); each half of U^{n+1} is copied to U on the
// transfer stream as soon as its launch is done.
struct HostOut {
  double* U;
  int zh;
};

static int copy_planes(mhd_ctx* c, double* dst, const double* src, int z0, int z1,
                       cudaMemcpyKind kind) {
  const long long plane = (long long)c->grid.n[0] * c->grid.n[1];
  const long long n = c->grid.ncell;
  for (int k = 0; k < 9; ++k)
    CK(c, cudaMemcpyAsync(dst + k * n + z0 * plane, src + k * n + z0 * plane,
                          (size_t)(z1 - z0) * plane * sizeof(double), kind, c->xfer));
  return MHD_OK;
}

static int step_impl(mhd_ctx* c, double dt, double ch, const HostOut* ho);

// The step-prepare kernel: dt and c_h of the step (as given, or from the
// wave speed in the scalar block), dt / dx_d, the damping factor, the time.
static int launch_prepare(mhd_ctx* c, double dt, double ch) {
  mhd::PrepArgs a;
  a.dt_req = dt;
  a.ch_req = ch;
  a.cfl = c->cfg.cfl;
  a.inv_dx_sum = c->inv_dx_sum;
  a.t_end = c->cfg.t_end;
  a.glm_alpha = c->cfg.glm_alpha;
  a.dh_min = c->dh_min;
  for (int d = 0; d < 3; ++d) {
    a.dx[d] = c->grid.dx[d];
    a.active[d] = c->grid.n[d] > 1;
  }
  ProfScope ps(c, 0);
  CK(c, mhd::launch_prep(a, &c->scal->sc, &c->scal->lam_bits, &c->scal->est_bits,
                         &c->scal->status, c->stream));
  return MHD_OK;
}

// The stages of one step: (kernel stage, profile class, input, U^n, output,
// a_n, a_w); returns their number.
struct St { int kind, cls; void *win, *un, *out; double an, aw; };
static int stage_sequence(const mhd_ctx* c, St seq[3]) {
  if (c->cfg.rk_order == 3) {
    seq[0] = {1, 1, c->Ua, nullptr, c->Ub, 0.0, 1.0};
    seq[1] = {3, 4, c->Ub, c->Ua, c->Uc, 0.75, 0.25};
    seq[2] = {2, 2, c->Uc, c->Ua, c->Ua, 1.0 / 3.0, 2.0 / 3.0};
    return 3;
  }
  seq[0] = {1, 1, c->Ua, nullptr, c->Ub, 0.0, 1.0};
  seq[1] = {2, 2, c->Ub, c->Ua, c->Ua, 0.5, 0.5};
  return 2;
}

// After an FP64 RK2 GLM step, U_b holds that step's first stage U1 (read by
// mhd_get_stage1); RK3 and constrained transport use U_b otherwise.
static bool keeps_stage1(const mhd_ctx* c) {
  return c->esize == 8 && c->cfg.rk_order != 3 && c->cfg.divb == MHD_DIVB_GLM;
}

int mhd_step(mhd_ctx* c, double dt, double ch) { return step_impl(c, dt, ch, nullptr); }

static int step_impl(mhd_ctx* c, double dt, double ch, const HostOut* ho) {
  if (!c) return MHD_ERR_INVALID;
  if (!c->have_state) return fail(c, MHD_ERR_STATE, "mhd_step before mhd_set_state");
  if (c->has_halo)
    return fail(c, MHD_ERR_STATE, "the context has halo faces: its ghost cells come from the "
                                  "caller (use mhd_step_begin / mhd_step_stage)");
  if (c->step_open)
    return fail(c, MHD_ERR_STATE, "a staged step (mhd_step_begin) is not finished");
  if (c->cfg.divb == MHD_DIVB_CT && !c->faces_set)
    return fail(c, MHD_ERR_STATE, "constrained transport: mhd_set_face_field after mhd_set_state");
  if (std::isnan(dt) || std::isnan(ch) || std::isinf(dt) || std::isinf(ch))
    return fail(c, MHD_ERR_INVALID, "mhd_step: non-finite dt or ch");
  if (!(dt > 0.0) || !(ch > 0.0)) {
    int rc = ensure_lambda(c);
    if (rc != MHD_OK) return rc;
  }
  c->stage1_valid = false;  // until this step has written its first stage
  int rc0 = launch_prepare(c, dt, ch);
  if (rc0 != MHD_OK) return rc0;
  St seq[3];
  const int nst = stage_sequence(c, seq);
  for (int i = 0; i < nst; ++i) {
    const St& q = seq[i];
    int rc = c->cfg.divb == MHD_DIVB_CT
                 ? (c->esize == 8 ? ct_stage<double>(c, q.kind, q.cls, q.win, q.un, q.out, q.an, q.aw)
                                  : ct_stage<float>(c, q.kind, q.cls, q.win, q.un, q.out, q.an, q.aw))
                 : MHD_OK;
    if (rc != MHD_OK) return rc;
    if (c->cfg.divb == MHD_DIVB_CT) continue;
    if (ho && i == nst - 1) {  // FP64, GLM, 3-D (checked by mhd_step_host)
      const int zs[3] = {0, ho->zh, c->grid.n[2]};
      for (int h = 0; h < 2; ++h) {
        {
          ProfScope ps(c, q.cls);
          CK(c, mhd::launch_stage<double>(c->grid, q.kind, static_cast<const double*>(q.win),
                                          static_cast<const double*>(q.un),
                                          static_cast<double*>(q.out), &c->scal->sc,
                                          &c->scal->lam_bits, c->scal->floor_cnt, c->stream,
                                          q.an, q.aw, nullptr, nullptr, zs[h], zs[h + 1],
                                          c->tz_half, &c->scal->est_bits));
        }
        CK(c, cudaEventRecord(c->xev[10 + h], c->stream));
        CK(c, cudaStreamWaitEvent(c->xfer, c->xev[10 + h], 0));
        rc = copy_planes(c, ho->U, static_cast<const double*>(q.out), zs[h], zs[h + 1],
                         cudaMemcpyDeviceToHost);
        if (rc != MHD_OK) return rc;
      }
      ProfScope ps(c, 3);
      CK(c, mhd::launch_speed_exact(c->grid, static_cast<const double*>(q.out),
                                    &c->scal->est_bits, &c->scal->lam_bits, c->stream));
      continue;
    }
    if (c->esize == 8) {
      {
        ProfScope ps(c, q.cls);
        CK(c, mhd::launch_stage<double>(c->grid, q.kind, static_cast<const double*>(q.win),
                                        static_cast<const double*>(q.un),
                                        static_cast<double*>(q.out), &c->scal->sc,
                                        &c->scal->lam_bits, c->scal->floor_cnt, c->stream, q.an,
                                        q.aw, nullptr, nullptr, 0, -1, 0, &c->scal->est_bits));
      }
      if (i == nst - 1) {  // the exact maximum speed of the new state (pass 2)
        ProfScope ps(c, 3);
        CK(c, mhd::launch_speed_exact(c->grid, static_cast<const double*>(q.out),
                                      &c->scal->est_bits, &c->scal->lam_bits, c->stream));
      }
    } else {
      ProfScope ps(c, q.cls);
      CK(c, mhd::launch_stage<float>(c->grid, q.kind, static_cast<const float*>(q.win),
                                     static_cast<const float*>(q.un), static_cast<float*>(q.out),
                                     &c->scal->sc, &c->scal->lam_bits, c->scal->floor_cnt,
                                     c->stream, q.an, q.aw));
    }
  }
  c->lam_valid = true;
  c->stage1_valid = keeps_stage1(c);
  return MHD_OK;
}

// ----------------------------------------------------- staged steps / halos --
static int ghost_width(const mhd_ctx* c) { return c->cfg.limiter == MHD_LIM_WENOZ ? 3 : 2; }

int mhd_halo_bytes(const mhd_ctx* c, int face, size_t* bytes) {
  if (!c || !bytes || face < 0 || face > 5) return MHD_ERR_INVALID;
  const int d = face >> 1;
  size_t area = 1;
  for (int e = 0; e < 3; ++e) area *= (size_t)(e == d ? ghost_width(c) : c->grid.n[e]);
  *bytes = 9 * area * c->esize;
  return MHD_OK;
}

int mhd_halo_pack(mhd_ctx* c, int face, void* d_dst) {
  if (!c) return MHD_ERR_INVALID;
  if (!d_dst || face < 0 || face > 5) return fail(c, MHD_ERR_INVALID, "mhd_halo_pack: bad argument");
  if (!c->have_state) return fail(c, MHD_ERR_STATE, "mhd_halo_pack before mhd_set_state");
  if (c->grid.n[face >> 1] < ghost_width(c))
    return fail(c, MHD_ERR_INVALID, "mhd_halo_pack: dimension %d has fewer cells than the "
                                    "ghost width", face >> 1);
  St seq[3];
  stage_sequence(c, seq);
  const void* W = c->step_open ? seq[c->stage_next].win : c->Ua;
  if (c->esize == 8)
    CK(c, mhd::launch_halo_pack<double>(c->grid, static_cast<const double*>(W), face,
                                        ghost_width(c), static_cast<double*>(d_dst), c->stream));
  else
    CK(c, mhd::launch_halo_pack<float>(c->grid, static_cast<const float*>(W), face,
                                       ghost_width(c), static_cast<float*>(d_dst), c->stream));
  return MHD_OK;
}

int mhd_lambda_max_into(mhd_ctx* c, void* d_bits) {
  if (!c) return MHD_ERR_INVALID;
  if (!d_bits) return fail(c, MHD_ERR_INVALID, "mhd_lambda_max_into: null pointer");
  if (!c->have_state) return fail(c, MHD_ERR_STATE, "mhd_lambda_max_into before mhd_set_state");
  if (c->step_open)
    return fail(c, MHD_ERR_STATE, "mhd_lambda_max_into inside a staged step");
  int rc = ensure_lambda(c);
  if (rc != MHD_OK) return rc;
  CK(c, mhd::launch_lambda_max_into(&c->scal->lam_bits, static_cast<unsigned long long*>(d_bits),
                                    c->stream));
  return MHD_OK;
}

int mhd_step_begin(mhd_ctx* c, double dt, double ch, const void* d_lambda_bits) {
  if (!c) return MHD_ERR_INVALID;
  if (!c->have_state) return fail(c, MHD_ERR_STATE, "mhd_step_begin before mhd_set_state");
  if (c->cfg.divb != MHD_DIVB_GLM)
    return fail(c, MHD_ERR_STATE, "staged steps are for GLM contexts");
  if (c->step_open) return fail(c, MHD_ERR_STATE, "the previous staged step is not finished");
  if (std::isnan(dt) || std::isnan(ch) || std::isinf(dt) || std::isinf(ch))
    return fail(c, MHD_ERR_INVALID, "mhd_step_begin: non-finite dt or ch");
  if (!(dt > 0.0) || !(ch > 0.0)) {
    if (d_lambda_bits) {
      CK(c, cudaMemcpyAsync(&c->scal->lam_bits, d_lambda_bits, sizeof(unsigned long long),
                            cudaMemcpyDeviceToDevice, c->stream));
    } else {
      int rc = ensure_lambda(c);
      if (rc != MHD_OK) return rc;
    }
  }
  c->stage1_valid = false;
  int rc = launch_prepare(c, dt, ch);
  if (rc != MHD_OK) return rc;
  c->step_open = true;
  c->stage_next = 0;
  return MHD_OK;
}

int mhd_step_stage(mhd_ctx* c, const void* const d_halo[6]) {
  if (!c) return MHD_ERR_INVALID;
  if (!c->step_open) return fail(c, MHD_ERR_STATE, "mhd_step_stage without mhd_step_begin");
  if (c->has_halo) {
    if (!d_halo) return fail(c, MHD_ERR_INVALID, "mhd_step_stage: the context has halo faces");
    for (int f = 0; f < 6; ++f)
      if (c->cfg.bc[f] == MHD_BC_HALO && !d_halo[f])
        return fail(c, MHD_ERR_INVALID, "mhd_step_stage: no halo buffer for face %d", f);
  }
  St seq[3];
  const int nst = stage_sequence(c, seq);
  const St& q = seq[c->stage_next];
  const bool last = c->stage_next == nst - 1;
  {
    ProfScope ps(c, q.cls);
    if (c->esize == 8) {
      const double* h[6];
      for (int f = 0; f < 6; ++f) h[f] = d_halo ? static_cast<const double*>(d_halo[f]) : nullptr;
      CK(c, c->has_halo
                ? mhd::launch_stage_halo<double>(
                      c->grid, q.kind, static_cast<const double*>(q.win),
                      static_cast<const double*>(q.un), static_cast<double*>(q.out), &c->scal->sc,
                      &c->scal->lam_bits, c->scal->floor_cnt, c->stream, q.an, q.aw, h,
                      &c->scal->est_bits)
                : mhd::launch_stage<double>(
                      c->grid, q.kind, static_cast<const double*>(q.win),
                      static_cast<const double*>(q.un), static_cast<double*>(q.out), &c->scal->sc,
                      &c->scal->lam_bits, c->scal->floor_cnt, c->stream, q.an, q.aw, nullptr,
                      nullptr, 0, -1, 0, &c->scal->est_bits));
    } else {
      const float* h[6];
      for (int f = 0; f < 6; ++f) h[f] = d_halo ? static_cast<const float*>(d_halo[f]) : nullptr;
      CK(c, c->has_halo
                ? mhd::launch_stage_halo<float>(
                      c->grid, q.kind, static_cast<const float*>(q.win),
                      static_cast<const float*>(q.un), static_cast<float*>(q.out), &c->scal->sc,
                      &c->scal->lam_bits, c->scal->floor_cnt, c->stream, q.an, q.aw, h, nullptr)
                : mhd::launch_stage<float>(c->grid, q.kind, static_cast<const float*>(q.win),
                                           static_cast<const float*>(q.un),
                                           static_cast<float*>(q.out), &c->scal->sc,
                                           &c->scal->lam_bits, c->scal->floor_cnt, c->stream,
                                           q.an, q.aw));
    }
  }
  if (last && c->esize == 8) {  // the exact maximum speed of the new state (pass 2)
    ProfScope ps(c, 3);
    CK(c, mhd::launch_speed_exact(c->grid, static_cast<const double*>(q.out), &c->scal->est_bits,
                                  &c->scal->lam_bits, c->stream));
  }
  if (last) {
    c->step_open = false;
    c->stage_next = 0;
    c->lam_valid = true;
  } else {
    c->stage_next++;
  }
  return MHD_OK;
}

int mhd_step_n(mhd_ctx* c, int nsteps) {
  if (!c) return MHD_ERR_INVALID;
  if (nsteps < 0) return fail(c, MHD_ERR_INVALID, "mhd_step_n: nsteps = %d < 0", nsteps);
  if (nsteps == 0) return MHD_OK;
  if (!c->have_state) return fail(c, MHD_ERR_STATE, "mhd_step_n before mhd_set_state");
  if (c->has_halo || c->step_open)
    return fail(c, MHD_ERR_STATE, "mhd_step_n: halo faces or an unfinished staged step");
  if (c->cfg.divb == MHD_DIVB_CT && !c->faces_set)
    return fail(c, MHD_ERR_STATE, "constrained transport: mhd_set_face_field after mhd_set_state");
  // the wave speed of the current state is reduced outside the graph: the
  // captured steps take it from the previous step, as mhd_step does
  int rc = ensure_lambda(c);
  if (rc != MHD_OK) return rc;
  if (c->prof_on) {  // per-launch timing needs the individual launches
    for (int i = 0; i < nsteps; ++i) {
      rc = step_impl(c, 0.0, 0.0, nullptr);
      if (rc != MHD_OK) return rc;
    }
    return MHD_OK;
  }
  if (!c->gexec || c->graph_steps != nsteps) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    if (!c->cap) CK(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    cudaStream_t keep = c->stream;
    c->stream = c->cap;  // every launch of the captured steps goes to the capture stream
    cudaError_t ce = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeRelaxed);
    if (ce == cudaSuccess) {
      for (int i = 0; i < nsteps && rc == MHD_OK; ++i) rc = step_impl(c, 0.0, 0.0, nullptr);
      cudaGraph_t graph = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(c->cap, &graph);
      if (rc == MHD_OK && ee == cudaSuccess) ce = cudaGraphInstantiate(&c->gexec, graph, 0);
      else if (ee != cudaSuccess) ce = ee;
      if (graph) cudaGraphDestroy(graph);
    }
    c->stream = keep;
    if (rc != MHD_OK) return rc;
    CK(c, ce);
    c->graph_steps = nsteps;
  }
  CK(c, cudaGraphLaunch(c->gexec, c->stream));
  c->lam_valid = true;
  c->stage1_valid = keeps_stage1(c);  // also when the graph was replayed, not captured
  return MHD_OK;
}

int mhd_step_host(mhd_ctx* c, const double* U_in, double* U_out, double dt, double ch) {
  if (!c) return MHD_ERR_INVALID;
  if (!U_in || !U_out) return fail(c, MHD_ERR_INVALID, "mhd_step_host: null buffer");
  if (c->has_halo)
    return fail(c, MHD_ERR_STATE, "mhd_step_host: the context has halo faces (use the staged "
                                  "calls mhd_step_begin / mhd_step_stage)");
  if (c->cfg.divb == MHD_DIVB_CT)
    return fail(c, MHD_ERR_INVALID,
                "mhd_step_host: constrained transport needs a face field; use mhd_set_state, "
                "mhd_set_face_field, mhd_step and mhd_get_state");
  if (std::isnan(dt) || std::isnan(ch) || std::isinf(dt) || std::isinf(ch))
    return fail(c, MHD_ERR_INVALID, "mhd_step_host: non-finite dt or ch");
  const int nz = c->grid.n[2];
  if (!(c->esize == 8 && c->grid.ndim == 3 && nz >= 8)) {
    // no overlap: the three calls in sequence
    int rc = mhd_set_state(c, U_in, MHD_HOST, MHD_CONS);
    if (rc == MHD_OK) rc = mhd_step(c, dt, ch);
    if (rc == MHD_OK) rc = mhd_get_state(c, U_out, MHD_HOST, MHD_CONS);
    return rc;
  }
  if (!c->xfer_ready) {
    CK(c, cudaStreamCreateWithFlags(&c->xfer, cudaStreamNonBlocking));
    for (int i = 0; i < 12; ++i) CK(c, cudaEventCreateWithFlags(&c->xev[i], cudaEventDisableTiming));
    c->xfer_ready = true;
  }
  double* A = static_cast<double*>(c->Ua);
  const long long plane = (long long)c->grid.n[0] * c->grid.n[1];
  // the copies start once the work already enqueued on the context's stream
  // (which may read the state) is done
  CK(c, cudaEventRecord(c->xev[0], c->stream));
  CK(c, cudaStreamWaitEvent(c->xfer, c->xev[0], 0));
  // as mhd_set_state: the time, counters and wave speed restart
  CK(c, cudaMemsetAsync(c->scal, 0, sizeof(Scalars), c->stream));
  c->have_state = true;
  c->lam_valid = false;
  c->faces_set = false;
  c->stage1_valid = false;
  const bool need_lam = !(dt > 0.0) || !(ch > 0.0);
  // eight input slabs; the wave-speed reduction follows each as it lands
  for (int k = 0; k < 8; ++k) {
    const int z0 = (int)((long long)nz * k / 8), z1 = (int)((long long)nz * (k + 1) / 8);
    int rc = copy_planes(c, A, U_in, z0, z1, cudaMemcpyHostToDevice);
    if (rc != MHD_OK) return rc;
    CK(c, cudaEventRecord(c->xev[1 + k], c->xfer));
    CK(c, cudaStreamWaitEvent(c->stream, c->xev[1 + k], 0));
    if (need_lam) {  // pass 1 of the wave-speed maximum, slab by slab
      ProfScope ps(c, 3);
      CK(c, mhd::launch_speed_estimate(c->grid, A, z0 * plane, z1 * plane, &c->scal->est_bits,
                                       c->stream));
    }
  }
  if (need_lam) {  // pass 2 once the whole state is on the device
    ProfScope ps(c, 3);
    CK(c, mhd::launch_speed_exact(c->grid, A, &c->scal->est_bits, &c->scal->lam_bits,
                                  c->stream));
  }
  c->lam_valid = need_lam;
  HostOut ho{U_out, nz / 2};
  int rc = step_impl(c, dt, ch, &ho);
  if (rc != MHD_OK) return rc;
  CK(c, cudaStreamSynchronize(c->xfer));
  return MHD_OK;
}

int mhd_step_info(mhd_ctx* c, double out[4]) {
  if (!c || !out) return MHD_ERR_INVALID;
  Scalars h;
  CK(c, cudaMemcpyAsync(&h, c->scal, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  out[0] = h.sc.t;
  out[1] = h.sc.dt;
  out[2] = h.sc.ch;
  out[3] = h.sc.steps;
  if (h.status) return fail(c, MHD_ERR_NONFINITE, "device flagged a non-finite dt or c_h");
  double lam;
  memcpy(&lam, &h.lam_bits, sizeof(lam));
  if (c->lam_valid && std::isnan(lam))
    return fail(c, MHD_ERR_NONFINITE, "non-finite state after the last step");
  return MHD_OK;
}

int mhd_step_record(mhd_ctx* c, double* d_out) {
  if (!c || !d_out) return MHD_ERR_INVALID;
  CK(c, mhd::launch_step_record(&c->scal->sc, d_out, c->stream));
  return MHD_OK;
}

int mhd_counters(mhd_ctx* c, long long counters[4]) {
  if (!c || !counters) return MHD_ERR_INVALID;
  Scalars h;
  CK(c, cudaMemcpyAsync(&h, c->scal, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  counters[0] = (long long)h.floor_cnt[0];
  counters[1] = (long long)h.floor_cnt[1];
  counters[2] = (long long)h.status;
  counters[3] = (long long)h.floor_cnt[2];
  return MHD_OK;
}

int mhd_conserved_sums(mhd_ctx* c, double out[8]) {
  if (!c || !out) return MHD_ERR_INVALID;
  if (!c->have_state) return fail(c, MHD_ERR_STATE, "mhd_conserved_sums before mhd_set_state");
  if (c->esize == 8)
    CK(c, mhd::launch_sums<double>(c->grid, static_cast<const double*>(c->Ua), c->partials,
                                   kSumBlocks, c->scal->sums, c->stream));
  else
    CK(c, mhd::launch_sums<float>(c->grid, static_cast<const float*>(c->Ua), c->partials,
                                  kSumBlocks, c->scal->sums, c->stream));
  CK(c, cudaMemcpyAsync(out, c->scal->sums, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

int mhd_flux_batch(const void* VL, const void* VR, void* F, long long nface, int dir, double ch,
                   double gamma, int precision, void* stream) {
  if (!VL || !VR || !F || nface < 0 || dir < 0 || dir > 2 || !(ch > 0.0) || !(gamma > 1.0) ||
      (precision != MHD_FP64 && precision != MHD_FP32))
    return mhd::free_fail(MHD_ERR_INVALID, "mhd_flux_batch: bad argument");
  if (nface == 0) return MHD_OK;
  cudaError_t e;
  if (precision == MHD_FP64)
    e = mhd::launch_flux_batch<double>(static_cast<const double*>(VL),
                                       static_cast<const double*>(VR), static_cast<double*>(F),
                                       nface, dir, ch, gamma, static_cast<cudaStream_t>(stream));
  else
    e = mhd::launch_flux_batch<float>(static_cast<const float*>(VL),
                                      static_cast<const float*>(VR), static_cast<float*>(F),
                                      nface, dir, ch, gamma, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess)
    return mhd::free_fail(MHD_ERR_CUDA, "mhd_flux_batch: %s", cudaGetErrorString(e));
  return MHD_OK;
}

int mhd_fp64_fma_rate(void* stream, unsigned warp_mask, double out[3]) {
  if (!out) return mhd::free_fail(MHD_ERR_INVALID, "mhd_fp64_fma_rate: out is NULL");
  const cudaError_t e =
      mhd::measure_fma_rate(static_cast<cudaStream_t>(stream), warp_mask, out);
  if (e != cudaSuccess)
    return mhd::free_fail(MHD_ERR_CUDA, "mhd_fp64_fma_rate: %s", cudaGetErrorString(e));
  return MHD_OK;
}

static int adjoint_impl(mhd_ctx* c, const double* U_n, const double* U1, const double* lam_np1,
                        double* lam_n, double dt, double ch) {
  if (!c) return MHD_ERR_INVALID;
  if (!(c->cfg.flags & MHD_FLAG_ADJOINT) || c->esize != 8)
    return fail(c, MHD_ERR_STATE, "context created without MHD_FLAG_ADJOINT / MHD_FP64");
  if (!U_n || !lam_np1 || !lam_n || lam_n == lam_np1 || !(dt > 0.0) || !(ch > 0.0) ||
      !std::isfinite(dt) || !std::isfinite(ch) || (U1 && (U1 == lam_n || U1 == U_n)))
    return fail(c, MHD_ERR_INVALID, "mhd_adjoint_step: bad argument");
  return mhd::adjoint_step(c->grid, dt, ch, c->cfg.glm_alpha, c->dh_min, U_n, U1, lam_np1,
                           lam_n, c->adj, c->adj_bytes, c->stream, c->err, sizeof(c->err));
}

int mhd_adjoint_step(mhd_ctx* c, const double* U_n, const double* lam_np1, double* lam_n,
                     double dt, double ch) {
  return adjoint_impl(c, U_n, nullptr, lam_np1, lam_n, dt, ch);
}

int mhd_adjoint_step_stage1(mhd_ctx* c, const double* U_n, const double* U1,
                            const double* lam_np1, double* lam_n, double dt, double ch) {
  if (c && !U1) return fail(c, MHD_ERR_INVALID, "mhd_adjoint_step_stage1: null U1");
  return adjoint_impl(c, U_n, U1, lam_np1, lam_n, dt, ch);
}

int mhd_get_stage1(mhd_ctx* c, double* U1, int where) {
  if (!c) return MHD_ERR_INVALID;
  if (!U1 || (where != MHD_HOST && where != MHD_DEVICE))
    return fail(c, MHD_ERR_INVALID, "mhd_get_stage1: bad argument");
  if (!c->stage1_valid)
    return fail(c, MHD_ERR_STATE,
                "mhd_get_stage1: no FP64 RK2 GLM step since the state was last set");
  const long long n = 9 * c->grid.ncell;
  CK(c, cudaMemcpyAsync(U1, c->Ub, n * 8,
                        where == MHD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                        c->stream));
  if (where == MHD_HOST) CK(c, cudaStreamSynchronize(c->stream));
  return MHD_OK;
}

int mhd_profile_enable(mhd_ctx* c, int enable) {
  if (!c) return MHD_ERR_INVALID;
  c->prof_on = enable != 0;
  return MHD_OK;
}

int mhd_profile_read(mhd_ctx* c, long long counts[6], double ms[6]) {
  if (!c || !counts || !ms) return MHD_ERR_INVALID;
  for (int k = 0; k < 6; ++k) {
    counts[k] = 0;
    ms[k] = 0.0;
  }
  CK(c, cudaStreamSynchronize(c->stream));
  for (auto& r : c->prof_recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      counts[r.kind] += 1;
      ms[r.kind] += t;
    }
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof_recs.clear();
  return MHD_OK;
}

const char* mhd_last_error(const mhd_ctx* c) { return c ? c->err : mhd::g_free_err; }

int mhd_destroy(mhd_ctx* c) {
  if (!c) return MHD_ERR_INVALID;
  for (auto& r : c->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->prof_pool) cudaEventDestroy(e);
  if (c->xfer_ready) {
    cudaStreamSynchronize(c->xfer);
    for (auto e : c->xev) cudaEventDestroy(e);
    cudaStreamDestroy(c->xfer);
  }
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
  return MHD_OK;
}

}  // extern "C"
