// Batched ensemble of independent 3-D boxes advanced in one persistent,
// cooperative, graph-captured launch (FP32 bulk).
//
// Each box is an ordinary context (its own state arrays, grid, boundary
// conditions, time step).  The persistent kernel walks one work list holding
// every box's stage tiles (column tile x z chunk); per step:
//   prepare (one thread per box: CFL dt and c_h from that box's reduced wave
//   speed) -> grid sync -> stage 1 over all tiles -> grid sync -> stage 2
//   over all tiles (reducing each box's next wave speed) -> grid sync.
// The tile code is the same stage_tile() the per-box launches use, so every
// box evolves bitwise as it would under its own mhd_step calls.  Grid syncs
// are cooperative-group barriers: the cooperative launch guarantees that all
// CTAs are co-resident (the launch fails otherwise), so no wait can hang.
// The tile shape -- the launch's tile height TY (32 x 8 or 32 x 4 columns,
// one instantiation of the persistent kernel each, both on 8-warp CTAs) and
// each box-size class's z-chunk depth tz -- is picked by a timing autotuner
// (mhd_ensemble_autotune).  (Both tile heights in one kernel, chosen per box,
// made it spill and ran slower.)
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "mhd_ctx.h"

namespace cg = cooperative_groups;

namespace mhd {

constexpr int kEnsNW = 8;
constexpr int kEnsTYs[2] = {8, 4};  // the tile heights of the two kernel instantiations

struct EnsBox {
  StageParams<float> p;  // geometry / physics; state pointers set per stage
  float* Ua;
  float* Ub;
  StepScalars sc;
  unsigned long long lam_bits[2];
  unsigned long long floor_cnt[3];
  unsigned int status;
  int cur;               // lam_bits slot holding the current state's wave speed
  double cfl, inv_dx_sum, t_end, glm_alpha, dh_min;
  double dx[3];
  int ty;                // tile height of the launch: 8 or 4 rows of 32 columns
  int ntx, nty, ntz;     // tiles per dimension
  long long item0;       // first work item of this box
};

struct EnsArgs {
  EnsBox* boxes;
  int nbox;
  long long nitems;
  int nsteps;
};

__device__ __forceinline__ void ens_prep(EnsBox& b) {
  const int cur = b.cur;
  const double lam = __longlong_as_double((long long)b.lam_bits[cur]);
  double ch = lam;
  const double t = b.sc.t;
  double dt = b.cfl / (ch * b.inv_dx_sum);
  if (b.t_end > 0.0) dt = fmin(dt, b.t_end - t);
  if (!(ch > 0.0) || !(ch < INFINITY) || !(dt >= 0.0) || !(dt < INFINITY)) {
    atomicOr(&b.status, 1u);
    dt = 0.0;
    ch = 1.0;
  }
  b.sc.dt = dt;
  b.sc.ch = ch;
  for (int d = 0; d < 3; ++d) b.sc.dtdx[d] = dt / b.dx[d];
  b.sc.damp = exp(-b.glm_alpha * ch * dt / b.dh_min);
  b.sc.t = t + dt;
  b.sc.lam = lam;
  b.sc.steps += 1.0;
  const int nxt = 1 - cur;
  b.lam_bits[nxt] = 0ull;  // stage 2 reduces the new state's wave speed here
  b.cur = nxt;
}

__device__ __forceinline__ int ens_find(const EnsBox* boxes, int nbox, long long item) {
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (boxes[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int TY, int STAGE>
__device__ __forceinline__ void ens_stage(const EnsArgs& a, unsigned char* smem, double* wmax) {
  for (long long it = blockIdx.x; it < a.nitems; it += gridDim.x) {
    const int bi = ens_find(a.boxes, a.nbox, it);
    EnsBox& B = a.boxes[bi];
    StageParams<float> p = B.p;
    p.win = STAGE == 1 ? B.Ua : B.Ub;
    p.un = STAGE == 1 ? nullptr : B.Ua;
    p.uout = STAGE == 1 ? B.Ub : B.Ua;
    p.lam_bits = &B.lam_bits[B.cur];
    p.floor_cnt = B.floor_cnt;
    p.a_n = 0.5f;
    p.a_w = 0.5f;
    const StepScalars sc = B.sc;
    const long long j = it - B.item0;
    const int bx = (int)(j % B.ntx);
    const int by = (int)((j / B.ntx) % B.nty);
    const int bz = (int)(j / ((long long)B.ntx * B.nty));
    // (no interior prefetch: the persistent kernel's registers are capped at
    // 128 for two CTAs per SM, and the prefetch registers spill there)
    stage_tile<float, TY, kEnsNW, STAGE, true, false, false, false>(p, sc, bx, by, bz, smem, wmax);
  }
}

template <int TY>
__global__ void __launch_bounds__(kEnsNW * 32, 2) ensemble_kernel(const EnsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double wmax[kEnsNW];
  cg::grid_group grid = cg::this_grid();
  for (int s = 0; s < a.nsteps; ++s) {
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gt < a.nbox) ens_prep(a.boxes[gt]);
    grid.sync();
    ens_stage<TY, 1>(a, smem_raw, wmax);
    grid.sync();
    ens_stage<TY, 2>(a, smem_raw, wmax);
    grid.sync();
  }
}

}  // namespace mhd

using mhd::EnsBox;

struct mhd_ensemble {
  int nbox;
  std::vector<mhd_ctx*> ctx;
  std::vector<EnsBox> h;       // host copy of the box records
  EnsBox* d;                   // device box records (in the workspace)
  std::vector<int> cur;        // host mirror of each box's lam slot
  std::vector<bool> lam_ok;    // box wave speed valid for the next step
  std::vector<int> tz;         // z-chunk depth per box
  int ty;                      // tile height of the launches (8 or 4)
  cudaStream_t stream;
  cudaStream_t cap;            // private stream the graph is captured on (the
                               // legacy default stream cannot be captured)
  size_t smem[2];              // per tile height (index of kEnsTYs)
  int grid_ctas[2];
  long long nitems;
  cudaGraphExec_t gexec;
  int graph_steps;
  bool graph_ok;
  char err[512];
};

static int efail(mhd_ensemble* e, int code, const char* fmt, ...) {
  if (e) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(e->err, sizeof(e->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define ECK(e, call)                                                                      \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return efail((e), MHD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

// Each box: a valid 3-D MHD_FP32 config with RK2, PLM and GLM, no adjoint.
// A failure leaves its reason for mhd_last_error(NULL).
static int ens_validate(const mhd_config* cfgs, int nbox) {
  if (!cfgs || nbox < 1)
    return mhd::free_fail(MHD_ERR_INVALID, "ensemble: no boxes (nbox = %d)", nbox);
  for (int b = 0; b < nbox; ++b) {
    size_t bytes;
    if (mhd_workspace_bytes(&cfgs[b], &bytes) != MHD_OK) {
      char why[256];  // the message is rewritten below: copy it out first
      snprintf(why, sizeof(why), "%s", mhd_last_error(nullptr));
      return mhd::free_fail(MHD_ERR_INVALID, "ensemble box %d: %s", b, why);
    }
    if (cfgs[b].precision != MHD_FP32 || cfgs[b].n[1] < 2 || cfgs[b].n[2] < 2 ||
        (cfgs[b].flags & MHD_FLAG_ADJOINT) || cfgs[b].rk_order != 2 ||
        cfgs[b].limiter == MHD_LIM_WENOZ || cfgs[b].divb != MHD_DIVB_GLM)
      return mhd::free_fail(MHD_ERR_INVALID,
                            "ensemble box %d: needs a 3-D MHD_FP32 RK2 PLM GLM config "
                            "without MHD_FLAG_ADJOINT", b);
  }
  return MHD_OK;
}

// Rebuilds the work list for the current tz choices and uploads the records.
static int ens_layout(mhd_ensemble* e) {
  long long item = 0;
  for (int b = 0; b < e->nbox; ++b) {
    EnsBox& B = e->h[b];
    const mhd::Grid& g = e->ctx[b]->grid;
    B.p.tz = e->tz[b];
    B.ty = e->ty;
    B.p.zlo = 0;
    B.p.zhi = g.n[2];
    B.ntx = (g.n[0] + 31) / 32;
    B.nty = (g.n[1] + B.ty - 1) / B.ty;
    B.ntz = (g.n[2] + B.p.tz - 1) / B.p.tz;
    B.item0 = item;
    item += (long long)B.ntx * B.nty * B.ntz;
  }
  e->nitems = item;
  // upload only the layout fields (scalars, wave speeds, counters stay on
  // the device): write whole records but with the device's current dynamic
  // fields read back first
  std::vector<EnsBox> dev(e->nbox);
  ECK(e, cudaMemcpyAsync(dev.data(), e->d, sizeof(EnsBox) * e->nbox, cudaMemcpyDeviceToHost,
                         e->stream));
  ECK(e, cudaStreamSynchronize(e->stream));
  for (int b = 0; b < e->nbox; ++b) {
    EnsBox r = e->h[b];
    r.sc = dev[b].sc;
    memcpy(r.lam_bits, dev[b].lam_bits, sizeof(r.lam_bits));
    memcpy(r.floor_cnt, dev[b].floor_cnt, sizeof(r.floor_cnt));
    r.status = dev[b].status;
    r.cur = dev[b].cur;
    e->h[b] = r;
  }
  ECK(e, cudaMemcpyAsync(e->d, e->h.data(), sizeof(EnsBox) * e->nbox, cudaMemcpyHostToDevice,
                         e->stream));
  ECK(e, cudaStreamSynchronize(e->stream));
  if (e->gexec) {
    cudaGraphExecDestroy(e->gexec);
    e->gexec = nullptr;
    e->graph_steps = -1;
  }
  return MHD_OK;
}

static cudaError_t ens_launch(mhd_ensemble* e, int nsteps, cudaStream_t s) {
  mhd::EnsArgs a{e->d, e->nbox, e->nitems, nsteps};
  const int k = e->ty == 4 ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(e->grid_ctas[k]);
  cfg.blockDim = dim3(mhd::kEnsNW * 32);
  cfg.dynamicSmemBytes = e->smem[k];
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return k ? cudaLaunchKernelEx(&cfg, mhd::ensemble_kernel<4>, a)
           : cudaLaunchKernelEx(&cfg, mhd::ensemble_kernel<8>, a);
}

extern "C" {

int mhd_ensemble_workspace_bytes(const mhd_config* cfgs, int nbox, size_t* bytes) {
  if (!bytes) return mhd::free_fail(MHD_ERR_INVALID, "mhd_ensemble_workspace_bytes: null bytes");
  if (ens_validate(cfgs, nbox) != MHD_OK) return MHD_ERR_INVALID;
  size_t total = 0;
  for (int b = 0; b < nbox; ++b) {
    size_t s = 0;
    mhd_workspace_bytes(&cfgs[b], &s);
    total += mhd::align256(s);
  }
  total += mhd::align256(sizeof(EnsBox) * (size_t)nbox);
  *bytes = total;
  return MHD_OK;
}

int mhd_ensemble_create(const mhd_config* cfgs, int nbox, void* d_workspace, size_t bytes,
                        void* stream, mhd_ensemble** out) {
  if (!out) return mhd::free_fail(MHD_ERR_INVALID, "mhd_ensemble_create: null out");
  *out = nullptr;
  if (ens_validate(cfgs, nbox) != MHD_OK) return MHD_ERR_INVALID;
  size_t need = 0;
  mhd_ensemble_workspace_bytes(cfgs, nbox, &need);
  if (!d_workspace || bytes < need || ((uintptr_t)d_workspace & 255))
    return mhd::free_fail(MHD_ERR_NOMEM,
                          "mhd_ensemble_create: workspace %p of %zu bytes (need %zu, "
                          "256-byte aligned)", d_workspace, bytes, need);
  mhd_ensemble* e = new (std::nothrow) mhd_ensemble();
  if (!e) return mhd::free_fail(MHD_ERR_NOMEM, "mhd_ensemble_create: host allocation failed");
  e->nbox = nbox;
  e->stream = static_cast<cudaStream_t>(stream);
  e->gexec = nullptr;
  e->graph_steps = -1;
  e->graph_ok = true;
  e->cap = nullptr;
  if (cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete e;
    return mhd::free_fail(MHD_ERR_CUDA, "mhd_ensemble_create: stream creation failed");
  }
  snprintf(e->err, sizeof(e->err), "no error");
  char* p = static_cast<char*>(d_workspace);
  for (int b = 0; b < nbox; ++b) {
    size_t s = 0;
    mhd_workspace_bytes(&cfgs[b], &s);
    mhd_ctx* c = nullptr;
    int rc = mhd_create(&cfgs[b], p, s, stream, &c);
    if (rc != MHD_OK) {
      for (auto* x : e->ctx) mhd_destroy(x);
      cudaStreamDestroy(e->cap);
      delete e;
      return rc;
    }
    e->ctx.push_back(c);
    p += mhd::align256(s);
  }
  e->d = reinterpret_cast<EnsBox*>(p);
  e->h.resize(nbox);
  e->cur.assign(nbox, 0);
  e->lam_ok.assign(nbox, false);
  e->tz.assign(nbox, 16);
  e->ty = 8;
  for (int b = 0; b < nbox; ++b) {
    mhd_ctx* c = e->ctx[b];
    EnsBox B;
    memset(&B, 0, sizeof(B));
    B.p.n[0] = c->grid.n[0];
    B.p.n[1] = c->grid.n[1];
    B.p.n[2] = c->grid.n[2];
    for (int d = 0; d < 3; ++d) {
      B.p.bc_lo[d] = c->grid.bc_lo[d];
      B.p.bc_hi[d] = c->grid.bc_hi[d];
      B.dx[d] = c->grid.dx[d];
    }
    B.p.sy = c->grid.n[0];
    B.p.sz = (long long)c->grid.n[0] * c->grid.n[1];
    B.p.sv = c->grid.ncell;
    B.p.limiter = c->grid.limiter;
    B.p.ph = mhd::make_phys<float>(c->grid);
    B.Ua = static_cast<float*>(c->Ua);
    B.Ub = static_cast<float*>(c->Ub);
    B.cfl = c->cfg.cfl;
    B.inv_dx_sum = c->inv_dx_sum;
    B.t_end = c->cfg.t_end;
    B.glm_alpha = c->cfg.glm_alpha;
    B.dh_min = c->dh_min;
    e->tz[b] = std::min(16, c->grid.n[2]);
    e->h[b] = B;
  }
  // zeroed dynamic fields on the device, then the layout
  cudaError_t ce = cudaMemsetAsync(e->d, 0, sizeof(EnsBox) * nbox, e->stream);
  // both instantiations: shared-memory limit and co-resident CTAs per SM
  // (the cooperative grid size)
  e->smem[0] = (size_t)mhd::TileGeom<8, true>::WORDS * sizeof(float);
  e->smem[1] = (size_t)mhd::TileGeom<4, true>::WORDS * sizeof(float);
  int per_sm[2] = {0, 0}, nsm = 0, dev = 0;
  if (ce == cudaSuccess)
    ce = cudaFuncSetAttribute(mhd::ensemble_kernel<8>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem[0]);
  if (ce == cudaSuccess)
    ce = cudaFuncSetAttribute(mhd::ensemble_kernel<4>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem[1]);
  if (ce == cudaSuccess) ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (ce == cudaSuccess)
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], mhd::ensemble_kernel<8>,
                                                       mhd::kEnsNW * 32, e->smem[0]);
  if (ce == cudaSuccess)
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], mhd::ensemble_kernel<4>,
                                                       mhd::kEnsNW * 32, e->smem[1]);
  if (ce != cudaSuccess || per_sm[0] < 1 || per_sm[1] < 1 || ens_layout(e) != MHD_OK) {
    for (auto* x : e->ctx) mhd_destroy(x);
    cudaStreamDestroy(e->cap);
    delete e;
    return mhd::free_fail(MHD_ERR_CUDA, "mhd_ensemble_create: kernel set-up failed (%s)",
                          cudaGetErrorString(ce));
  }
  e->grid_ctas[0] = per_sm[0] * nsm;
  e->grid_ctas[1] = per_sm[1] * nsm;
  *out = e;
  return MHD_OK;
}

int mhd_ensemble_set_state(mhd_ensemble* e, int box, const double* U, int where, int kind) {
  if (!e || box < 0 || box >= e->nbox) return MHD_ERR_INVALID;
  int rc = mhd_set_state(e->ctx[box], U, where, kind);
  if (rc != MHD_OK) return efail(e, rc, "box %d: %s", box, mhd_last_error(e->ctx[box]));
  // restart this box: time, steps, wave-speed slots and counters
  EnsBox r = e->h[box];
  memset(&r.sc, 0, sizeof(r.sc));
  r.lam_bits[0] = r.lam_bits[1] = 0ull;
  r.floor_cnt[0] = r.floor_cnt[1] = r.floor_cnt[2] = 0ull;
  r.status = 0;
  r.cur = 0;
  e->h[box] = r;
  ECK(e, cudaMemcpyAsync(e->d + box, &e->h[box], sizeof(EnsBox), cudaMemcpyHostToDevice,
                         e->stream));
  ECK(e, cudaStreamSynchronize(e->stream));
  e->cur[box] = 0;
  e->lam_ok[box] = false;
  return MHD_OK;
}

int mhd_ensemble_get_state(mhd_ensemble* e, int box, double* U, int where, int kind) {
  if (!e || box < 0 || box >= e->nbox) return MHD_ERR_INVALID;
  int rc = mhd_get_state(e->ctx[box], U, where, kind);
  if (rc != MHD_OK) return efail(e, rc, "box %d: %s", box, mhd_last_error(e->ctx[box]));
  return MHD_OK;
}

int mhd_ensemble_step(mhd_ensemble* e, int nsteps) {
  if (!e || nsteps < 1) return MHD_ERR_INVALID;
  for (int b = 0; b < e->nbox; ++b) {
    if (!e->ctx[b]->have_state) return efail(e, MHD_ERR_STATE, "box %d has no state", b);
    if (!e->lam_ok[b]) {
      ECK(e, mhd::launch_max_speed<float>(e->ctx[b]->grid, static_cast<const float*>(e->ctx[b]->Ua),
                                          &e->d[b].lam_bits[e->cur[b]], nullptr, e->stream));
      e->lam_ok[b] = true;
    }
  }
  if (e->graph_ok) {
    if (!e->gexec || e->graph_steps != nsteps) {
      if (e->gexec) {
        cudaGraphExecDestroy(e->gexec);
        e->gexec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        cudaError_t le = ens_launch(e, nsteps, e->cap);
        ce = cudaStreamEndCapture(e->cap, &graph);
        if (le != cudaSuccess) ce = le;
      }
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&e->gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        cudaGetLastError();
        e->graph_ok = false;  // launch directly from now on
        e->gexec = nullptr;
      } else {
        e->graph_steps = nsteps;
      }
    }
  }
  if (e->graph_ok)
    ECK(e, cudaGraphLaunch(e->gexec, e->stream));
  else
    ECK(e, ens_launch(e, nsteps, e->stream));
  for (int b = 0; b < e->nbox; ++b)
    if (nsteps % 2) e->cur[b] ^= 1;
  return MHD_OK;
}

int mhd_ensemble_info(mhd_ensemble* e, int box, double out[7]) {
  if (!e || !out || box < 0 || box >= e->nbox) return MHD_ERR_INVALID;
  EnsBox r;
  ECK(e, cudaMemcpyAsync(&r, e->d + box, sizeof(r), cudaMemcpyDeviceToHost, e->stream));
  ECK(e, cudaStreamSynchronize(e->stream));
  out[0] = r.sc.t;
  out[1] = r.sc.dt;
  out[2] = r.sc.ch;
  out[3] = r.sc.steps;
  out[4] = (double)e->tz[box];
  out[5] = e->graph_ok ? 1.0 : 0.0;
  out[6] = (double)e->ty;
  if (r.status) return efail(e, MHD_ERR_NONFINITE, "box %d: non-finite dt or c_h", box);
  return MHD_OK;
}

int mhd_ensemble_set_tiles(mhd_ensemble* e, int box, int ty, int tz) {
  if (!e) return MHD_ERR_INVALID;
  if (box < 0 || box >= e->nbox || (ty != 8 && ty != 4) || tz < 1)
    return efail(e, MHD_ERR_INVALID, "mhd_ensemble_set_tiles: box %d, tile height %d (8 or 4), "
                 "z-chunk depth %d (>= 1)", box, ty, tz);
  e->ty = ty;  // the launch's tile height: every box
  e->tz[box] = std::min(tz, e->ctx[box]->grid.n[2]);
  return ens_layout(e);
}

int mhd_ensemble_autotune(mhd_ensemble* e, int trial_steps) {
  if (!e || trial_steps < 1) return MHD_ERR_INVALID;
  // size classes: boxes with the same grid
  std::map<long long, std::vector<int>> cls;
  for (int b = 0; b < e->nbox; ++b) {
    const mhd::Grid& g = e->ctx[b]->grid;
    cls[((long long)g.n[0] << 40) | ((long long)g.n[1] << 20) | g.n[2]].push_back(b);
  }
  cudaEvent_t t0, t1;
  ECK(e, cudaEventCreate(&t0));
  ECK(e, cudaEventCreate(&t1));
  // the best of two timed launches after a warm-up launch (which also
  // builds the graph)
  auto time_one = [&](float* ms) -> int {
    int rc = ens_layout(e);
    if (rc != MHD_OK) return rc;
    rc = mhd_ensemble_step(e, trial_steps);
    if (rc != MHD_OK) return rc;
    *ms = 1e30f;
    for (int r = 0; r < 2; ++r) {
      ECK(e, cudaEventRecord(t0, e->stream));
      rc = mhd_ensemble_step(e, trial_steps);
      if (rc != MHD_OK) return rc;
      ECK(e, cudaEventRecord(t1, e->stream));
      ECK(e, cudaEventSynchronize(t1));
      float m = 0.f;
      ECK(e, cudaEventElapsedTime(&m, t0, t1));
      *ms = std::min(*ms, m);
    }
    return MHD_OK;
  };
  float best = 0.f;
  int rc = MHD_OK;
  // A candidate is kept only when more than 1 % faster than the incumbent
  // (timing noise).  First the launch's tile height, then -- one pass of
  // coordinate descent over the size classes -- each class's z-chunk depth.
  rc = time_one(&best);
  const int ty0 = e->ty;
  for (int ty : mhd::kEnsTYs) {
    if (rc != MHD_OK || ty == ty0) continue;
    const int prev = e->ty;
    e->ty = ty;
    float ms = 0.f;
    rc = time_one(&ms);
    if (rc == MHD_OK && ms < 0.99f * best)
      best = ms;
    else
      e->ty = prev;
  }
  const int cands[] = {4, 8, 16, 32, 64};
  for (auto& kv : cls) {
    const int nz = e->ctx[kv.second[0]]->grid.n[2];
    int keep = e->tz[kv.second[0]];
    if (rc == MHD_OK) rc = time_one(&best);  // the incumbent, timed afresh
    for (int c : cands) {
      if (rc != MHD_OK) break;
      if (c > nz || c == keep) continue;
      for (int b : kv.second) e->tz[b] = c;
      float ms = 0.f;
      rc = time_one(&ms);
      if (rc == MHD_OK && ms < 0.99f * best) {
        best = ms;
        keep = c;
      }
    }
    for (int b : kv.second) e->tz[b] = keep;
  }
  if (rc == MHD_OK) rc = ens_layout(e);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return rc;
}

const char* mhd_ensemble_last_error(const mhd_ensemble* e) { return e ? e->err : "null"; }

int mhd_ensemble_destroy(mhd_ensemble* e) {
  if (!e) return MHD_ERR_INVALID;
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  if (e->cap) cudaStreamDestroy(e->cap);
  for (auto* c : e->ctx) mhd_destroy(c);
  delete e;
  return MHD_OK;
}

}  // extern "C"
