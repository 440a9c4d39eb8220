// Context object of the C ABI (internal; shared by mhd_api.cu and
// mhd_ensemble.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/mhd.h"
#include "mhd_internal.h"

namespace mhd {

constexpr int kSumBlocks = 1024;

struct Scalars {  // device block at the start of the scalar region
  StepScalars sc;
  unsigned long long lam_bits;
  unsigned long long floor_cnt[3];  // rho floor, p floor, FP32 p recomputed in FP64
  unsigned int status;
  unsigned int est_bits;  // FP64: max reliable FP32 speed estimate (FP32 bits)
  double sums[8];
  unsigned long long aux_bits;  // scratch max (face divergence)
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace mhd

struct mhd_ctx {
  mhd_config cfg;
  mhd::Grid grid;
  size_t esize;          // bytes per state element (8 or 4)
  size_t state_bytes;    // 9 * ncell * esize
  char* ws;
  size_t ws_bytes;
  void* Ua;              // U^n (and U^{n+1}, in place)
  void* Ub;              // U1 / staging
  void* Uc;              // U2 of SSP-RK3 (rk_order 3), else null
  // constrained transport (cfg.divb == MHD_DIVB_CT), else null: the face
  // fields belonging to Ua / Ub / Uc, the CT buffer of the stage kernels and
  // the edge fields
  void* fa;
  void* fb;
  void* fc;
  void* ctf;
  void* edge;
  bool faces_set;
  mhd::Scalars* scal;
  double* partials;
  void* adj;             // adjoint scratch (MHD_FLAG_ADJOINT)
  size_t adj_bytes;
  cudaStream_t stream;
  bool have_state;
  bool lam_valid;
  // halo faces (a side with MHD_BC_HALO) and the staged step of
  // mhd_step_begin / mhd_step_stage: a step is open between the two, and
  // stage_next is the next stage's index in the step's stage sequence
  bool has_halo;
  bool step_open;
  int stage_next;
  bool stage1_valid;     // U_b holds the last step's first stage (mhd_get_stage1)
  double inv_dx_sum, dh_min;
  // mhd_step_host: a transfer stream and its events (made on first use), and
  // the z-chunk depth of the last stage's half launches
  bool xfer_ready;
  cudaStream_t xfer;
  cudaEvent_t xev[12];
  int tz_half;
  // mhd_step_n: a capture stream and the graph of graph_steps steps
  cudaStream_t cap;
  cudaGraphExec_t gexec;
  int graph_steps;
  // CUDA-event timing (mhd_profile_enable)
  bool prof_on;
  struct Rec { cudaEvent_t a, b; int kind; };
  std::vector<Rec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  char err[512];
};
