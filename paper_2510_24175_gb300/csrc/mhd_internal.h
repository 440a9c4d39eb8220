// Host-side launcher interface between the C ABI (mhd_api.cu) and the kernel
// translation units.  Plain types only; every launcher enqueues on `stream`
// and returns the cudaError_t of the launch.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "mhd_stage.cuh"

namespace mhd {

// Message of a failing call that has no context (configuration checks,
// mhd_create, mhd_flux_batch, mhd_ensemble_create, the no-alloc sums): kept
// per host thread, returned by mhd_last_error(NULL).  Returns code.
int free_fail(int code, const char* fmt, ...);

// Geometry + physics of one context, shared by all launchers.
struct Grid {
  int n[3];
  int ndim;              // number of active dims (prefix x, y, z)
  long long ncell;       // nx * ny * nz
  int bc_lo[3], bc_hi[3];
  int limiter;
  double gamma, rho_floor, p_floor;
  double dx[3];
  int tz;                // z planes per CTA of the stage kernel
  int nsm;               // SM count of the device
};

template <class T>
Phys<T> make_phys(const Grid& g);

// Stage kernel (mhd_stage_f64.cu / mhd_stage_f32.cu).  stage 1: first stage;
// 2: last stage (combination with a_n, a_w + damping + wave-speed
// reduction); 3: SSP-RK3 middle stage (combination only).
// Constrained transport (bw, ctf non-null; 3-D): bw = the input's face field
// (three planes), ctf = the kCtPlanes-plane CT buffer.  3-D grids: the launch
// covers z planes [zlo, zhi) (zhi < 0: all) in chunks of tz planes per CTA
// (tz <= 0: the grid's own choice); the result of a cell does not depend on
// the decomposition.
template <class T>
cudaError_t launch_stage(const Grid& g, int stage, const T* win, const T* un, T* uout,
                         const StepScalars* sc, unsigned long long* lam_bits,
                         unsigned long long* floor_cnt, cudaStream_t stream,
                         double a_n = 0.5, double a_w = 0.5, const T* const* bw = nullptr,
                         T* ctf = nullptr, int zlo = 0, int zhi = -1, int tz = 0,
                         unsigned int* est_bits = nullptr);

// Constrained-transport kernels (mhd_ct.cu); face / edge arrays are three
// planes of ncell values, b_d on each cell's lower d-face.
template <class T>
cudaError_t launch_ct_edges(const Grid& g, const T* ctf, T* edge, cudaStream_t s);
// first: bout = bw - dt curl E; else bout = a_n bn + a_w (bw - dt curl E).
template <class T>
cudaError_t launch_ct_faces(const Grid& g, bool first, const T* edge, const T* bw, const T* bn,
                            T* bout, const StepScalars* sc, double a_n, double a_w,
                            cudaStream_t s);
// U's cell-centred B := face means; last: also the max wave speed into lam_bits.
template <class T>
cudaError_t launch_ct_cells(const Grid& g, bool last, const T* b, T* U,
                            unsigned long long* lam_bits, cudaStream_t s);
// U's cell-centred B := face means with the pressure kept (after a new face field).
template <class T>
cudaError_t launch_ct_set_cells(const Grid& g, const T* b, T* U, cudaStream_t s);
template <class T>
cudaError_t launch_ct_divb(const Grid& g, const T* b, unsigned long long* out_bits,
                           cudaStream_t s);

// Sets the shared-memory limit of every stage-kernel variant the grid
// launches (constrained transport or not), outside any stream capture.
template <class T>
cudaError_t prepare_stage_kernels(const Grid& g, bool ct);

// Shared-memory bytes and threads of the stage kernel for this grid.
template <class T>
void stage_shape(const Grid& g, size_t* smem, int* threads, int* ty);

// Auxiliary kernels (mhd_aux.cu).
struct PrepArgs {
  double dt_req, ch_req;  // > 0: use as given
  double cfl, inv_dx_sum, t_end, glm_alpha, dh_min;
  double dx[3];
  int active[3];
};
cudaError_t launch_prep(const PrepArgs& a, StepScalars* sc, unsigned long long* lam_bits,
                        unsigned int* est_bits, unsigned int* status, cudaStream_t stream);
// out[0..3] = (t, dt, c_h, steps) of the last step (device array).
cudaError_t launch_step_record(const StepScalars* sc, double* out, cudaStream_t stream);

// Maximum wave speed of a state into lam_bits (FP64 bits; both words cleared
// first).  FP32: every cell evaluated.  FP64: the two passes of
// mhd_physics.cuh (estimates into est_bits, then the exact evaluation of the
// cells that can hold the maximum).
template <class T>
cudaError_t launch_max_speed(const Grid& g, const T* U, unsigned long long* lam_bits,
                             unsigned int* est_bits, cudaStream_t stream);
// FP64 pass 1 over cells [c0, c1): the maximum reliable estimate, accumulated
// into est_bits (not cleared first).
cudaError_t launch_speed_estimate(const Grid& g, const double* U, long long c0, long long c1,
                                  unsigned int* est_bits, cudaStream_t stream);
// FP64 pass 2 over all cells: the exact maximum of the cells whose estimate
// reaches 0.999 of *est_bits or is not reliable, accumulated into lam_bits.
cudaError_t launch_speed_exact(const Grid& g, const double* U, const unsigned int* est_bits,
                               unsigned long long* lam_bits, cudaStream_t stream);

template <class T>
cudaError_t launch_sums(const Grid& g, const T* U, double* partials, int nblocks,
                        double* out8, cudaStream_t stream);

// U (type T) <- V (double), prim -> cons computed in FP64 per cell.
template <class T>
cudaError_t launch_prim_to_cons(const Grid& g, const double* V, T* U, cudaStream_t stream);
// In place: U (type T) holds primitives on entry, conservatives on exit.
template <class T>
cudaError_t launch_prim_to_cons_inplace(const Grid& g, T* U, cudaStream_t stream);
// V (double) <- cons -> prim of U (type T).
template <class T>
cudaError_t launch_cons_to_prim(const Grid& g, const T* U, double* V, cudaStream_t stream);
// Elementwise conversions.
cudaError_t launch_f64_to_f32(const double* in, float* out, long long n, cudaStream_t stream);
cudaError_t launch_f32_to_f64(const float* in, double* out, long long n, cudaStream_t stream);

// Stage kernels with halo faces (mhd_stage_halo_f64.cu / _f32.cu): as
// launch_stage for a 3-D GLM grid, the ghost cells of every kBcHalo side read
// from halo[f] (f = 2 d + side; layout at halo_cell in mhd_stage.cuh; halo
// may be null when no side is kBcHalo).  FP64 3-D GLM grids always run these
// kernels (launch_stage forwards), so that a grid and the blocks of its
// decomposition execute the same code and agree bit for bit.
template <class T>
cudaError_t launch_stage_halo(const Grid& g, int stage, const T* win, const T* un, T* uout,
                              const StepScalars* sc, unsigned long long* lam_bits,
                              unsigned long long* floor_cnt, cudaStream_t stream, double a_n,
                              double a_w, const T* const* halo, unsigned int* est_bits,
                              int zlo = 0, int zhi = -1, int tz = 0);
template <class T>
cudaError_t prepare_stage_kernels_halo(const Grid& g);

// The gh interior layers of W next to face f (f = 2 d + side) into dst, in the
// layout of the halo buffer of the opposite face of the neighbour across f.
template <class T>
cudaError_t launch_halo_pack(const Grid& g, const T* W, int face, int gh, T* dst,
                             cudaStream_t stream);
// atomicMax of the wave-speed word *lam_bits (FP64 bits; a NaN made the
// canonical quiet NaN, a negative zero +0) into *dst.
cudaError_t launch_lambda_max_into(const unsigned long long* lam_bits, unsigned long long* dst,
                                   cudaStream_t stream);

template <class T>
cudaError_t launch_flux_batch(const T* VL, const T* VR, T* F, long long nface, int dir,
                              double ch, double gamma, cudaStream_t stream);

// Measured FP64 fused multiply-add throughput of the current device (see
// mhd_fp64_fma_rate).
cudaError_t measure_fma_rate(cudaStream_t stream, unsigned warp_mask, double out[3]);

}  // namespace mhd
