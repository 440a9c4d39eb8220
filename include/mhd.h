/*
 * mhd.h -- C ABI of the GB300 GLM-MHD hot path.
 *
 * One call of mhd_step() advances a 3-D Cartesian grid of the 9-variable
 * ideal-MHD + GLM system by one two-stage Runge-Kutta step.  Each stage runs
 * the five per-stage steps of the paper (Section 3.2, "Porting of gPLUTO"):
 * boundary calculation (ghost zones), conservative->primitive map,
 * reconstruction of interface values (PLM, minmod or MC limiter), Riemann
 * solver (HLLD, Section 4.2) and the right-hand side of the conservation law,
 * with divergence cleaning (GLM, Section 4.2 strong-scaling paragraph) as the
 * div-B control.  The CFL time step is a global max-wavespeed reduction.
 *
 * Conventions shared by every entry point
 *   - Variables: conservative U = (rho, mx, my, mz, Bx, By, Bz, E, psi),
 *     primitive V = (rho, vx, vy, vz, Bx, By, Bz, p, psi);
 *     E = p/(gamma-1) + rho|v|^2/2 + |B|^2/2 (4 pi absorbed into B).
 *   - User arrays are interior-only SoA float64, index
 *     [var][z][y][x] with x fastest, shape 9 x nz x ny x nx (no ghosts).
 *   - Dimensions with n == 1 are inactive: no ghosts, no fluxes, no dt term.
 *   - The library never allocates device memory.  The caller passes one
 *     device workspace of mhd_workspace_bytes() bytes (256-byte aligned) that
 *     holds the state; the library keeps no pointer to user arrays after a
 *     call returns.
 *   - All device work is enqueued on the context's CUDA stream and is
 *     asynchronous, except the calls documented as synchronising.
 *   - Return value: MHD_OK (0) or a negative MHD_ERR_* code; the context keeps
 *     a message for mhd_last_error() (calls without a context keep it per host
 *     thread: mhd_last_error(NULL)).  Device-side faults of the numerics
 *     (non-finite state or time step) are recorded in a device status word and
 *     reported as MHD_ERR_NONFINITE by the next synchronising call.  No kernel
 *     traps.
 */
#ifndef MHD_H
#define MHD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MHD_OK = 0,
  MHD_ERR_INVALID = -1,   /* bad argument or configuration */
  MHD_ERR_NOMEM = -2,     /* workspace too small */
  MHD_ERR_CUDA = -3,      /* a CUDA runtime call failed */
  MHD_ERR_NONFINITE = -4, /* the device saw a non-finite state or time step */
  MHD_ERR_TIMEOUT = -5,   /* a bounded device wait gave up */
  MHD_ERR_STATE = -6      /* call out of order (e.g. step before set_state) */
};

/* Reconstruction: flat (first order), PLM with minmod or MC limiter, or
 * WENO-Z (Borges et al. 2008; the reconstruction of the paper's runs,
 * Section 4.2; needs active dimensions of at least 3 cells). */
enum { MHD_LIM_FLAT = 0, MHD_LIM_MINMOD = 1, MHD_LIM_MC = 2, MHD_LIM_WENOZ = 3 };
/* Boundary conditions of a side.  MHD_BC_HALO: the side is a subdomain
 * boundary of a decomposed grid -- its ghost cells are supplied by the caller
 * before every stage (mhd_step_stage), the paper's boundary exchange between
 * processes (Section 3.2); needs three active GLM dimensions (not the
 * adjoint), and may face MHD_BC_OUTFLOW or MHD_BC_HALO on the other side. */
enum { MHD_BC_PERIODIC = 0, MHD_BC_OUTFLOW = 1, MHD_BC_HALO = 2 };
/* MHD_FP64: all arithmetic in FP64.  MHD_FP32: FP32 state and stage
 * arithmetic; FP64 for the time-step reduction result and dt, the
 * conservation sums, and the pressure-floor branch of cons->prim. */
enum { MHD_FP64 = 0, MHD_FP32 = 1 };
enum { MHD_HOST = 0, MHD_DEVICE = 1 };
enum { MHD_CONS = 0, MHD_PRIM = 1 };
/* mhd_config.flags */
enum { MHD_FLAG_ADJOINT = 1 };
/* Divergence control (Section 3.2: one of several mutually exclusive
 * algorithms; Section 4.2: divergence cleaning in the strong-scaling runs,
 * constrained transport in the weak-scaling runs).
 * MHD_DIVB_GLM: Dedner et al. (2002) mixed GLM cleaning with the psi field.
 * MHD_DIVB_CT: constrained transport (Evans & Hawley 1988): a staggered
 *   face field b (b_d on each cell's lower d-face) advanced by Faraday's law
 *   with edge electric fields from the upwind CT-contact average of Gardiner
 *   & Stone (2005); the face divergence is preserved to round-off; psi is
 *   identically 0; the cell-centred B of the state is the mean of each
 *   cell's two faces.  Needs three active dimensions and periodic boundaries;
 *   not available for the adjoint or the ensemble. */
enum { MHD_DIVB_GLM = 0, MHD_DIVB_CT = 1 };

typedef struct mhd_config {
  int n[3];              /* nx, ny, nz >= 1; active dims need n >= 2          */
  double xmin[3], xmax[3]; /* domain; dx_d = (xmax_d - xmin_d) / n_d          */
  double gamma;          /* adiabatic index > 1                               */
  double cfl;            /* Courant number of the dt rule (0, 1]              */
  double glm_alpha;      /* GLM damping: psi *= exp(-alpha c_h dt / dh_min)   */
  double rho_floor;      /* absolute floors of cons->prim (counted)           */
  double p_floor;
  double t_end;          /* > 0: CFL steps are clamped to end exactly at t_end */
  int limiter;           /* MHD_LIM_* (reconstruction)                        */
  int bc[6];             /* MHD_BC_* for x-, x+, y-, y+, z-, z+ (periodic must
                            be set on both sides of a dimension)              */
  int precision;         /* MHD_FP64 or MHD_FP32                              */
  int flags;             /* MHD_FLAG_* (ADJOINT reserves adjoint buffers)     */
  int rk_order;          /* 2: RK2 (default); 3: SSP-RK3 of Shu & Osher,
                            the time integrator of the paper's runs          */
  int divb;              /* MHD_DIVB_GLM (default) or MHD_DIVB_CT             */
  double dx[3];          /* > 0: the cell size of dimension d as given (a block
                            of a decomposed grid passes the whole grid's, so
                            its steps round as the whole grid's do); 0 (the
                            default): (xmax_d - xmin_d) / n_d                 */
} mhd_config;

typedef struct mhd_ctx mhd_ctx;

/* Fills *cfg with defaults: gamma 5/3, cfl 0.8, glm_alpha 0.1, floors 1e-12,
 * MC limiter, periodic BCs, FP64, RK2, GLM, unit domain, n = (1,1,1). */
int mhd_config_default(mhd_config* cfg);

/* Device workspace the context needs for cfg (bytes, before alignment). */
int mhd_workspace_bytes(const mhd_config* cfg, size_t* bytes);

/* Creates a context over the caller's device workspace (256-byte aligned,
 * at least mhd_workspace_bytes()).  stream: a cudaStream_t (NULL = legacy
 * default stream).  The context does not own the workspace; it must outlive
 * the context.  Host memory for the context object is allocated here and
 * released by mhd_destroy(). */
int mhd_create(const mhd_config* cfg, void* d_workspace, size_t bytes, void* stream,
               mhd_ctx** out);

/* Replaces the stream later calls enqueue on. */
int mhd_set_stream(mhd_ctx* ctx, void* stream);

/* Sets the state from a float64 array U (where = MHD_HOST or MHD_DEVICE),
 * kind = MHD_CONS (conservative) or MHD_PRIM (primitive, converted on the
 * device).  In FP32 mode values are rounded to FP32 (primitive input from the
 * host is rounded before the conversion).  Resets the time to 0. */
int mhd_set_state(mhd_ctx* ctx, const double* U, int where, int kind);

/* Copies the state out as float64 (conservative; kind = MHD_PRIM converts on
 * the device and needs where = MHD_DEVICE).  where = MHD_HOST synchronises. */
int mhd_get_state(mhd_ctx* ctx, double* U, int where, int kind);

/* MHD_DIVB_CT only.  Sets the staggered face field from a float64 array b of
 * [3][nz][ny][nx] (where = MHD_HOST or MHD_DEVICE): b[d] holds the normal
 * field on each cell's lower d-face (at x_d = xmin_d + i_d dx_d).  Rounded to
 * FP32 in FP32 mode.  The state's cell-centred B becomes the mean of each
 * cell's two faces and its total energy is changed by the magnetic-energy
 * difference, so the pressure is kept (a state whose B already equals the
 * face means is unchanged).  Needs a state (mhd_set_state first); every
 * mhd_set_state must be followed by a face field before mhd_step.  The field
 * should be divergence free (mhd_divb_max): constrained transport preserves
 * whatever divergence it starts with. */
int mhd_set_face_field(mhd_ctx* ctx, const double* b, int where);

/* MHD_DIVB_CT only: copies the face field out as float64 [3][nz][ny][nx].
 * where = MHD_HOST synchronises. */
int mhd_get_face_field(mhd_ctx* ctx, double* b, int where);

/* MHD_DIVB_CT only: max over cells of |sum_d (b_d(+1/2) - b_d(-1/2)) / dx_d|
 * of the face field, computed in FP64.  Synchronises. */
int mhd_divb_max(mhd_ctx* ctx, double* out);

/* CFL time step of the current state (Section 3.2's explicit scheme; the rule
 * is lambda = max over cells and active d of |v_d| + c_f,d, c_h = lambda,
 * dt = cfl / (c_h sum_d 1/dx_d)).  Synchronises.  Either pointer may be NULL. */
int mhd_dt(mhd_ctx* ctx, double* dt, double* ch);

/* One Runge-Kutta step (Section 3.2: every stage runs the five steps listed
 * at the top of this file to form L; SSP-RK3 is the integrator of the
 * paper's runs, Section 4.2).  RK2:  U1 = U + dt L(U);  U' = (U + U1 + dt L(U1))/2.
 * SSP-RK3 (rk_order 3):  U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));
 * U' = 1/3 U + 2/3 (U2 + dt L(U2)).  GLM: then psi' *= exp(-glm_alpha c_h dt /
 * dh_min).  CT: the face field takes the same stages (its L is -curl E), and
 * c_h only enters the (unused) psi flux.  dt > 0 and ch > 0 are used as
 * given; dt <= 0 uses the CFL rule on the device (clamped to t_end when
 * t_end > 0); ch <= 0 uses c_h = lambda of the current state.  Does not
 * synchronise: dt and c_h stay on the device (see mhd_step_info).  Contexts
 * with halo faces step with the staged calls (mhd_step_begin) instead:
 * MHD_ERR_STATE here. */
int mhd_step(mhd_ctx* ctx, double dt, double ch);

/* nsteps steps with the CFL time step and c_h = lambda, as nsteps calls of
 * mhd_step(ctx, 0, 0) (same results), launched as one CUDA graph: the steps'
 * launches are captured on a private stream the first time a given nsteps
 * is asked for (again when nsteps changes) and the graph is replayed on the
 * context's stream, so a small grid pays one launch instead of four per
 * step.  With profiling on (mhd_profile_enable) the steps are launched one
 * by one.  Asynchronous. */
int mhd_step_n(mhd_ctx* ctx, int nsteps);

/* One step of a state that lives in host memory: U_in (host, float64,
 * conservative, [9][nz][ny][nx]) becomes the context's state, is advanced by
 * mhd_step(dt, ch), and the result is copied to U_out (host; may be U_in).
 * The same result, time and counters as mhd_set_state(U_in, MHD_HOST,
 * MHD_CONS) + mhd_step(dt, ch) + mhd_get_state(U_out, MHD_HOST, MHD_CONS)
 * (the time restarts at 0).  FP64 3-D contexts with nz >= 8 overlap the copies
 * with the device work: U_in goes over in eight z slabs on a second stream,
 * made on first use, each followed by its part of the wave-speed reduction,
 * and the last Runge-Kutta stage runs as two half-depth launches whose
 * outputs are copied back while the other half computes.  Other contexts run
 * the three calls in sequence.  Page-locked host buffers (cudaHostAlloc /
 * cudaHostRegister) are needed for the overlap.  Synchronous: returns when
 * U_out holds the new state.  MHD_DIVB_CT is rejected (it needs a face field:
 * use the separate calls).  Not to be mixed with other work on the context's
 * state from other streams while it runs. */
int mhd_step_host(mhd_ctx* ctx, const double* U_in, double* U_out, double dt, double ch);

/* out[0] = time t, out[1] = dt and out[2] = c_h of the last step,
 * out[3] = steps taken since set_state.  Synchronises; reports
 * MHD_ERR_NONFINITE if the device flagged a non-finite dt or state. */
int mhd_step_info(mhd_ctx* ctx, double out[4]);

/* mhd_step_info without the synchronisation: enqueues a copy of (t, dt,
 * c_h, steps) of the last step into d_out, 4 doubles of device memory, on the
 * context's stream (e.g. to record a rollout's time steps without a host
 * round trip per step). */
int mhd_step_record(mhd_ctx* ctx, double* d_out);

/* Counters since set_state (synchronises), each counted once per Runge-Kutta
 * stage for every cell whose conversion of that stage's input (step 2 of
 * the stage, Section 3.2) took the branch; conversions inside the wave-speed
 * reduction are not counted:
 *   counters[0]: density floor (rho < rho_floor: rho = rho_floor);
 *   counters[1]: pressure floor (p < p_floor: p = p_floor);
 *   counters[2]: device status bits (non-zero: a non-finite dt or c_h);
 *   counters[3]: MHD_FP32 only: cells whose FP32 pressure fell below p_floor
 *                or below 1e-3 (gamma-1) E and was recomputed in FP64 (the
 *                floor decision then taken in FP64). */
int mhd_counters(mhd_ctx* ctx, long long counters[4]);

/* Conservation sums: sum over cells of (rho, mx, my, mz, E, Bx, By, Bz) times
 * the cell volume, accumulated in FP64 in a fixed order (deterministic).
 * Synchronises. */
int mhd_conserved_sums(mhd_ctx* ctx, double out[8]);

/* Interface flux for nface primitive face pairs along direction dir
 * (0 = x, 1 = y, 2 = z): GLM interface step (Dedner et al. 2002) then HLLD
 * (Miyoshi & Kusano 2005).  VL, VR, F: device arrays [9][nface] of float64
 * (precision = MHD_FP64) or float32 (MHD_FP32).  Enqueued on stream. */
int mhd_flux_batch(const void* VL, const void* VR, void* F, long long nface, int dir,
                   double ch, double gamma, int precision, void* stream);

/* Discrete adjoint of one RK2 step (reverse-mode derivative of mhd_step with
 * dt and c_h frozen):  lam_n = (dU^{n+1}/dU^n)^T lam_np1.  The paper has no
 * adjoint; this differentiates the step of Section 3.2 as mhd_step computes
 * it.  Needs RK2 and a
 * PLM limiter (MHD_LIM_FLAT / MINMOD / MC).
 * U_n: the step's input state; lam_np1, lam_n: adjoints; all device float64
 * arrays [9][nz][ny][nx].  lam_n may not alias lam_np1.  Needs a context
 * created with MHD_FLAG_ADJOINT and MHD_FP64.  Does not change the context's
 * state.  The slope derivatives are accumulated with FP64 atomics, so
 * results vary run to run in the last few bits. */
int mhd_adjoint_step(mhd_ctx* ctx, const double* U_n, const double* lam_np1, double* lam_n,
                     double dt, double ch);

/* The first Runge-Kutta stage U1 = U^n + dt L(U^n) of the context's last
 * step (mhd_step, mhd_step_n or mhd_step_host), so that a checkpointed
 * reverse pass can keep it beside U^n instead of recomputing it inside
 * mhd_adjoint_step_stage1.  Valid after an FP64 RK2 step with GLM; any
 * mhd_set_state / mhd_set_face_field clears it (MHD_ERR_STATE until the next
 * step).  U1: float64 [9][nz][ny][nx], host (where = MHD_HOST; synchronises)
 * or device (MHD_DEVICE; enqueued on the context's stream). */
int mhd_get_stage1(mhd_ctx* ctx, double* U1, int where);

/* mhd_adjoint_step with the step's first stage supplied: U1 is the state
 * mhd_get_stage1 returned after stepping U_n with the same dt and c_h (device
 * float64 [9][nz][ny][nx], not aliasing U_n or lam_n).  Same result as
 * mhd_adjoint_step(ctx, U_n, lam_np1, lam_n, dt, ch) up to the order of the
 * FP64 atomic accumulation both use (which varies run to run by a few ulp);
 * saves the recomputation of the first stage (one of the forward step's two
 * stage kernels).  A U1 that does not belong to U_n gives the adjoint about a
 * different trajectory; nothing checks it. */
int mhd_adjoint_step_stage1(mhd_ctx* ctx, const double* U_n, const double* U1,
                            const double* lam_np1, double* lam_n, double dt, double ch);

/* Per-kernel timing of the context's launches with CUDA events recorded on
 * the context's stream (off by default; the events are created on the host
 * when enabled).  Kernel classes: 0 = step prepare, 1 = first RK stage,
 * 2 = last RK stage, 3 = max-wave-speed reduction, 4 = middle stage of
 * SSP-RK3, 5 = constrained-transport edge / face / cell kernels (one record
 * per stage).  mhd_profile_read() synchronises, returns the launch count and
 * total milliseconds per class since the last read, and clears the record. */
int mhd_profile_enable(mhd_ctx* ctx, int enable);
int mhd_profile_read(mhd_ctx* ctx, long long counts[6], double ms[6]);

/* Conservation sums for callers that can't allocate device memory: a host
 * application whose GPU memory is owned by another allocator, or a code that
 * forbids allocations once its time loop runs.  The paper has no
 * counterpart; this is a library service.
 * Same result as mhd_conserved_sums() (up to the summation order) for a state
 * U held by the caller in device memory: float64 (cfg->precision = MHD_FP64)
 * or float32 (MHD_FP32), conservative, [9][nz][ny][nx]; out: 8 host doubles.
 * Needs no context and no workspace and allocates nothing: the scratch is a
 * fixed 1 MiB device array inside the library (16384 partial sums), which
 * every GPU that loads the library holds until the process exits.  Grids of
 * more than 16384 * 32768 cells are rejected with MHD_ERR_NOMEM.  Each call
 * looks up that array's device address on the current device (nothing is
 * cached, so a cudaDeviceReset between calls is harmless).  All calls share
 * the one array: calls that overlap on the GPU (other streams, other host
 * threads) race.  Enqueues on stream and synchronises it; a stream that is
 * being captured is refused with MHD_ERR_INVALID before anything is
 * enqueued. */
int mhd_conserved_sums_noalloc(const mhd_config* cfg, const void* U, double out[8],
                               void* stream);

/* ---------------------------------------------------------------------------
 * Staged steps and halo faces: a grid decomposed into blocks, one context
 * per block (in one process or one per GPU), advanced together.  Section 3.2:
 * the boundary exchange is the only communication between processes; the
 * method also needs the global maximum wave speed for the common dt and c_h.
 * Per step, for every block:
 *   lam = 0 (device 64-bit word); mhd_lambda_max_into(ctx, lam) for every
 *   block (then an allreduce(MAX) of lam across processes);
 *   mhd_step_begin(ctx, 0, 0, lam);
 *   per stage (2 for RK2, 3 for SSP-RK3): fill every halo face's buffer of
 *   every block (mhd_halo_pack of the neighbour across the face, into the
 *   buffer directly or through a send/receive), then mhd_step_stage(ctx,
 *   halo buffers) for every block.
 * Each block's cells then evolve bitwise as in the undecomposed grid.
 * Halo buffer of face f (f = 2 d + side: 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+):
 * mhd_halo_bytes() bytes of device memory owned by the caller, holding the
 * block's ghost cells on that side in the context's precision with the
 * grid's SoA layout restricted to the ghost slab: [9][nz][ny][g] for x faces,
 * [9][nz][g][nx] for y faces, [9][g][ny][nx] for z faces, g = 2 (PLM) or 3
 * (WENO-Z); layer l holds ghost index l - g (low side) or n_d + l (high
 * side).  The stage kernels read only face ghosts (no edge or corner cells).
 * ------------------------------------------------------------------------- */

/* Bytes of the halo buffer of face f (see above). */
int mhd_halo_bytes(const mhd_ctx* ctx, int face, size_t* bytes);

/* Packs the g interior layers of this block next to face f, taken from the
 * input of the next stage (U^n outside a staged step, then each stage's
 * output), into d_dst (device) with the layout of the halo buffer of the
 * opposite face of the block across f (whose extents in the two tangential
 * dimensions must equal this block's).  Enqueued on the context's stream. */
int mhd_halo_pack(mhd_ctx* ctx, int face, void* d_dst);

/* Raises *d_bits (device, 64-bit; zero it before the first block) to this
 * block's maximum wave speed lambda (reduced on the device first if the
 * state is new): the FP64 bit pattern, which orders like the value for the
 * non-negative speeds, so an integer maximum over blocks (atomic here, an
 * allreduce(MAX) of int64 or uint64 across processes) is the exact global
 * maximum.  A NaN speed is written as the canonical quiet NaN, which
 * dominates.  Not inside a staged step.  Enqueued on the context's stream. */
int mhd_lambda_max_into(mhd_ctx* ctx, void* d_bits);

/* Opens a step of a GLM context (with or without halo faces): dt and c_h as
 * in mhd_step (dt <= 0 or ch <= 0: the CFL rule), lambda taken from
 * d_lambda_bits (device word filled by mhd_lambda_max_into: the maximum over
 * all blocks) or, when NULL, from this context's own state.  Enqueues the
 * step-prepare kernel.  The step's stages follow with mhd_step_stage. */
int mhd_step_begin(mhd_ctx* ctx, double dt, double ch, const void* d_lambda_bits);

/* Runs the next stage of the open step, reading the ghost cells of every
 * MHD_BC_HALO side from d_halo[f] (device buffers of mhd_halo_bytes; entries
 * of other sides are ignored, d_halo may be NULL without halo faces).  The
 * last stage also applies the GLM damping and reduces this block's new
 * maximum wave speed, and closes the step.  Enqueued on the context's
 * stream; the buffers must hold the ghosts of this stage's input when the
 * stage runs (stream order). */
int mhd_step_stage(mhd_ctx* ctx, const void* const d_halo[6]);

/* ---------------------------------------------------------------------------
 * Batched ensemble: independent 3-D boxes (each with its own grid, domain,
 * boundary conditions and CFL time step) advanced together by ONE
 * persistent cooperative kernel launch per mhd_ensemble_step call, captured
 * in a CUDA graph.  Boxes must be 3-D and MHD_FP32.  Every box evolves
 * bitwise as it would under its own mhd_step calls (same tile code).  The
 * caller allocates one device workspace (mhd_ensemble_workspace_bytes,
 * 256-byte aligned).
 * ------------------------------------------------------------------------- */
typedef struct mhd_ensemble mhd_ensemble;
int mhd_ensemble_workspace_bytes(const mhd_config* cfgs, int nbox, size_t* bytes);
int mhd_ensemble_create(const mhd_config* cfgs, int nbox, void* d_workspace, size_t bytes,
                        void* stream, mhd_ensemble** out);
/* Same conventions as mhd_set_state / mhd_get_state, for box `box`;
 * set_state restarts that box's time and step count. */
int mhd_ensemble_set_state(mhd_ensemble* ens, int box, const double* U, int where, int kind);
int mhd_ensemble_get_state(mhd_ensemble* ens, int box, double* U, int where, int kind);
/* nsteps CFL steps of every box in one persistent launch (per step: per-box
 * dt and c_h, stage 1, grid barrier, stage 2, grid barrier).  Asynchronous. */
int mhd_ensemble_step(mhd_ensemble* ens, int nsteps);
/* out[0] = t, out[1] = dt, out[2] = c_h, out[3] = steps of box `box`,
 * out[4] = its z-chunk depth, out[5] = 1 if launches are graph-captured,
 * out[6] = its tile height (column tiles of 32 x out[6] cells).
 * Synchronises; MHD_ERR_NONFINITE if the box saw a non-finite dt. */
int mhd_ensemble_info(mhd_ensemble* ens, int box, double out[7]);
/* Tile shape: column tiles of 32 x ty cells (ty = 8 or 4; the tile height of
 * the launch, so it applies to every box) marching z chunks of tz planes for
 * box `box` (clamped to its nz).  Every tile shape gives the same results
 * bit for bit; only the speed differs.  Synchronises. */
int mhd_ensemble_set_tiles(mhd_ensemble* ens, int box, int ty, int tz);
/* Timing autotuner: the launch's tile height {8, 4}, then for each box-size
 * class the z-chunk depth {4, 8, 16, 32, 64} (one pass of coordinate
 * descent over the classes; each candidate the best of two timed
 * trial_steps-step launches, kept only when more than 1 % faster).  Every
 * box evolves bitwise alike under any tile shape.  ADVANCES every box by the
 * trial steps: save and restore the states around it.  Synchronises. */
int mhd_ensemble_autotune(mhd_ensemble* ens, int trial_steps);
const char* mhd_ensemble_last_error(const mhd_ensemble* ens);
int mhd_ensemble_destroy(mhd_ensemble* ens);

/* ---- Diagnostics ----------------------------------------------------------
 * Measured FP64 throughput of the current device, the denominator of the
 * FP64 stage kernels' roofline (their bound is the SM's FP64 unit, not HBM):
 * one CTA of 8 warps per SM; every thread of the warps that warp_mask selects
 * (bit w: warp w; warp w runs on scheduler w mod 4; 0 or 0xff: all 8) runs 16
 * independent fused multiply-add chains, timed with CUDA events on `stream`
 * (NULL: the legacy default stream) after one warm-up launch.  out[0] =
 * lane-FMAs per second over the device, out[1] = lane-FMAs per clock per SM
 * at the clock rate the device reports, out[2] = milliseconds of the timed
 * launch.  Allocates and frees (SM count x 256) doubles of device memory;
 * synchronises with the stream.  Errors: MHD_ERR_INVALID (out NULL),
 * MHD_ERR_CUDA (message in mhd_last_error(NULL)). */
int mhd_fp64_fma_rate(void* stream, unsigned warp_mask, double out[3]);

/* Launch planning, on the host only (no GPU, no CUDA call): the z-chunk depth
 * *tz (planes per CTA) that the 3-D stage launches of an n[0] x n[1] x n[2]
 * grid use, for column tiles of 32 x ty cells (ty: 8 for the PLM kernels, 4
 * for FP64 WENO-Z, 8 for FP32 WENO-Z) on nsm SMs holding ctas_per_sm stage
 * CTAs each (1 for FP64 and FP32 WENO-Z, 2 for FP32 PLM), and, if span is not
 * NULL, the modelled duration of one launch in plane iterations.  The model:
 * the CTAs start in launch order -- every column tile's full chunks, then
 * every column tile's last, possibly shorter, chunk -- each on the slot that
 * frees first, and a CTA takes its planes plus one for its warm-up; the
 * depth is the candidate (256, 192, 128, 96, 80, 64, 56, 48, 40, 32, 24, 20,
 * 16, 12, 8, 4; at most n[2], or 4) with the shortest launch, the deeper one
 * on a tie.  A grid with an extent of 1 is not 3-D: *tz = 1.  The paper has
 * no counterpart: this is how the library spreads its stage launches over
 * the SMs.  Errors: MHD_ERR_INVALID (an extent, ty, nsm or ctas_per_sm below
 * 1, n or tz NULL; message in mhd_last_error(NULL)). */
int mhd_plan_z_chunks(const int n[3], int ty, int nsm, int ctas_per_sm, int* tz,
                      double* span);

/* Message of the last failing call on ctx (never NULL).  ctx = NULL: the
 * message of the calling host thread's last failing call that has no context
 * (mhd_workspace_bytes, mhd_create, mhd_flux_batch, mhd_ensemble_create,
 * mhd_ensemble_workspace_bytes, mhd_conserved_sums_noalloc, mhd_fp64_fma_rate,
 * mhd_plan_z_chunks). */
const char* mhd_last_error(const mhd_ctx* ctx);

/* Releases the context (not the workspace). */
int mhd_destroy(mhd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MHD_H */
