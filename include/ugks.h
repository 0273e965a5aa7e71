/*
 * ugks.h -- C ABI of the GB300 (sm_103a) library for the explicit 2D Unified Gas-Kinetic
 * Scheme step of Liu, Hu & Li, "Performance Comparison on Parallel CPU and GPU Algorithms
 * for Unified Gas-Kinetic Scheme" (arXiv:1810.08137).
 *
 * One step (ugks_step) is, for every cell and discrete velocity (Sec. 2):
 *   - the interface distribution of the BGK integral solution (Eq. 2), built per interface by
 *     the flux steps S1-S8 of the Sec. 2.B table (velocity moments, Maxwellian moments, time
 *     weights, micro slopes, equilibrium and free-transport flux parts, micro flux);
 *   - the conservative update of the macroscopic variables W = (rho, rho U, rho V, rho E)
 *     (Eq. 4);
 *   - the implicit (trapezoidal collision term) update of the distribution function (Eq. 3).
 * The problem statement -- mesh, velocity grid, tau, CFL, wall and inlet/outlet conditions --
 * is the one of Sec. 2 and Sec. 3.A (2D pressure-driven channel).
 *
 * Conventions for every call:
 *   - The library owns all device memory it uses; host pointers are only read or written
 *     during the call (the data is copied).  Device pointers passed to *_device calls must
 *     stay valid until the call's work on the handle's stream has completed.
 *   - Every call returns a status; ugks_last_error() gives a text for the last failure on a
 *     handle.  No call aborts the process or traps the device.
 *   - Work is enqueued on the CUDA stream given at creation (NULL: the legacy default
 *     stream).  Calls that return data to the host synchronise that stream.
 *   - Numerical failure (rho <= 0, T <= 0 or NaN in a cell) is recorded on the device and
 *     reported as UGKS_ENUMERIC by the next synchronising call.
 *
 * Host array layouts (the same for both precisions; FP32 storage converts on copy):
 *   cell index   c = j*nx + i                 (x fastest), 0 <= i < nx, 0 <= j < ny
 *   velocity     q = m*nu + k                 (u fastest), u_k, v_m
 *   f[c][q][2]   double; component 0 = h = int f dxi, component 1 = b = int xi^2 f dxi
 *                (reduced distributions over the K internal degrees of freedom)
 *   W[4][c]      double; rho, rho U, rho V, rho E
 */
#ifndef UGKS_H
#define UGKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  UGKS_OK = 0,
  UGKS_EINVAL = 1,    /* invalid argument or configuration */
  UGKS_ENOMEM = 2,    /* device allocation failed */
  UGKS_ECUDA = 3,     /* a CUDA runtime call failed */
  UGKS_ETIMEOUT = 4,  /* a bounded device wait gave up: a grid barrier of the batch's
                         persistent step (ugks_batch_sync), or the FP32-f update walk's wait
                         for its asynchronous record copies (next synchronising call) */
  UGKS_ENUMERIC = 5   /* rho <= 0, T <= 0 or NaN appeared in a cell */
} ugks_status;

typedef enum {
  UGKS_BC_PERIODIC = 0,  /* wrap around */
  UGKS_BC_WALL = 1,      /* diffuse isothermal wall: zero net mass flux, wall Maxwellian */
  UGKS_BC_PRESSURE = 2   /* ghost Maxwellian (rho_bc, U and V of the adjacent cell, T_bc) */
} ugks_bc_kind;

typedef enum {
  UGKS_FP64 = 0,   /* f stored and transported in FP64, all arithmetic FP64 */
  UGKS_FP32F = 1   /* f stored and transported in FP32 as f - g_ref.  FP64 for: the
                      velocity-space moment accumulation (FP32 products summed over chunks
                      of at most 8 rows of one warp, every sum across chunks in FP64, then
                      the exact FP64 sums of g_ref added), the interface scalars S2-S5 (W0,
                      primitive variables, half-range moments, Mt1..Mt5 including the
                      exp(-dt/tau) series at small tau, the micro-slope solves a_L, a_R, b, A,
                      the macroscopic flux), the conservative W update (Eq. 4), the cell
                      coefficients of Eq. 3 and the exponents of the collision and wall
                      Maxwellians relative to g_ref.  FP32 for the per-velocity work on f:
                      reconstruction, micro flux and the Eq. 3 update, from FP32 records of
                      those FP64 coefficients */,
  UGKS_DF64 = 2    /* FP64-accurate, on the FP32 pipe: f stored as double-FP32 pairs (an
                      unevaluated sum of two FP32 numbers, about 48 significand bits) and
                      every per-velocity operation (van Leer slopes, velocity sums, micro
                      flux, Eq. 3) in double-FP32 arithmetic built from error-free
                      transformations; interface and cell scalars (S2-S5, Eq. 4) in FP64.
                      Meets the FP64 form's tolerance (1e-12 per field per step) */
} ugks_precision;

enum { UGKS_SIDE_W = 0, UGKS_SIDE_E = 1, UGKS_SIDE_S = 2, UGKS_SIDE_N = 3 };

typedef struct {
  int kind;      /* ugks_bc_kind */
  double rho;    /* UGKS_BC_PRESSURE: ghost density */
  double T;      /* UGKS_BC_PRESSURE: ghost temperature; UGKS_BC_WALL: wall temperature */
  double U;      /* UGKS_BC_WALL: tangential wall velocity */
} ugks_bc;

/* Problem statement (Sec. 2, Sec. 3.A).  Units: velocities in sqrt(2 k T0 / m), so the
 * Maxwellian of Eq. 1 is g = rho (lam/pi) exp(-lam((u-U)^2+(v-V)^2)) with lam = 1/T. */
typedef struct {
  int nx, ny;            /* cells, >= 1 each; uniform Cartesian mesh */
  double lx, ly;         /* domain size */
  int nu, nv;            /* discrete velocities per axis, >= 1, nu*nv <= 65536 */
  double umin, umax;     /* uniform grid including both ends, trapezoid weights */
  double vmin, vmax;
  int K;                 /* internal degrees of freedom, 0 <= K <= 8 (1: monatomic) */
  double kn;             /* Knudsen number; tau = mu/p, mu = mu_ref T^omega */
  double omega, alpha;   /* viscosity index and VSS alpha (0.5, 1.0: hard sphere) */
  double cfl;            /* dt = cfl / (max|u|/dx + max|v|/dy) when dt <= 0 */
  double dt;             /* > 0: fixed time step */
  ugks_bc bc[4];         /* W, E, S, N; periodic must be paired (W with E, S with N) */
  int precision;         /* ugks_precision */
  /* UGKS_FP32F only: reference Maxwellian g_ref(rho, U, V, T).  The FP32 buffers hold
   * f - g_ref and every velocity sum and flux adds the exact FP64 contribution of g_ref,
   * so FP32 rounding acts on the (small) deviation from it; a reference near the flow's
   * mean state keeps that deviation small.  ref_T <= 0 selects (1, 0, 0, 1).  The state
   * exchanged through this ABI is always f itself. */
  double ref_rho, ref_U, ref_V, ref_T;
  /* Prandtl number.  1 (or <= 0, the value of a zero-initialised config) selects the BGK
   * model of Eq. 1; any other value the Shakhov model, whose equilibrium
   * g+ = g [1 + (1 - Pr) (c.q) (c_t^2/RT - (D+2)) / ((D+2) p RT)] (D = 2 + K, c the
   * peculiar velocity, c_t^2 = |c|^2 + xi^2, q the heat flux, RT = 1/(2 lam)) replaces g in
   * the collision term.  The paper uses BGK; the Shakhov model follows the UGKS papers it
   * cites, with these readings: at an interface the heat flux of the upwind interface
   * values about the interface velocity, on the zeroth-order equilibrium term (Mt1) of the
   * integral solution; in Eq. 3 the heat flux of f^n in the g+ of both steps n and n+1.  Supported
   * by the UGKS_FP64 and UGKS_FP32F forms (UGKS_EINVAL for UGKS_DF64 and for
   * ugks_step_noalloc). */
  double pr;
} ugks_config;

typedef struct ugks_ctx* ugks_handle;

/* Validate cfg, build the velocity grid, weights and time step, allocate device state
 * (two copies of f with a two-cell ghost ring, W, per-cell velocity sums, per-face
 * coefficients).  cuda_stream: a cudaStream_t or NULL.  On success *out is a new handle.
 * Errors: UGKS_EINVAL (bad cfg, NULL out), UGKS_ENOMEM, UGKS_ECUDA. */
ugks_status ugks_create(const ugks_config* cfg, void* cuda_stream, ugks_handle* out);

/* Free everything owned by h (NULL is allowed). */
void ugks_destroy(ugks_handle h);

/* Text of the last error on h (never NULL; "" if none). */
const char* ugks_last_error(ugks_handle h);

/* Time step and velocity grid actually used: u[nu], v[nv], w[nq] (any may be NULL). */
ugks_status ugks_get_grid(ugks_handle h, double* dt, double* u, double* v, double* w);

/* Device bytes owned by h. */
size_t ugks_device_bytes(ugks_handle h);

/* Copy a state from host memory: f_host[nc][nq][2], W_host[4][nc] (layouts above).
 * Synchronises; the host arrays are only read during the call.  FP32-f form: page-locked
 * (pinned or registered) f_host is read in place by the conversion kernel; pageable memory
 * goes through a device staging buffer.  f_host must hold the whole array either way. */
ugks_status ugks_set_state(ugks_handle h, const double* f_host, const double* W_host);

/* Same from device memory (same layouts, FP64).  Enqueued; returns without waiting. */
ugks_status ugks_set_state_device(ugks_handle h, const double* f_dev, const double* W_dev);

/* Pointwise Maxwellian state built on the device from per-cell primitive fields
 * (host arrays of nc values): f = g(rho, U, V, T) per velocity, b = K T/2 h,
 * W = (rho, rho U, rho V, rho (|U|^2/2 + (K+2) T / 4)). */
ugks_status ugks_init_maxwellian(ugks_handle h, const double* rho, const double* U,
                                 const double* V, const double* T);

/* Advance nsteps explicit UGKS steps (Eq. 2-4).  Enqueued on the stream; returns without
 * waiting.  Errors found later surface at the next synchronising call.  The first call
 * captures the step's kernels into CUDA graphs (one per ping-pong parity, on a private
 * stream) and later calls replay them; while tracing is on (ugks_profile) the kernels are
 * launched directly instead. */
ugks_status ugks_step(ugks_handle h, int nsteps);

/* Wait for the stream and report a recorded failure: UGKS_ENUMERIC, or UGKS_ETIMEOUT when a
 * bounded device wait gave up.  A new state (ugks_set_state*, ugks_init_maxwellian) clears
 * the recorded failures. */
ugks_status ugks_sync(ugks_handle h);

/* Bound of the FP32-f update walk's wait for its asynchronous record copies, in polls of
 * the mbarrier (each suspends the waiting lanes for a hardware-chosen time; the default
 * 2^22 is at least about a second).  When a wait runs out the walk records it and returns
 * after draining its copies in flight; the next synchronising call reports UGKS_ETIMEOUT
 * and the state is undefined until set again.  No effect on the other forms.
 * Synchronises. */
ugks_status ugks_set_wait_limit(ugks_handle h, long long polls);

/* Velocity-space split of the FP32-f sums (S1 + S7 of the Sec. 2.B flux table; the paper's
 * large-velocity-space regime of Sec. 3.B): `warps` warps (1, 2 or 4) share each cell's
 * velocity space, each summing a contiguous range of velocity rows per half of the v axis,
 * and their FP64 face sums are added in shared memory in a fixed order.  0 selects the
 * automatic choice that ugks_create also makes: more warps per cell while the cells alone
 * would leave the kernel's resident warps under-filled (small meshes, large velocity
 * grids) and every warp keeps at least 16 velocity rows.  The result depends on `warps` only
 * through the order of the FP64 additions.  UGKS_EINVAL for other values or another form.
 * Synchronises; the next ugks_step captures its graphs again. */
ugks_status ugks_set_sums_split(ugks_handle h, int warps);
/* Current warps per cell of the FP32-f sums (0 for another form or a NULL handle). */
int ugks_get_sums_split(ugks_handle h);

/* Copy W (host W_host[4][nc]) and, if prim_host != NULL, primitive variables
 * prim_host[4][nc] = (rho, U, V, T).  Synchronises. */
ugks_status ugks_moments(ugks_handle h, double* W_host, double* prim_host);

/* Checkpoint: copy the full state (f_host[nc][nq][2], W_host[4][nc]).  Synchronises.
 * FP32-f form: page-locked f_host is written in place by the conversion kernel, pageable
 * memory through a device staging buffer. */
ugks_status ugks_get_state(ugks_handle h, double* f_host, double* W_host);

/* Same into device memory (FP64 layouts above).  Enqueued; returns without waiting. */
ugks_status ugks_get_state_device(ugks_handle h, double* f_dev, double* W_dev);

/* Residual of the last step, per component c of W:
 *   res[c] = sqrt(mean_cells (W_c^{n+1} - W_c^n)^2) / max(max_cells |W_c^{n+1}|, 1e-300).
 * Synchronises.  Before any step res[] = 0. */
ugks_status ugks_residual(ugks_handle h, double res[4]);

/* Tracing.  enable != 0: every later ugks_step records CUDA events on the handle's
 * stream around each of its kernels; enable == 0 stops recording and discards the
 * records.  ugks_kernel_times synchronises and returns, per kernel of the step (order:
 * ugks_kernel_name(0..UGKS_NKERNELS-1)), the launches recorded and their total device
 * time in ms.  ms and launches must hold UGKS_NKERNELS entries (either may be NULL). */
#define UGKS_NKERNELS 6
ugks_status ugks_profile(ugks_handle h, int enable);
ugks_status ugks_kernel_times(ugks_handle h, double* ms, long* launches);
const char* ugks_kernel_name(int i);

/* Device bytes ugks_create would allocate for cfg (0 if cfg is invalid). */
size_t ugks_state_bytes(const ugks_config* cfg);

/* Measured FP64 arithmetic rate of the current device (GFLOP/s, a fused multiply-add
 * counted as 2): independent chains of FP64 FMAs on every SM, best of three timed launches
 * on cuda_stream (NULL: the legacy stream).  A diagnostic for the FP64 form's roofline; the
 * paper has no counterpart.  Synchronises. */
ugks_status ugks_fp64_rate(void* cuda_stream, double* gflops);

/* ---- Batch of independent instances ------------------------------------------------
 * Many independent channel solves stepped together (the FP32-f form only): every phase of
 * the step runs once per step for all active instances, as a persistent grid over a
 * device-resident table of (instance, tile) work items, and one step of the whole batch
 * is one CUDA graph replay.  By default the step is ONE cooperative launch of a persistent
 * kernel that runs the six phases (ghost x, ghost y, sums, interfaces, cells, walk) with a
 * grid-wide barrier between them; ugks_batch_set_persistent(b, 0) selects seven phase
 * launches instead (the same phase code and order of work).  Instances are admitted into free slots while the batch is in
 * use (admission checks an HBM budget) and retired when done; the table and each
 * instance's ping-pong parity live in device memory, so admission and retirement change
 * data, not the captured graph.  Each instance's results are bitwise those of the same
 * instance stepped alone with ugks_step (same kernels, same order of work). */
typedef struct ugks_batch_ctx* ugks_batch;

/* max_slots <= 256 instances at a time; hbm_budget: total state bytes of the admitted
 * instances (0: no limit); cuda_stream: cudaStream_t or NULL. */
ugks_status ugks_batch_create(int max_slots, size_t hbm_budget, void* cuda_stream, ugks_batch* out);
void        ugks_batch_destroy(ugks_batch b);
const char* ugks_batch_last_error(ugks_batch b);
size_t      ugks_batch_bytes_used(ugks_batch b);

/* Admit one instance (cfg->precision must be UGKS_FP32F): allocates its state if it fits
 * the budget and a slot is free, writes the slot to *slot.  UGKS_ENOMEM: no budget or slot
 * left (nothing allocated); UGKS_EINVAL: bad cfg. */
ugks_status ugks_batch_admit(ugks_batch b, const ugks_config* cfg, int* slot);

/* Free a slot (waits for the batch's stream first). */
ugks_status ugks_batch_retire(ugks_batch b, int slot);

/* The instance in a slot, for the single-instance calls that move state and read results
 * (ugks_init_maxwellian, ugks_set_state(_device), ugks_get_state(_device), ugks_moments,
 * ugks_residual, ugks_sync).  Do not call ugks_step or ugks_destroy on it.  NULL if the
 * slot is free. */
ugks_handle ugks_batch_instance(ugks_batch b, int slot);

/* Advance every active instance by nsteps steps (one graph replay each).  Enqueued. */
ugks_status ugks_batch_step(ugks_batch b, int nsteps);

/* Wait for the batch's stream; UGKS_ENUMERIC if any instance recorded a failure;
 * UGKS_ETIMEOUT if a grid barrier of the persistent step gave up waiting since the last
 * call (the flag is cleared; the instances' states are then undefined and must be set
 * again before stepping). */
ugks_status ugks_batch_sync(ugks_batch b);

/* Step mode: enable != 0, one cooperative launch per step (the default where the device
 * supports cooperative launch); 0, seven phase launches.  Synchronises; UGKS_EINVAL if
 * cooperative launch is unavailable. */
ugks_status ugks_batch_set_persistent(ugks_batch b, int enable);
int         ugks_batch_get_persistent(ugks_batch b);

/* Bound of every wait at the persistent step's grid barriers, in polls of about 0.13 us
 * (default 8e6, about 1 s).  A block that waits longer, or that sees another block give
 * up, ends the launch; ugks_batch_sync then reports UGKS_ETIMEOUT.  Synchronises. */
ugks_status ugks_batch_set_wait_limit(ugks_batch b, unsigned long long polls);

/* Tile shape of the f-update walk for one slot: the cell tile (rows per tile; a tile is
 * 4 columns wide) and the velocity tile (chunks of 32 velocity slots walked by consecutive
 * warps for the same cell tile; 0 = all chunks of the cell).  The autotuner: for each
 * velocity-grid class present (nu*nv <= 576, <= 1600, <= 4096, larger) it times
 * trial_steps batch steps for every cell tile of 16, 32, 64, 128 rows times velocity tile
 * of all, 2 and 1 chunks, and keeps the fastest for that class; then it times the step
 * in both modes (ugks_batch_set_persistent) and keeps the faster.  Neither the tile shape
 * nor the mode changes the arithmetic, so tuning steps are real steps of every active
 * instance (each advances by 12 (trial_steps + 1) per class present, plus
 * 2 (trial_steps + 1)).  *best_ms: time per batch step in the chosen mode (may be NULL). */
ugks_status ugks_batch_set_walk_rows(ugks_batch b, int slot, int rows);
int         ugks_batch_get_walk_rows(ugks_batch b, int slot);
ugks_status ugks_batch_set_walk_vtile(ugks_batch b, int slot, int chunks);
int         ugks_batch_get_walk_vtile(ugks_batch b, int slot);
ugks_status ugks_batch_tune(ugks_batch b, int trial_steps, double* best_ms);

/* One FP64 UGKS step on caller-owned device buffers that allocates no device memory.
 * For callers that cannot call cudaMalloc at all -- code running where the CUDA allocator
 * is off limits, such as inside a host framework that owns every device allocation, or
 * where an allocation could block or fail at an awkward time -- and who therefore cannot
 * use ugks_create.  The paper has no counterpart; it is an interface convenience.
 *   cfg          problem statement; cfg->precision must be UGKS_FP64, and the collision
 *                model BGK (cfg->pr <= 0 or 1: the Shakhov model's extra sums need
 *                ugks_create).
 *   f_in, W_in   device state at t^n, layouts f[nc][nq][2], W[4][nc] (FP64), read only.
 *   f_out, W_out device buffers for t^{n+1}, same layouts; must not overlap the inputs.
 *   cuda_stream  cudaStream_t or NULL.  The call is synchronous: it waits for its own work
 *                on that stream before returning, and reports UGKS_ENUMERIC for rho <= 0,
 *                T <= 0 or NaN in a cell.
 * All intermediates live in one fixed device array inside the library, of
 * UGKS_NOALLOC_SCRATCH_BYTES bytes, that every GPU which loads the library holds until the
 * process exits.  Problems whose intermediates do not fit are rejected with UGKS_EINVAL and
 * a message on stderr; the need is about 32 (nx+4)(ny+4) nu nv + 1000 (nx+2)(ny+2) bytes.
 * Every call made outside stream capture looks up that array's device address
 * (cudaGetSymbolAddress), so a device reset or a recreated context is picked up by the
 * next such call; a call made while its stream is being captured uses the address found by
 * the last call outside capture on that device (none: UGKS_ECUDA).  So make the first call
 * on a device, and the first call after a reset, before any stream capture.  Every call
 * shares the array: calls that overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.
 * Errors: UGKS_EINVAL (bad or oversize cfg, pr != 1, NULL pointer), UGKS_ECUDA, UGKS_ENUMERIC. */
#define UGKS_NOALLOC_SCRATCH_BYTES (64u << 20)
ugks_status ugks_step_noalloc(const ugks_config* cfg, const double* f_in, const double* W_in,
                              double* f_out, double* W_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
