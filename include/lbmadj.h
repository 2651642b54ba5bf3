/*
 * lbmadj -- windowed regularized lattice-Boltzmann LES and its discrete adjoint
 * on one NVIDIA B300 (sm_103a).
 *
 * The library advances a D2Q9 or D3Q19 lattice with the regularized BGK
 * collision and Smagorinsky eddy viscosity (Sec. 2.1.2, Eqs. 9-16), partial
 * bounce-back driven by a design field (Sec. 2.2, Eq. 23), streaming and
 * boundary rules (Sec. 2.1.3, Eqs. 19-21), one time window at a time.  It
 * samples a window-averaged objective and a monitored quantity (Sec. 3.1-3.3,
 * Eqs. 24-27, 42), evaluates the consecutive-window test (Eq. 26), sweeps the
 * discrete adjoint backward over the last window (Eqs. 30-39) with checkpoint
 * recompute, and accumulates the design sensitivity (Eq. 40).
 *
 * Conventions shared by every call:
 *  - Every function returns an lbm_status; nothing throws across the ABI.
 *    lbm_last_error() gives a one-line reason for the last failure on the
 *    calling thread.
 *  - The caller owns every buffer, including the device workspace passed to
 *    lbm_create; the library makes no device allocation of its own.  The
 *    context itself is a small host object freed by lbm_destroy.
 *  - All device work is enqueued on the CUDA stream given to lbm_create.
 *    Calls that return host scalars synchronise that stream before returning.
 *  - Population order: D2Q9 in the paper's order (Eq. 2): c0=(0,0), c1=(1,0),
 *    c2=(0,1), c3=(-1,0), c4=(0,-1), c5=(1,1), c6=(-1,1), c7=(-1,-1),
 *    c8=(1,-1).  D3Q19: c0 rest; c1..c6 = +x,-x,+y,-y,+z,-z; c7..c18 =
 *    (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),
 *    (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1).
 *  - Node index i = x + nx*(y + ny*z).  Population arrays are [Q][N] with N
 *    = nx*ny*nz (structure of arrays, x fastest).
 *  - Pointers documented "host or device" may point to either; the library
 *    tells them apart through unified addressing.
 *  - The design field gamma is the solid fraction (1 = solid); the paper's
 *    design variable is phi = 1 - gamma.  Gradients returned are dJ/dgamma.
 */
#ifndef LBMADJ_H
#define LBMADJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,        /* invalid argument or configuration (nothing changed) */
  LBM_ERR_WORKSPACE = 2,  /* workspace pointer misaligned or too small           */
  LBM_ERR_CUDA = 3,       /* a CUDA runtime call failed                          */
  LBM_ERR_STATE = 4,      /* call out of order (e.g. adjoint before a window)    */
  LBM_ERR_NONFINITE = 5,  /* a density <= 0 or a non-finite value was produced   */
  LBM_NOT_CONVERGED = 6   /* lbm_run_until_converged reached its window cap       */
} lbm_status;

enum { LBM_D2Q9 = 9, LBM_D3Q19 = 19 };
enum { LBM_FP32 = 0, LBM_FP64 = 1 };

/* Node classes.  Only nodes on the domain faces may be non-FLUID.
 *  WALL: on-node bounce-back; an unknown population takes the value of its
 *        opposite (Eq. 19); a link whose opposite is unknown too (a corner)
 *        takes its rest weight w_a.
 *  INLET: velocity inlet on the x=0 face with x-velocity inlet_u[z][y]:
 *        Zou-He (Eq. 20) for D2Q9; moving-wall bounce-back for D3Q19.
 *  OUTLET_PRESSURE: Zou-He pressure outlet (Eq. 21) on the x=nx-1 face,
 *        density rho_out; D2Q9 only.
 *  OUTLET_ZEROGRAD: unknown populations copied from the neighbour along the
 *        inward x normal, on the x=0 or x=nx-1 face. */
enum { LBM_FLUID = 0, LBM_WALL = 1, LBM_INLET = 2, LBM_OUTLET_PRESSURE = 3, LBM_OUTLET_ZEROGRAD = 4 };

/* Instantaneous objective j(t) = sum_i w_i psi_i (window mean: Eq. 27, 42).
 *  DISSIPATION:   psi = (tau_eff - 1/2) Pi:Pi / (2 rho cs^2 tau_eff^2)
 *  VELOCITY_DEV:  psi = |u - objective_uref|^2
 *  PRESSURE:      psi = cs^2 rho (signed weights give a pressure drop, Eq. 47)
 *  DRAG:          psi = sum_a c_xa F_a with F from Eq. 23 (Eq. 44) */
enum { LBM_OBJ_DISSIPATION = 0, LBM_OBJ_VELOCITY_DEV = 1, LBM_OBJ_PRESSURE = 2, LBM_OBJ_DRAG = 3 };

/* Monitored quantity of the window test: the drag coefficient of Eq. 25,
 * sum_i sum_a c_xa F_a / (rho_out monitor_u^2 monitor_l / 2), or j itself. */
enum { LBM_MON_DRAG = 0, LBM_MON_OBJECTIVE = 1 };

/* Checkpoint storage for the adjoint's recompute:
 *  NATIVE: the carried field in the working precision (Q values per node).
 *  FP16, BF16: the deviation from equilibrium in 16 bits with one power-of-two
 *        scale per block of nodes plus FP32 density and momentum (lossy; FP32
 *        solver only).
 *  MOMENT: lossless and smaller (a library design with no counterpart in the
 *        paper).  Every carried value is p~_a = w_a (a0 + b m.c_a + 4.5
 *        c_a.X.c_a), evaluated with fused multiply-adds in a fixed order,
 *        from the node's a0, b, momentum m and symmetric X = m u^T + om Pi
 *        (the regularized collision and blend of Eqs. 16 and 23).
 *        Checkpoints 1 .. S-1 keep those 7 (2D) or 11 (3D) values, stored by
 *        the step that produces the field, and regenerate it bitwise.
 *        Checkpoint 0, the window's start field, which need not come from a
 *        step, stays native. */
enum { LBM_CKPT_NATIVE = 0, LBM_CKPT_FP16 = 1, LBM_CKPT_BF16 = 2, LBM_CKPT_MOMENT = 3 };

typedef struct {
  int32_t lattice;          /* LBM_D2Q9 or LBM_D3Q19                                  */
  int32_t nx, ny, nz;       /* lattice size; for D2Q9, nz > 1 stacks nz independent 2D
                               lattices (a batch of replicas: c_z = 0, slices never mix) */
  int32_t precision;        /* LBM_FP32 or LBM_FP64 (populations and adjoint)          */
  int32_t periodic[3];      /* 1 = periodic along x / y / z                           */
  double tau;               /* molecular relaxation time, nu = (tau - 1/2)/3 (Eq. 8)  */
  double cs_smag;           /* Smagorinsky constant C_s, filter width 1 (Eq. 9)       */
  double q_interp;          /* interpolation parameter of g(phi) (Sec. 2.2)           */
  double g_max;             /* g at phi = 0; the paper's value is 0.5                 */
  double rho_out;           /* outlet and reference density rho_0                     */
  int32_t objective_kind;   /* LBM_OBJ_*                                              */
  int32_t monitor_kind;     /* LBM_MON_*                                              */
  double objective_uref[3]; /* reference velocity of LBM_OBJ_VELOCITY_DEV              */
  double monitor_u;         /* reference velocity of the drag coefficient             */
  double monitor_l;         /* reference length of the drag coefficient               */
  int32_t window_len;       /* |W|, steps per window                                  */
  int32_t sample_every;     /* Delta W; must divide window_len                        */
  double conv_tol;          /* epsilon of Eq. 26                                      */
  int32_t ckpt_every;       /* K; must divide window_len                              */
  int32_t ckpt_format;      /* LBM_CKPT_*                                             */
  int32_t obj_box[6];       /* x0,x1,y0,y1,z0,z1 (half-open): weights read only here  */
  int32_t design_box[6];    /* x0,x1,y0,y1,z0,z1 (half-open): gradient nonzero only here */
  int32_t pipeline;         /* 1: recompute segment s-1 while the adjoint sweeps segment s
                               (twice the segment buffer); 0: one after the other        */
} lbm_config;

typedef struct lbm_ctx lbm_ctx;

/* Phase timings measured with CUDA events on the context's stream when timing
 * is enabled: milliseconds and launch counts per phase since the last reset.
 * Phase 0: forward steps of lbm_step_window; 1: recompute steps of
 * lbm_adjoint_window; 2: adjoint steps; 3: checkpoint copies/encodes/decodes. */
#define LBM_NUM_PHASES 4
typedef struct {
  double ms[LBM_NUM_PHASES];
  int64_t launches[LBM_NUM_PHASES];
  int64_t lattice_updates[LBM_NUM_PHASES];
} lbm_timing;

/* Bytes of device workspace lbm_create needs for cfg (validates cfg).
 * Returns LBM_ERR_ARG for an invalid configuration. */
lbm_status lbm_workspace_size(const lbm_config* cfg, size_t* bytes);

/* Create a solver.  Inputs are copied; the caller may free them afterwards.
 *   node_class        host, uint8 [N], LBM_FLUID..LBM_OUTLET_ZEROGRAD
 *   design_gamma      host or device, float [N], values in [0, 1]
 *   objective_weights host or device, float [N] (read inside obj_box only) or NULL = 0
 *   inlet_u           host or device, float [nz][ny] x-velocity on the x=0 face, or NULL = 0
 *   workspace         device, >= lbm_workspace_size bytes, 256-byte aligned, owned by the
 *                     caller and kept alive until lbm_destroy
 *   stream            cudaStream_t to enqueue on (NULL = legacy default stream)
 * The carried populations start at rest equilibrium (rho = 1, u = 0; Eq. 18).
 * Errors: LBM_ERR_ARG (bad cfg, classes or values), LBM_ERR_WORKSPACE, LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_config* cfg, const uint8_t* node_class, const float* design_gamma,
                      const float* objective_weights, const float* inlet_u, void* workspace,
                      size_t workspace_bytes, void* stream, lbm_ctx** out);

/* Run one window of |W| steps (Alg. 1 inner loop, Eqs. 24, 27, 42) and store
 * its checkpoints.  Returns the window means of the objective and of the
 * monitored quantity.  Synchronises the stream.
 * Errors: LBM_ERR_NONFINITE (the window produced rho <= 0 or NaN/Inf; the
 * window is not recorded), LBM_ERR_CUDA. */
lbm_status lbm_step_window(lbm_ctx* ctx, double* J_window, double* monitor_window);

/* Window means of the objective and monitor of every slice of a D2Q9 batch
 * (nz independent 2D lattices) for the last completed window; J and monitor
 * are host arrays of nslices = nz doubles (monitor may be NULL).  The
 * gradient of lbm_design_gradient at slice s is dJ_s/dgamma_s, since the
 * slices are independent.  Errors: LBM_ERR_ARG for D3Q19 or nslices != nz,
 * LBM_ERR_STATE before a window. */
lbm_status lbm_window_objectives(lbm_ctx* ctx, double* J, double* monitor, size_t nslices);

/* Alg. 1's outer loop: windows of lbm_step_window until the consecutive-window
 * test of Eq. 26 holds (converged = ratio < conv_tol between the last two
 * windows; a window never converges on its own), at most max_windows of them.
 * Returns the number of windows run and the last window's means and ratio
 * (each pointer may be NULL).  LBM_OK when the test held; LBM_NOT_CONVERGED
 * when the cap was reached first, the flow advanced and the last window
 * recorded, so lbm_adjoint_window may still follow.  Errors of
 * lbm_step_window stop the loop and are returned as they are. */
lbm_status lbm_run_until_converged(lbm_ctx* ctx, int32_t max_windows, int32_t* windows, double* J_window,
                                   double* monitor_window, double* ratio);

/* Consecutive-window test of Eq. 26 between the last two windows:
 * ratio = |(M_i - M_{i-1}) / M_i| (absolute difference when |M_i| < 1e-30),
 * converged = ratio < conv_tol.  Before two windows: converged = 0,
 * ratio = +inf.  Host only, no GPU work. */
lbm_status lbm_window_converged(lbm_ctx* ctx, int* converged, double* ratio);

/* Discrete adjoint over the last completed window (Alg. 2 reverse loop,
 * Eqs. 35-39), recomputing each segment of K steps from its checkpoint, and
 * the design sensitivity (Eq. 40) accumulated in FP64 with compensated
 * summation.  Returns that window's objective J_eff (Eq. 27).  Synchronises.
 * Errors: LBM_ERR_STATE if no window has completed since the last
 * lbm_create / lbm_set_state / lbm_set_design. */
lbm_status lbm_adjoint_window(lbm_ctx* ctx, double* J_eff);

/* dJ_eff/dgamma of the last adjoint window into grad (host or device, FP64
 * [N]): the sensitivity of Eq. 40, sum over the window's steps of the adjoint
 * times dp/dphi = g'(phi) (h_abar - h_a), with the sign flipped for
 * gamma = 1 - phi; zero outside design_box.  n must equal N.
 * Errors: LBM_ERR_STATE before lbm_adjoint_window, LBM_ERR_ARG for n != N. */
lbm_status lbm_design_gradient(lbm_ctx* ctx, double* grad, size_t n);

/* Replace the design field (host or device, float [N]); geometry unchanged.
 * Invalidates the recorded window and gradient. */
lbm_status lbm_set_design(lbm_ctx* ctx, const float* design_gamma);

/* Design pre-processing of Sec. 3.3: a linear density filter of radius r over
 * design_box (weights max(0, r - distance), normalised per node) followed by
 * the Heaviside projection of Wang et al. (2011),
 *   gamma = (tanh(beta eta) + tanh(beta (x~ - eta))) / (tanh(beta eta) + tanh(beta (1 - eta))).
 * Outside design_box gamma = x.  The projection acts on the solid fraction
 * gamma; for eta = 1/2 this equals projecting phi = 1 - gamma. */
typedef struct {
  double radius;   /* filter radius in lattice units (the paper uses 4)   */
  double beta;     /* projection steepness (the paper: 2 doubling to 16)   */
  double eta;      /* projection threshold (the paper: 0.5)                */
} lbm_filter;

/* Set the design from raw variables x (host or device, float [N], in [0,1])
 * through the filter and projection; like lbm_set_design it invalidates the
 * recorded window.  Errors: LBM_ERR_ARG for bad parameters or values. */
lbm_status lbm_set_design_filtered(lbm_ctx* ctx, const float* x_raw, const lbm_filter* f);

/* dJ_eff/dx for the raw variables of the last lbm_set_design_filtered: the
 * chain rule through the projection and the filter applied to dJ/dgamma
 * (host or device, FP64 [N]).  Errors: LBM_ERR_STATE before an adjoint
 * window or when the design was not set through the filter. */
lbm_status lbm_design_gradient_filtered(lbm_ctx* ctx, double* grad, size_t n);

/* Chain rule of the density filter and Heaviside projection (Sec. 3.3) for
 * any sensitivity: dx = (d gamma / d x)^T dgamma, both host or device, double
 * [N] (dgamma is read inside and outside design_box; outside, gamma = x).
 * This is what lbm_design_gradient_filtered applies to dJ/dgamma; the
 * optimization loop applies it to the volume constraint's gradient.
 * Errors: LBM_ERR_STATE unless the design was set by lbm_set_design_filtered,
 * LBM_ERR_ARG for n != N. */
lbm_status lbm_filter_chain_rule(lbm_ctx* ctx, const double* dgamma, double* dx, size_t n);

/* Volume fraction of Sec. 3.3, V = (1/n_D) sum over the design box of
 * (1 - phi_i), i.e. the mean of the current gamma over design_box; its
 * gradient with respect to gamma is 1/n_D inside the box.  FP64 sum in a
 * fixed order.  Errors: LBM_ERR_ARG for an empty design box. */
lbm_status lbm_design_volume(lbm_ctx* ctx, double* volume);

/* The current (physical) design field gamma (host or device, float [N]). */
lbm_status lbm_get_design(lbm_ctx* ctx, float* gamma, size_t n);

/* Read / write the carried post-collision populations p (FP64, [Q][N], host
 * or device, n = Q*N).  lbm_set_state invalidates the recorded window. */
lbm_status lbm_get_state(lbm_ctx* ctx, double* f, size_t n);
lbm_status lbm_set_state(lbm_ctx* ctx, const double* f, size_t n);

/* dJ_eff / d p^{n0-1}: the adjoint of the field the last adjoint window
 * started from (FP64, [Q][N], host or device, n = Q*N). */
lbm_status lbm_get_adjoint_state(lbm_ctx* ctx, double* a, size_t n);

/* Advance nsteps steps without sampling or checkpoints (spin-up). */
lbm_status lbm_advance(lbm_ctx* ctx, int32_t nsteps);

/* Enable (1) / disable (0) phase timing; lbm_get_timing copies and resets. */
lbm_status lbm_set_timing(lbm_ctx* ctx, int32_t enable);
lbm_status lbm_get_timing(lbm_ctx* ctx, lbm_timing* out);

/* Replay each window and each adjoint sweep as one CUDA graph (1, the
 * default) or launch every kernel individually (0).  Results are identical;
 * graphs remove the per-launch host overhead that dominates small lattices.
 * Graphs are captured on first use on a private stream and launched into the
 * context's stream. */
lbm_status lbm_set_graphs(lbm_ctx* ctx, int32_t enable);

/* Launch the step kernels with programmatic dependent launch (1, the default)
 * so that each launch overlaps the tail of the previous one, or plainly (0).
 * Results are identical either way. */
lbm_status lbm_set_pdl(lbm_ctx* ctx, int32_t enable);

/* One window of ctx along the trajectory of ref: ctx runs its window as
 * lbm_step_window does, except that each checkpoint segment s starts from
 * ref's checkpoint s of ref's last window (decoded if 16-bit or moment,
 * converted to ctx's precision).  ctx's checkpoints, window sums and the
 * adjoint of a following lbm_adjoint_window(ctx) then follow ref's primal
 * trajectory, up to ctx's own arithmetic within each segment.  This is the
 * "same trajectory" comparison of an FP32 (or mixed-precision) adjoint with
 * an FP64 one on a chaotic flow, where independent FP32 and FP64 runs over a
 * long window drift apart.  Both contexts need the same lattice, window
 * length and checkpoint interval, and ctx must not use moment checkpoints
 * (its segments restart from ref's fields): LBM_ERR_ARG otherwise; ref needs
 * a completed window (LBM_ERR_STATE).  ref's segment buffer serves as decode
 * scratch, which a later lbm_adjoint_window(ref) overwrites anyway.
 * Synchronises both streams; launched directly, not as a replayed graph. */
lbm_status lbm_step_window_along(lbm_ctx* ctx, lbm_ctx* ref, double* J_window, double* monitor_window);

/* First sampled step of each following window: the objective and monitor
 * means (Eq. 42) and the adjoint's objective sources use the steps first,
 * first + sample_every, ... < window_len, weighted by
 * sample_every / (window_len - first).  0 (the default) is the window of the
 * consecutive-window scheme (Sec. 3.1).  A window of T steps run from the
 * initial field with first = T - |W| is the full-time adjoint of Sec. 4.2.3
 * (the comparison with full-time adjoint optimization): the objective is the
 * mean over the final |W| steps, the whole history is checkpointed, and
 * lbm_adjoint_window traces the adjoint back to the initial time.  Its J
 * equals, bit for bit, that of a |W|-step window after the same T - |W|
 * unsampled steps.  Invalidates the recorded window and gradient; the
 * consecutive-window test keeps comparing successive windows as sampled.
 * Errors: LBM_ERR_ARG unless 0 <= first < window_len and
 * (window_len - first) is a multiple of sample_every.  The no-allocation
 * entry point always samples from step 0. */
lbm_status lbm_set_sample_start(lbm_ctx* ctx, int32_t first);

/* How the context launches its work. */
typedef struct {
  int32_t graphs;           /* 1: windows and sweeps replay as CUDA graphs            */
  int32_t pdl;              /* 1: programmatic dependent launch                       */
  int64_t kernels_window;   /* kernels enqueued by the last window (0 before one)     */
  int64_t kernels_adjoint;  /* kernels enqueued by the last adjoint sweep             */
} lbm_schedule;

lbm_status lbm_get_schedule(lbm_ctx* ctx, lbm_schedule* out);

/* Total steps advanced and windows completed since lbm_create. */
lbm_status lbm_get_counters(lbm_ctx* ctx, int64_t* steps, int64_t* windows);

/* One forward window, like lbm_step_window, for callers that cannot allocate
 * device memory: a host process that hands this library only buffers it
 * registered up front (a serving runtime with a fixed memory pool, a plug-in
 * living inside another application's allocator), or a sandbox that does not
 * expose the CUDA allocator.  There is no counterpart in the paper: it is a
 * deployment aid.
 *   cfg                 as for lbm_create (precision must be LBM_FP32; the
 *                       checkpoint fields are ignored)
 *   node_class          device, uint8 [N]: a map that lbm_create would accept.
 *                       It is not checked on the host; every node checks its
 *                       own class on the device, and a map that breaks the
 *                       rules (class out of range, a non-FLUID interior node,
 *                       a boundary class on the wrong face) fails the call
 *                       with LBM_ERR_ARG, leaving pop undefined
 *   design_gamma, objective_weights
 *                       device, float [N]
 *   inlet_u             device, float [nz][ny]
 *   pop                 device, float [Q][N], in/out: the carried field stored
 *                       shifted by the rest weights, p_a - w_a (the library's
 *                       internal FP32 layout); holds the window's last field
 *                       on return
 *   pop_tmp             device, float [Q][N], caller-owned second buffer
 *   stream              cudaStream_t to enqueue on (NULL = legacy default)
 * Returns the window means of the objective and the monitor like
 * lbm_step_window.  The call reads them back to the host and waits for the
 * stream before it returns; a stream that is capturing a CUDA graph is
 * refused with LBM_ERR_ARG before anything is enqueued.  It allocates
 * nothing: its only scratch is a 512 KiB + 256 B array inside the library
 * image, present on every GPU that loads the library until the process exits.
 * Limit: at most 16384 blocks of 128 nodes, i.e. ceil(nx/128) * ny * nz <=
 * 16384; larger lattices return LBM_ERR_ARG.  The first call on a device
 * looks up the array's device address.  All calls share the array and each
 * call clears what it needs at zero: calls that overlap on the GPU race.  g(phi) is
 * evaluated per node and step from gamma in FP64 (the rounding of the design
 * kernel), and the pressure objective samples cs^2 rho directly, so the
 * window means agree with lbm_step_window's to FP32 summation error.  No
 * checkpoints are stored, so lbm_adjoint_window cannot follow it.  Every
 * failure sets lbm_last_error. */
lbm_status lbm_step_window_noalloc(const lbm_config* cfg, const uint8_t* node_class, const float* design_gamma,
                                   const float* objective_weights, const float* inlet_u, float* pop,
                                   float* pop_tmp, void* stream, double* J_window, double* monitor_window);

/* ---- Design update: the Method of Moving Asymptotes ---------------------
 * The optimization loop of the paper (Sec. 3.3, topology optimization
 * procedure; Alg. 2) updates the design variables with MMA (Svanberg 1987)
 * under the volume constraint.  An lbm_mma holds one run's state for n
 * variables x in [xmin, xmax] and m constraints f_i(x) <= 0 (1 <= m <=
 * LBM_MMA_MAX_M).  Each lbm_mma_update takes the objective and constraint
 * values at x and their gradients, builds the moving asymptotes (x -/+ 0.5
 * span at the first two iterations, then contracted by 0.7 where x_j
 * oscillates and widened by 1.2 where it moves monotonically, kept within
 * [0.01, 10] span of x_j), the move limits (10% of the way to each
 * asymptote) and the convex separable approximations
 * r_i + sum_j p_ij/(U_j - z_j) + q_ij/(z_j - L_j), and solves the resulting
 * subproblem (with artificial variables of cost 1000 that keep it feasible)
 * by the dual method in FP64.  The per-variable work runs on the device. */
#define LBM_MMA_MAX_M 8
typedef struct lbm_mma lbm_mma;

/* Bytes of device workspace lbm_mma_create needs for n variables and m
 * constraints.  Errors: LBM_ERR_ARG for n = 0 or m outside [1, LBM_MMA_MAX_M]. */
lbm_status lbm_mma_workspace_size(size_t n, int32_t m, size_t* bytes);

/* Start an MMA run.
 *   xmin, xmax   host or device, double [n], finite, xmin < xmax (copied)
 *   workspace    device, >= lbm_mma_workspace_size bytes, 256-byte aligned, owned
 *                by the caller and kept alive until lbm_mma_destroy
 *   stream       cudaStream_t to enqueue on (NULL = legacy default stream)
 * Errors: LBM_ERR_ARG, LBM_ERR_WORKSPACE, LBM_ERR_CUDA. */
lbm_status lbm_mma_create(size_t n, int32_t m, const double* xmin, const double* xmax, void* workspace,
                          size_t workspace_bytes, void* stream, lbm_mma** out);

/* One MMA iteration.
 *   x        device, double [n], in/out: the current point, replaced by the next
 *   fval     host, double [m+1]: f_0(x) (the objective), then f_1(x) .. f_m(x)
 *   dfdx     device, double [m+1][n]: the gradients, objective first
 *   lam_out  host, double [m] or NULL: the subproblem's multipliers
 * Synchronises the stream.  Errors: LBM_ERR_ARG (null pointers, non-finite
 * fval, x or dfdx not device memory), LBM_ERR_CUDA. */
lbm_status lbm_mma_update(lbm_mma* mma, double* x, const double* fval, const double* dfdx, double* lam_out);

lbm_status lbm_mma_destroy(lbm_mma* mma);

const char* lbm_status_string(lbm_status s);
const char* lbm_last_error(void);
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBMADJ_H */
