/*
 * hosc.h -- C ABI of the GB300 (sm_103a) implementation of the higher-order super-compact (HOSC)
 * implicit finite-difference scheme for 3D natural convection of power-law fluids in a
 * differentially heated cubic cavity (Punia & Ray, arXiv:2411.06563).
 *
 * Problem (Sec. 2.1): dimensionless Boussinesq momentum, energy and continuity equations with the
 * power-law stress tau* = 2 eta eps, eta = I2^((n-1)/2) (Eqs. 6-8), gravity along -y; hot wall
 * theta = 1 at x = 0, cold wall theta = 0 at x = 1, the other walls adiabatic, no slip on every
 * wall, zero normal pressure gradient on every wall. Parameters Ra, Pr and n (Sec. 2.1), the
 * uniform N^3 node grid with h = k = l = 1/(N-1) (or, for a box 1 x Ly x Lz, h = 1/(N-1),
 * k = Ly/(N-1), l = Lz/(N-1); see hosc_params) and the pseudo-time step dt (Sec. 3.1).
 *
 * One pseudo-time step (Sec. 2.2):
 *   S1  power-law viscosity eta and L = 1/(Pr eta) from the local strain rate (Eqs. 7-8);
 *   S2  momentum sources E* (pressure gradient, eps . grad eta, buoyancy);
 *   S3  the fourth-order compact right-hand sides of Eq. (5)/(6) for u, v, w and theta;
 *   S4  the seven-point level-(n+1) operator of Eq. (5) (weights L1..L7 of Eq. 6);
 *   S5  unpreconditioned BiCGSTAB on the four systems (BiCGSTAB(2) as an option);
 *   S6  wall conditions; S7 div V and the modified artificial-compressibility correction
 *       p <- p - lambda div V (Sec. 2.2, last paragraph); S8 the steady-state change max|chi^{n+1}-chi^n|.
 * Diagnostics (Sec. 4.2-4.3): local / average Nusselt numbers, entropy generation, Bejan number.
 *
 * Conventions
 *  - Every call returns an hosc_status; nothing aborts and no C++ exception crosses the ABI.
 *  - Fields are N^3 arrays of double, x fastest: node (i, j, k) at index i + N*(j + N*k),
 *    x_i = i/(N-1), y_j = j Ly/(N-1), z_k = k Lz/(N-1) (Ly = Lz = 1 for the cube).
 *  - Host buffers passed in are owned by the caller and only read/written during the call.
 *  - A context owns its device memory (or uses a caller-supplied device workspace) and all work
 *    is enqueued on one CUDA stream (the caller's, or one it creates). A context must not be used
 *    from two host threads at once; different contexts may run concurrently.
 *  - Errors: HOSC_EINVAL for bad arguments (the context is unchanged), HOSC_ECUDA when a CUDA call
 *    fails (the context should be destroyed), HOSC_ENOCONV / HOSC_EDIVERGED are numerical outcomes
 *    reported by a step (the fields hold the state after that step).
 */
#ifndef HOSC_H
#define HOSC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HOSC_OK = 0,
  HOSC_EINVAL = 1,     /* invalid argument or parameter */
  HOSC_ENOMEM = 2,     /* device or host allocation failed, or workspace too small */
  HOSC_ECUDA = 3,      /* a CUDA runtime call failed */
  HOSC_ENOCONV = 4,    /* BiCGSTAB reached max_lin_iter or broke down */
  HOSC_EDIVERGED = 5,  /* a field became NaN or Inf */
  HOSC_ESTEPLIMIT = 6, /* hosc_solve_steady reached max_steps before the steady criterion */
  HOSC_ESTATE = 7      /* call not valid in the current state */
} hosc_status;

/* Arithmetic of the step. HOSC_FP64: every kernel in double. HOSC_MIXED: the state (u, v, w,
 * theta, p), the divergence / pressure update, every norm and reduction and the diagnostics stay in
 * double; the viscosity, sources and right-hand-side sweeps run in float (differences of the state
 * taken in double first), and the BiCGSTAB vectors and operator weights are float. When the step
 * change stalls at the float rounding level the context switches to FP64 defect sweeps (the
 * right-hand side dt (R - B chi^n) in double, the Krylov solve still float), whose fixed point is
 * the FP64 steady state. tol_lin is raised to at least 3e-6 for the float solves. */
typedef enum { HOSC_FP64 = 0, HOSC_MIXED = 1 } hosc_precision;

/* Field selectors for hosc_get_field / hosc_set_field. */
typedef enum {
  HOSC_U = 0, HOSC_V = 1, HOSC_W = 2, HOSC_THETA = 3, HOSC_P = 4,
  /* level-n quantities computed by a step (read-only) */
  HOSC_ETA = 5,    /* apparent viscosity eta (S1) */
  HOSC_LCOEF = 6,  /* L = 1/(Pr eta) (S1) */
  HOSC_EU = 7, HOSC_EV = 8, HOSC_EW = 9, /* momentum sources E* (S2) */
  HOSC_RHS_U = 10, HOSC_RHS_V = 11, HOSC_RHS_W = 12, HOSC_RHS_THETA = 13,
      /* dt (R - B chi^n) at interior nodes, the right-hand side of the increment form of Eq. (6) (S3) */
  HOSC_DX_U = 14, HOSC_DX_V = 15, HOSC_DX_W = 16, HOSC_DX_THETA = 17,
      /* BiCGSTAB solution chi^{n+1} - chi^n of the last solve (S5) */
  /* level n-1 history used by delta_t^- (settable, for restart / checkpoint) */
  HOSC_PREV_L = 18, HOSC_PREV_U = 19, HOSC_PREV_V = 20, HOSC_PREV_W = 21,
  HOSC_PREV_EU = 22, HOSC_PREV_EV = 23, HOSC_PREV_EW = 24,
  HOSC_DIV = 25,   /* central div V^{n+1} at interior nodes (S7) */
  /* level-(n+1) weights of Eq. (6) (S4, read-only): centre, x+, x-, y+, y-, z+, z- */
  HOSC_A_MOM = 26, /* 26..32: momentum operator, shared by u, v, w */
  HOSC_A_ENE = 33, /* 33..39: energy operator */
  HOSC_NFIELDS = 40
} hosc_field;

/* Stages of one step, for stage-by-stage use (tests, checkpointing). */
typedef enum {
  HOSC_STAGE_VISCOSITY = 0, /* S1: eta, L */
  HOSC_STAGE_SOURCES = 1,   /* S2: E* of the three momentum equations */
  HOSC_STAGE_RHS = 2,       /* S3/S4: right-hand sides and the level-(n+1) operators */
  HOSC_STAGE_SOLVE = 3,     /* S5: BiCGSTAB (or BiCGSTAB(2)) on the four systems */
  HOSC_STAGE_UPDATE = 4     /* S6-S8: increments, walls, div V, pressure, history */
} hosc_stage;

typedef struct {
  int N;              /* nodes per side including walls, 5 <= N <= 1025 */
  double Ra;          /* Rayleigh number (Sec. 2.1), >= 0 */
  double Pr;          /* Prandtl number (Sec. 2.1), > 0 */
  double n;           /* power-law index (Eq. 7), > 0 */
  double dt;          /* pseudo-time step (Sec. 3.1 uses 0.02), > 0 */
  double lambda;      /* relaxation of p <- p - lambda div V (Sec. 2.2), > 0 */
  double theta_ref;   /* buoyancy reference temperature: the y source has Ra (theta - theta_ref)/eta */
  double theta_init;  /* initial interior temperature (fluid at rest, constant pressure) */
  double I2_eps;      /* regulariser: eta = (I2 + I2_eps)^((n-1)/2); unused when n == 1 */
  double phi;         /* irreversibility distribution ratio of E_FF (Sec. 4.3), 1e-4 */
  double tol_steady;  /* hosc_solve_steady stops when max|chi^{n+1}-chi^n| / dt < tol_steady and
                         max|div V| < div_steady (below) */
  double tol_div;     /* the pressure is corrected while max|div V| > tol_div (Sec. 2.2) */
  double tol_lin;     /* BiCGSTAB stops when ||r_k||_2 <= tol_lin ||r_0||_2 */
  int max_lin_iter;   /* BiCGSTAB iteration limit per system and step, >= 1 */
  int precision;      /* hosc_precision */
  void* cuda_stream;  /* cudaStream_t to enqueue on, or NULL for a stream owned by the context */
  double a_limit;     /* lower limit of the diagonal term M18 of the level-(n+1) operator, in units
                         of L (keeps its mass positive when L changes fast); 0 disables */
  double a_boost;     /* factor of the pseudo-time mass added to the level-(n+1) operator where the
                         cell Reynolds number |G*| h is high (keeps every grid mode damped);
                         0 disables. Neither changes the steady state B chi = R. */
  int use_history;    /* 1: the delta_t^- terms of Eq. (5) use the level n-1 history (the paper's
                         second-order-in-time scheme); 0: delta_t^- = 0 at every step, a
                         first-order pseudo-time march with the same steady state */
  int auto_defect;    /* HOSC_MIXED: 1 switches from FP32 to FP64 defect sweeps by itself when the
                         step change stalls: 200 steps without a 5 % improvement once it is below
                         1e-3 of the largest step change of the solve, or 2000 steps at any level
                         (counted from the largest step change so far, so a spin-up whose step
                         change still grows is no stall); 0 keeps the phase chosen with
                         hosc_set_phase */
  int precond;        /* 0: BiCGSTAB on the systems as assembled (the paper's unpreconditioned
                         solver, the default); 1: Jacobi row scaling, each row of the level-(n+1)
                         system and its right-hand side divided by the row's diagonal before the
                         solve (same solution; the stopping test then measures the scaled
                         residual). Not in the paper. */
  int inner_max;      /* 0 (default): one pressure correction per step. >= 1: while max|div V| >
                         tol_div after the correction, up to inner_max inner pressure passes: E*
                         again with the corrected pressure (level-n velocities and viscosity, the
                         new temperature), u, v, w solved again from level n, div V, correction
                         (Sec. 2.2's "previous pressure iteration"; theta is not solved again).
                         Such steps are issued from the host (not captured); pools reject it. */
  double Ly, Lz;      /* box 1 x Ly x Lz (lengths in units of the hot-cold wall distance, the x
                         length): N nodes per side, spacings h = 1/(N-1), k = Ly/(N-1),
                         l = Lz/(N-1) along x, y, z (the scheme of Sec. 2.2 is written for unequal
                         spacings). 0 stands for 1 (the paper's cube, the default); otherwise
                         1/64 <= Ly, Lz <= 64. Wall means are averages over the wall; E_total,
                         E_HT, E_FF are integrals over the box volume. */
  int solver;         /* level-(n+1) solver: 0 (default) BiCGSTAB, the reading of Sec. 2.2's
                         solver used throughout; 1 BiCGSTAB(2) (Sleijpen-Fokkema: two BiCG steps
                         and a two-term minimal-residual update per cycle), the other reading of
                         its "hybrid" BiCGSTAB. Iterations are counted as two per cycle (each
                         iteration applies the operator twice, as a BiCGSTAB iteration does) and
                         max_lin_iter limits them. 1 needs HOSC_FP64 (HOSC_EINVAL otherwise) and
                         adds three N^3 vectors per system to the workspace. */
  int lambda_mode;    /* pressure correction p <- p - lambda_c div V (Sec. 2.2, last paragraph):
                         0 (default) lambda_c = lambda, the paper's single relaxation parameter;
                         1 lambda_c = min(lambda eta, 0.9 h_min^2 / dt) at each node, with eta the
                         node's apparent viscosity at level n: the relaxation follows the local
                         viscous time scale of the pressure modes (a steady-solve accelerator, not
                         in the paper; the fixed point div V = 0 is the same). */
  double div_steady;  /* the steady stop's divergence test: max|div V| < div_steady; 0 (the
                         default) means tol_div, the paper's single threshold. hosc_steady_params
                         sets it to tol_steady and tol_div, the correction's threshold, far below */
} hosc_params;

typedef struct {
  long steps;         /* steps taken by this call */
  long lin_iters;     /* BiCGSTAB iterations summed over systems and steps of this call (two per
                         BiCGSTAB(2) cycle) */
  int last_iters[4];  /* iterations of the last step's u, v, w, theta solves */
  double res_steady;  /* max over u, v, w, theta of max|chi^{n+1} - chi^n| of the last step */
  double div_max;     /* max|div V^{n+1}| at interior nodes of the last step */
  double lin_res;     /* largest ||r_k|| / ||r_0|| of the last step's four solves */
  int status;         /* hosc_status of the last step */
  long inner_passes;  /* inner pressure passes summed over the steps of this call */
  long sys_iters[4];  /* iterations of the u, v, w, theta solves, each summed over the steps */
  long solve_iters;   /* the largest of the four systems' iterations, summed over the steps: the
                         passes of the mixed-precision solve, which iterates the four systems
                         together until the last one has converged */
} hosc_info;

typedef struct {
  double Nu_hot_max;   /* max over z of Nu_avg(z) at x = 0 (the quantity of Table 2) */
  double Nu_hot_mean;  /* surface mean of Nu_local at x = 0 */
  double Nu_cold_mean; /* surface mean of -d theta/dx at x = 1 */
  double E_total;      /* volume integral of E_local = E_HT + E_FF (Simpson) */
  double E_HT;         /* volume integral of |grad theta|^2 */
  double E_FF;         /* volume integral of phi eta I2 */
  double Be;           /* E_HT / E_total */
} hosc_diag;

/* Fill *p with defaults for grid N and (Ra, Pr, n): dt = 0.02, lambda = min(h^2/(4 dt), Pr/10),
 * theta_ref = theta_init = 0.5, I2_eps = 1e-10, phi = 1e-4, tol_steady = 1e-6, tol_div = 1e-6,
 * tol_lin = 1e-10, max_lin_iter = 1000, HOSC_FP64, own stream, a_limit = 0.25, a_boost = 1,
 * use_history = 1, auto_defect = 1, div_steady = 0 (the stop tests tol_div). After changing
 * dt, set lambda again (it must stay below h^2/dt). */
hosc_status hosc_default_params(hosc_params* p, int N, double Ra, double Pr, double n);

/* Parameters for a steady solve (a pseudo-time march to the fixed point B chi = R of Eq. 5, which
 * depends on neither dt nor lambda): the defaults of hosc_default_params, then
 *   lambda = 2 Pr min(1, 2 eta_bl), dt = min(dt_stab, 0.9 h^2 / lambda), use_history = 0,
 * with h = 1/(N-1), u = max(1, 1.5 c sqrt(Ra)), c = 0.12 * 2^(4 (1 - n)) (a velocity scale of the
 * converged cavity), eta_bl = min(1, (u^2 sqrt(Ra))^((n-1)/2)) for n < 1 (the boundary-layer
 * viscosity; 1 otherwise), dt_stab = min(0.02, Pr eta_min / u^2) with eta_min = eta_bl for n < 1,
 * 1 for n = 1 and I2_eps^((n-1)/2) for n > 1 (a factor 4 inside the bound dt |G*|^2 <= 4 L of
 * the explicit compact terms). A large lambda speeds up the slowest pressure modes, which
 * contract by a fixed fraction of lambda per step; lambda dt must stay below h^2. The rule uses
 * the cube's spacing: for a box (Ly, Lz) set dt and lambda again. tol_div = tol_steady h /
 * (2 lambda): while the pressure correction runs, the step change it causes (about lambda
 * tol_div / h per unit pseudo-time) stays below tol_steady, so the correction is never switched
 * off and on around its threshold near the steady state. The stop's divergence test is kept at
 * the steady criterion itself: div_steady = tol_steady (if tol_steady is changed, set tol_div and
 * div_steady again). HOSC_EINVAL for N < 5, Ra < 0, Pr <= 0 or n <= 0. */
hosc_status hosc_steady_params(hosc_params* p, int N, double Ra, double Pr, double n);

/* Bytes of device workspace a context with these parameters needs (0 if invalid). */
size_t hosc_workspace_bytes(const hosc_params* p);

/* Create a context: validates *p, allocates device memory with cudaMalloc, sets the initial
 * state (V = 0, p = 0, theta = theta_init inside with the wall temperatures). */
hosc_status hosc_create(const hosc_params* p, void** ctx_out);

/* As hosc_create but carves all device arrays out of a caller-owned device buffer of at least
 * hosc_workspace_bytes(p) bytes, aligned to 256 bytes (e.g. a PyTorch allocation). The buffer
 * must outlive the context. */
hosc_status hosc_create_in(const hosc_params* p, void* dev_workspace, size_t bytes, void** ctx_out);

/* Free everything the context owns. NULL is accepted. */
void hosc_destroy(void* ctx);

/* Back to the initial state (fields, history and step counter). */
hosc_status hosc_reset(void* ctx);

/* Take nsteps >= 1 pseudo-time steps. Enqueues the work and waits for it once at the end.
 * Stops early at the first step whose status is not HOSC_OK and returns that status. */
hosc_status hosc_step(void* ctx, int nsteps, hosc_info* out);

/* Step until max|chi^{n+1}-chi^n| / dt < tol_steady and max|div V| < div_steady (tol_div when
 * div_steady is 0) (HOSC_OK), or
 * max_steps (HOSC_ESTEPLIMIT), or a numerical failure. */
hosc_status hosc_solve_steady(void* ctx, long max_steps, hosc_info* out);

/* Run a single stage of the next step (see hosc_stage); stages must be run in order. */
hosc_status hosc_run_stage(void* ctx, int stage, hosc_info* out);

/* Diagnostics of the current fields (Sec. 4.2-4.3). nu_avg_z (N doubles) and fields (3 N^3
 * doubles: E_HT, E_FF, E_local) are optional host outputs. */
hosc_status hosc_diagnostics(void* ctx, hosc_diag* out, double* nu_avg_z, double* fields);

/* Copy a field (hosc_field) to / from a host buffer of N^3 doubles. Setting U, V, W, THETA or P
 * replaces the state as given (walls included); setting a PREV_* field marks the level n-1
 * history as present (hosc_clear_history removes it, so delta_t^- = 0 at the next step). */
hosc_status hosc_get_field(void* ctx, int which, double* host_out);
hosc_status hosc_set_field(void* ctx, int which, const double* host_in);
hosc_status hosc_clear_history(void* ctx);

/* Copy a state field between the context and a device buffer of N^3 doubles on the context's
 * stream (no synchronisation). */
hosc_status hosc_get_field_device(void* ctx, int which, double* dev_out);
hosc_status hosc_set_field_device(void* ctx, int which, const double* dev_in);

/* Parameters the context runs with, and its stream (cudaStream_t). */
hosc_status hosc_get_params(void* ctx, hosc_params* out);

/* Per-launch timing of every kernel class with CUDA events on the context's stream (adds two event
 * records per launch). enable(on != 0) resets the accumulators; read returns, for one kernel
 * class, the summed event milliseconds, the launch count and the algorithmic bytes those launches
 * moved (each array element read or written once per launch, counting only the systems still
 * iterating). The algorithmic-byte counters run whether or not timing is on. Outputs may be NULL. */
hosc_status hosc_profile_enable(void* ctx, int on);
hosc_status hosc_profile_read(void* ctx, int kernel_id, double* total_ms, long* launches,
                              double* alg_bytes);

/* Time one kernel class in isolation (kernel_id HOSC_K_VISC .. HOSC_K_BICG_XR): between steps,
 * launch that kernel reps times back to back on the context's stream between two CUDA events,
 * on the current state (the BiCGSTAB kernels on the buffers of the last solve, with all four
 * systems marked as iterating; the marking kernel's time is measured apart and subtracted).
 * Returns the mean milliseconds per launch and the algorithmic bytes of one launch. The fields
 * u, v, w, theta, p and the history keep their values; the derived arrays and the Krylov
 * buffers are overwritten and recomputed by the next step. HOSC_EINVAL for another id or
 * reps < 1, and for the BiCGSTAB classes when solver = 1 (BiCGSTAB(2): its five kernels are
 * counted under the p/v, s/t and x/r classes by hosc_profile_read but not timed alone);
 * HOSC_ESTATE in the middle of a stage-by-stage step. */
hosc_status hosc_time_kernel(void* ctx, int kernel_id, int reps, double* ms_per_launch,
                             double* bytes_per_launch);

/* Launch shape of the mixed-precision BiCGSTAB kernels, which store the four systems interleaved
 * (one float4 per node) and give each thread one interior (i, j) column over kz consecutive
 * planes: kblock threads per block (a multiple of 32, 64..384; at most 256 with narrow = 1 or
 * the merged iteration form), kz in 1..N-2, and at most N^3/16 + 1024 blocks per launch;
 * narrow = 1 selects the kernels compiled for at most 64 registers per thread (more resident
 * blocks), 0 those with more (80 for the three-kernel form, 128 for the merged form). The
 * default (128 threads, wide, kz from the wave model below) is chosen from N at creation.
 * Changing it drops the captured steps (captured again at the next step). HOSC_EINVAL for a shape
 * outside these limits, HOSC_ESTATE in the middle of a stage-by-stage step. The FP64 solve has
 * one thread per node and ignores the setting. */
hosc_status hosc_set_tiles(void* ctx, int kblock, int kz, int narrow);
hosc_status hosc_get_tiles(void* ctx, int* kblock, int* kz, int* narrow);

/* Staged stencil kernels of the mixed-precision solve (the p/v and s/t kernels with their reads
 * staged through shared memory by cp.async, several planes ahead): a block owns sx * sy interior
 * columns (one thread each; sx * sy a multiple of 32 in 32..256) and skz consecutive planes
 * (1..N-2). sx == 0
 * selects the register kernels of hosc_set_tiles for p/v and s/t (the default). HOSC_EINVAL for
 * a shape that does not fit (shared memory above 200 KB per block, too many blocks),
 * HOSC_ESTATE in the middle of a stage-by-stage step. Changing it drops the captured steps. */
hosc_status hosc_set_stencil_tiles(void* ctx, int sx, int sy, int skz);
hosc_status hosc_get_stencil_tiles(void* ctx, int* sx, int* sy, int* skz);

/* Bulk-copy (TMA) stencil kernels of the mixed-precision solve: the p/v and s/t kernels with
 * their reads moved by the GPU's bulk-copy engine (tensor-map box copies of each z-plane into a
 * ring of `stages` shared-memory stages, 3, 4, 6 or 8, stages - 2 planes ahead of the one being
 * computed; one producer thread, mbarrier completion), so that the bytes in flight do not
 * depend on registers or resident warps. A block owns tty rows of the
 * plane's interior columns (whole rows up to 126 columns; wider planes are cut into equal
 * pieces) and tkz consecutive planes (1..N-2). tty == 0 selects the register kernels (the
 * default; tkz and stages are then ignored); setting tiles here clears hosc_set_stencil_tiles
 * and the reverse. HOSC_EINVAL for a
 * shape that does not fit (at most 512 threads and 200 KB of shared memory per block, too many
 * blocks), HOSC_ECUDA when the driver cannot encode the tensor maps, HOSC_ESTATE mid-step.
 * kernels selects which of the two run in this form: 1 p/v only (s/t keeps the register kernel
 * of hosc_set_tiles), 2 s/t only, 3 both (HOSC_EINVAL otherwise).
 * Three-kernel iteration form only (the merged form keeps its own kernels). Changing it drops
 * the captured steps. A wait of these kernels that runs out (2 s) ends the step with HOSC_ECUDA
 * instead of hanging. */
hosc_status hosc_set_tma_tiles(void* ctx, int tty, int tkz, int stages, int kernels);
hosc_status hosc_get_tma_tiles(void* ctx, int* tty, int* tkz, int* stages, int* kernels);

/* Form of the mixed-precision x/r kernel (three-kernel iteration): flat = 0 (the default) the
 * column march of hosc_set_tiles; 1 one flat grid-stride stream over the interior planes (the
 * i and j wall nodes included, where every vector is zero), each thread issuing the loads of
 * four nodes before their arithmetic. HOSC_EINVAL for another value, HOSC_ESTATE mid-step.
 * Drops the captured steps. hosc_get_xr_form returns the form (-1 for a NULL context). */
hosc_status hosc_set_xr_form(void* ctx, int flat);
int hosc_get_xr_form(void* ctx);

/* Form of the mixed-precision BiCGSTAB iteration: merged = 1 runs two kernels per iteration,
 * folding the x, r update of iteration i-1 into the p, v kernel of iteration i and obtaining
 * r_0.r_{i+1} for beta from r_0.s and r_0.t of the s, t kernel (the same method; the
 * convergence test sees the true residual one kernel later); 0 (the default) runs the three
 * kernels p/v, s/t, x/r. HOSC_EINVAL for another value or when the current launch shape does not suit the form,
 * HOSC_ESTATE mid-step. Drops the captured steps. hosc_get_krylov_merged returns the current
 * form (-1 for a NULL context). */
hosc_status hosc_set_krylov_merged(void* ctx, int merged);
int hosc_get_krylov_merged(void* ctx);

/* Autotuner for the launch shape above: after at least one completed step, time the three
 * BiCGSTAB kernels (hosc_time_kernel, reps launches each) for the valid shapes with kblock in
 * {64, 96, 128, 160, 192, 256, 320, 384} and kz in 1..33 whose modelled cost (waves of
 * resident blocks on this GPU, from the kernels' occupancy, times kz + 2 planes streamed per
 * block) is within 1.5x of the least, for both register budgets (narrow 0 and 1), time the
 * four fastest again with 4 reps launches each and keep the fastest; then time the other
 * iteration form (hosc_set_krylov_merged)
 * at that shape and keep the faster; with the three-kernel form, then time the
 * staged p/v and s/t kernels (hosc_set_stencil_tiles) for tiles sx in {8, 16, ..., 64},
 * sy in {4, 8} and skz in 1..33 within 1.5x of their least modelled cost, and the bulk-copy
 * kernels (hosc_set_tma_tiles) for stages in {3, 4, 6, 8}, tty in 1..8 and tkz in 1..50 within
 * 1.5x of their least modelled cost (waves times planes streamed over planes in flight), and keep
 * the fastest of: both register, both staged, both bulk-copy at their best shape, bulk-copy p/v
 * at its best shape with the register s/t; then the two x/r forms (hosc_set_xr_form) with
 * 4 reps launches each, keeping the flat stream only when it is at least 5 % faster. Reports
 * the register shape (any output pointer may be NULL; ms_out = the three kernels' summed mean
 * milliseconds with the chosen kernels). Mixed precision only (HOSC_EINVAL for FP64). The fields
 * keep their values. */
hosc_status hosc_autotune(void* ctx, int reps, int* kblock_out, int* kz_out, double* ms_out);

/* Kernel classes for hosc_profile_read and hosc_time_kernel. */
enum { HOSC_K_VISC = 0, HOSC_K_SOURCES = 1, HOSC_K_RHS = 2, HOSC_K_BICG_PV = 3,
       HOSC_K_BICG_ST = 4, HOSC_K_BICG_XR = 5, HOSC_K_UPDATE = 6, HOSC_K_COUNT = 7 };

/* Mixed precision only: select FP32 sweeps (0) or FP64 defect sweeps (1) for the next steps (the
 * automatic switch, when auto_defect is set, is re-armed); get returns the current phase. With
 * HOSC_FP64, phase 0 is accepted and 1 rejected. */
hosc_status hosc_set_phase(void* ctx, int phase);
int hosc_get_phase(void* ctx);

/* Number of kernel launches the library has made since the context was created. */
long hosc_kernel_launches(void* ctx);

/* Allocation-free BiCGSTAB solve of the four level-(n+1) systems of one step, for callers that
 * cannot call cudaMalloc: hosts whose own allocator (a framework's caching allocator, a memory
 * pool sized at start-up) already owns the device memory, so that a cudaMalloc beside it would
 * fail or fragment the pool, and solvers that run under a fixed device-memory budget decided
 * before the first step. The paper has no counterpart; this is an interface of this library.
 * The call is synchronous: every 4 to 16 iterations it copies the four systems' solver scalars to
 * a host array and waits for the stream (cudaStreamSynchronize) to test convergence, and it
 * returns once the solve has finished.
 *
 * Solves A_mom x_s = rhs_s for s = u, v, w and A_ene x_theta = rhs_theta with the same kernels as
 * hosc_step (FP64 BiCGSTAB from x = 0, stop when ||r|| <= tol ||r_0||), on the interior nodes of
 * an N^3 grid. weights: host array of 14 device pointers, N^3 doubles each, in the order
 * centre, x+, x-, y+, y-, z+, z- of the momentum operator then of the energy operator (the
 * layout of HOSC_A_MOM / HOSC_A_ENE); rhs: host array of 4 device pointers (N^3 doubles, interior
 * nodes read); x: host array of 4 device pointers (N^3 doubles; interior nodes written, walls
 * untouched). iters_out: host int[4] or NULL. stream: cudaStream_t or NULL.
 * The caller owns every input and output. Scratch (Krylov vectors, partial sums, solver scalars)
 * is one file-scope device array of 13.3 MB sized for N <= HOSC_NOALLOC_MAX_N, which every GPU
 * that loads the library holds until the process exits; larger N returns HOSC_EINVAL. The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current: make that first call before any stream capture. All calls share the array and it keeps
 * the last call's contents (each call clears what must start at zero), so calls that overlap on
 * the GPU race: serialise them (one stream, or wait between calls). Returns HOSC_ENOCONV if a
 * system did not converge within max_iter, HOSC_ECUDA on a CUDA error. */
#define HOSC_NOALLOC_MAX_N 41
hosc_status hosc_bicgstab_noalloc(int N, const double* const* weights, const double* const* rhs,
                                  double* const* x, double tol, int max_iter, int* iters_out,
                                  void* stream);

/* ------------------------------------------------------------------------------------------
 * Pools: many cavity solves advancing together on one GPU (batching and serving). Not in the
 * paper, which solves one cavity at a time; each member runs the same step as hosc_step.
 *
 * Members are contexts admitted against a device-memory budget (the sum of their
 * hosc_workspace_bytes). hosc_pool_run advances every active member by rounds of
 * steps_per_round captured steps; each member stops on the device at its first steady step
 * (the hosc_solve_steady criterion). After each round the host folds the step records and
 * completes a member that is steady (status HOSC_OK), failed (its step status) or has taken at
 * least max_steps steps (HOSC_ESTEPLIMIT; the last round may overrun max_steps by fewer than
 * steps_per_round steps). Diagnostics are computed at completion. A completed member keeps its
 * device memory (its fields can be read through the context that hosc_pool_result returns)
 * until hosc_pool_retire.
 *
 * mode HOSC_POOL_STREAMS: each member launches its captured steps on its own stream.
 * mode HOSC_POOL_GRAPH: a whole round of every active member is one captured graph with one
 *   branch per member (steps_per_round must be even); it is captured again when membership,
 *   or a member's level parity, history, phase or launch shape, changes.
 * mode HOSC_POOL_PERSISTENT: a whole round of every active member is one launch of a
 *   persistent kernel (a cooperative grid of all resident blocks) that walks, phase after phase
 *   of each step, a work list of (member, tile) items of all members, with a grid barrier
 *   between phases (each wait bounded: a wait that gives up ends the round with HOSC_ECUDA).
 *   Members must be mixed precision with BiCGSTAB, use_history = 0 and inner_max = 0
 *   (HOSC_EINVAL at admission otherwise); launch shapes are the kernel's own (autotune unused).
 * autotune != 0: after the first round of the first mixed-precision member of each N, the pool
 *   runs hosc_autotune on it and gives later members of that N the same launch shape.
 * The pool's calls are single-threaded; members use their own streams and the pool's stream. */
enum { HOSC_POOL_STREAMS = 0, HOSC_POOL_GRAPH = 1, HOSC_POOL_PERSISTENT = 2 };

typedef struct {
  int active;          /* members still advancing */
  int completed;       /* members completed and not yet retired */
  int tuned_sizes;     /* grid sizes N with a tuned launch shape */
  size_t bytes_used;   /* device bytes held by members */
  size_t budget;
  long rounds;         /* rounds run */
  long captures;       /* round graphs captured (HOSC_POOL_GRAPH) */
  double capture_ms;   /* host milliseconds spent capturing and instantiating them */
} hosc_pool_info;

/* budget_bytes > 0; 1 <= steps_per_round <= 256. */
hosc_status hosc_pool_create(size_t budget_bytes, int steps_per_round, int mode, int autotune,
                             void** pool);
void hosc_pool_destroy(void* pool);  /* destroys every member */
/* Create a member for *params (its cuda_stream is ignored: each member has its own stream).
 * HOSC_ENOMEM when it does not fit the budget now (it may after retirements), HOSC_EINVAL when
 * it can never fit or the parameters are invalid. *slot: the member's index. */
hosc_status hosc_pool_admit(void* pool, const hosc_params* params, long max_steps, int* slot);
/* Run up to `rounds` rounds, returning after the first round in which a member completed. The
 * completed slots go to done_slots[0 .. min(*ndone, cap)). HOSC_ECUDA stops the pool. */
hosc_status hosc_pool_run(void* pool, int rounds, int* done_slots, int cap, int* ndone);
/* Result of a member: status (HOSC_ESTATE while active), steps and iterations over its whole
 * solve, diagnostics (after completion), and its context (for hosc_get_field, until retire).
 * Any output pointer may be NULL. */
hosc_status hosc_pool_result(void* pool, int slot, hosc_status* status, hosc_info* info,
                             hosc_diag* diag, void** ctx);
/* Free a member's context and device memory (active or completed). */
hosc_status hosc_pool_retire(void* pool, int slot);
hosc_status hosc_pool_stats(void* pool, hosc_pool_info* out);

/* Measured FP64 arithmetic rate of the current GPU in TFLOP/s (no counterpart in the paper): the
 * denominator of the roofline of the all-FP64 sweep kernels, which the FP64 pipe bounds. A grid
 * of 8 blocks of 256 threads per SM runs chains of fused multiply-adds (2 flops each) `reps`
 * times after one warm-up launch, timed with CUDA events on the default stream. Allocates and
 * frees a small device buffer. HOSC_EINVAL for reps < 1 or a NULL output, HOSC_ECUDA on a CUDA
 * error. */
hosc_status hosc_fp64_peak(int reps, double* tflops_out);

const char* hosc_strerror(int status);

/* Text of the last CUDA failure seen by this host thread (for HOSC_ECUDA / HOSC_ENOMEM). */
const char* hosc_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* HOSC_H */
