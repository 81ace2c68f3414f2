/*
 * ns3d.h -- C ABI of libns3d.so: GB300 (sm_103a) evaluation of the right-hand
 * side of the 3D compressible Navier-Stokes equations on a triply periodic
 * Cartesian grid, and its Runge-Kutta time integration, as stated in
 * arXiv 2211.16718 (Kim, Ghosh, Constantinescu, Balakrishnan):
 *
 *   du/dt = R(u) = -(df/dx + dg/dy + dh/dz) + (df^v/dx + dg^v/dy + dh^v/dz)
 *
 * (Sec. 2.1, Eq. NS), u = [rho, rho u, rho v, rho w, e], with
 *  - convective terms: conservative finite differences of interface fluxes
 *    (Sec. 2.2), each scalar component of u and f reconstructed by WENO5 with
 *    the Jiang-Shu weights (Sec. 2.2), upwinded by the Roe flux with Harten's
 *    entropy fix (Sec. 2.2, Eq. Roe);
 *  - viscous and heat-flux terms: 4th-order central finite differences
 *    (Sec. 2.1 stresses and heat flux; Sec. 2.2);
 *  - time integration: classical RK4 or the three-stage TVD (SSP) RK
 *    (Sec. 2.2).
 *
 * Conventions shared by every call
 *  - State layout: contiguous FP64 structure-of-arrays u[5][nz][ny][nx]
 *    (variable slowest, x fastest), i.e. element (v, k, j, i) at
 *    v*N + (k*ny + j)*nx + i with N = nx*ny*nz.  Grid point i has
 *    x_i = i*lx/nx (periodic).  Pointers named *_dev are device memory of the
 *    current CUDA device, 16-byte aligned; *_host are host memory (pinned or
 *    pageable).  The caller owns every buffer it passes.
 *  - Streams: all device work of a call is enqueued on the context's stream
 *    (given to ns3d_init, changeable with ns3d_set_stream).  Only the calls
 *    that return host data (ns3d_stats, ns3d_check, ns3d_step_host,
 *    ns3d_dt_from_cfl, ns3d_timing_read) synchronise that stream.
 *  - Errors: every int-returning call returns NS3D_OK (0) or a negative code;
 *    nothing aborts or traps.  ns3d_last_error(ctx) gives a message.
 *    Non-physical states (rho <= 0, p <= 0, a non-finite value, or a negative
 *    Roe-averaged sound speed squared) set a sticky device status word that
 *    ns3d_stats / ns3d_check report as NS3D_ENONPHYSICAL and then clear;
 *    data outside the range of the double-float weights set it too and are
 *    reported as NS3D_ERANGE.
 *  - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef NS3D_H
#define NS3D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  NS3D_OK = 0,
  NS3D_EINVAL = -1,        /* bad parameter, size, null or aliasing pointer */
  NS3D_ENOMEM = -2,        /* device or pinned-host allocation failed */
  NS3D_ECUDA = -3,         /* CUDA launch/runtime error (see ns3d_last_error) */
  NS3D_ENONPHYSICAL = -4,  /* non-physical state detected by a kernel */
  NS3D_ETIMEOUT = -5,      /* reserved for a bounded device-side wait that gives up; no call
                              returns it: no kernel of the library spins on a flag (the
                              persistent ensemble kernel separates its phases with the grid
                              barriers of a cooperative launch, whose CTAs are co-resident) */
  NS3D_ERANGE = -6         /* data beyond the range of the double-float WENO weights
                              (differences of the data above ~1e9): use NS3D_FP64_STRICT */
};

enum { NS3D_RK4 = 0, NS3D_SSPRK3 = 1 };           /* time integrators (Sec. 2.2) */
/* Arithmetic of the reconstruction and upwinding:
 *  NS3D_FP64        FP64 state, point values and their first differences, point fluxes,
 *                   interface-flux sums and RK update; what only multiplies small
 *                   differences or enters through a dissipation or viscous term (the
 *                   nonlinear WENO weights and offsets, the interface jumps, the Roe
 *                   dissipation, the viscous fluxes and their divergence, the statistics'
 *                   kinetic energy, vorticity and wave speed) in double-float arithmetic
 *                   (two FP32 words, ~48 bits) on the FP32 pipe.  Agrees with the all-FP64
 *                   evaluation to within the parity tolerance of the FP64 path (1e-12
 *                   relative on the right-hand side).  Requires weno_eps >= 1e-15.
 *  NS3D_FP32_BULK   primitive variables, point fluxes, smoothness indicators, weights,
 *                   interface values, Roe flux and viscous fluxes in FP32; the total
 *                   interface flux is widened to FP64 before the conservative difference
 *                   (exact telescoping: a free stream gives a zero RHS, the grid sums are
 *                   conserved to FP64 rounding); state, RK accumulation and reductions in
 *                   FP64.  Relative RHS error ~1e-7 of the flux scale max|f|/dx.
 *                   Requires weno_eps >= 1e-15.
 *  NS3D_FP64_STRICT every operation in FP64 (one FP64 division per reconstruction). */
enum { NS3D_FP64 = 0, NS3D_FP32_BULK = 1, NS3D_FP64_STRICT = 2 };
/* Storage of the viscous flux vectors (same results, bitwise, in every mode):
 *  NS3D_STORAGE_FULL  all three directions' fluxes at once, 12*N doubles;
 *  NS3D_STORAGE_LEAN  the flux of one direction before each direction pass, 4*N
 *                     doubles (the gradients are evaluated three times): lets a
 *                     1024^3 grid with SSP-RK3 fit in one GB300's HBM;
 *  NS3D_STORAGE_AUTO  FULL if its scratch fits in the free device memory at
 *                     ns3d_init with a 4 GB margin, else LEAN. */
enum { NS3D_STORAGE_AUTO = 0, NS3D_STORAGE_FULL = 1, NS3D_STORAGE_LEAN = 2 };

typedef struct ns3d_ctx ns3d_ctx;                 /* opaque; owned by the library */

typedef struct {
  int nx, ny, nz;       /* points per direction, each >= 1 */
  int rk;               /* NS3D_RK4 (default) or NS3D_SSPRK3 */
  int precision;        /* NS3D_FP64 (default), NS3D_FP32_BULK or NS3D_FP64_STRICT */
  int weno_p;           /* exponent p of the WENO weights; only 2 is supported */
  double lx, ly, lz;    /* periodic box lengths (> 0); default 2*pi */
  double gamma;         /* ratio of specific heats, default 1.4 (Sec. 2.1) */
  double mu_eff;        /* mu * M_inf / Re_inf (Sec. 2.1), >= 0; 0 = Euler */
  double prandtl;       /* Prandtl number, default 0.72 (Sec. 2.1) */
  double weno_eps;      /* epsilon of the WENO weights, default 1e-6 (Sec. 2.2) */
  double harten_delta;  /* entropy-fix width as a fraction of the Roe sound speed, >= 0 */
  int storage;          /* NS3D_STORAGE_AUTO (default), _FULL or _LEAN */
} ns3d_params;

/* Statistics of a state (all FP64 reductions over the grid). */
typedef struct {
  double mass, momx, momy, momz, energy;  /* sum of rho, rho u, rho v, rho w, e times dx dy dz */
  double ke;                              /* mean of rho |v|^2 / 2 */
  double enstrophy;                       /* mean of rho |omega|^2 / 2, omega by 4th-order central differences */
  double rho_min, p_min;
  double max_wavespeed_over_dx;           /* max over points, d of (|u_d| + c)/dx_d; CFL = dt * this */
  int status;                             /* NS3D_OK, NS3D_ENONPHYSICAL or NS3D_ERANGE */
  int reserved;
} ns3d_stats_t;

/* Number of doubles ns3d_stats_async writes: the 10 fields above in order, then
 * the status word as a double, then one reserved slot. */
#define NS3D_STATS_NDOUBLE 12

/* Fill *p with the paper's defaults for an nx x ny x nz grid on [0, 2pi)^3:
 * gamma 1.4, Pr 0.72, eps 1e-6, p = 2, harten_delta 0.1, mu_eff 0, RK4, FP64,
 * NS3D_STORAGE_AUTO. */
void ns3d_default_params(ns3d_params *p, int nx, int ny, int nz);

/* Create a context: validates *p (NS3D_EINVAL), allocates the library-owned
 * device scratch (NS3D_ENOMEM): primitive variables 7*N, viscous fluxes 12*N
 * (4*N with NS3D_STORAGE_LEAN; none if mu_eff = 0), RHS accumulator 5*N doubles,
 * reduction partials and a status word.  The first Runge-Kutta step allocates
 * two stage states 10*N (and for RK4 an accumulator 5*N) doubles.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream). */
int ns3d_init(const ns3d_params *p, void *cuda_stream, ns3d_ctx **out);

/* Release every resource of ctx (NULL is a no-op).  Synchronises its stream. */
void ns3d_free(ns3d_ctx *ctx);

/* Change the stream that later calls enqueue on. */
int ns3d_set_stream(ns3d_ctx *ctx, void *cuda_stream);

/* rhs_dev = R(u_dev) (Sec. 2.1 Eq. NS with the Sec. 2.2 discretisation).
 * u_dev, rhs_dev: 5*N doubles each, must not overlap. */
int ns3d_rhs(ns3d_ctx *ctx, const double *u_dev, double *rhs_dev);

/* Advance u_dev in place by nsteps (>= 0) steps of size dt (finite) with the
 * context's integrator (Sec. 2.2).  No host synchronisation (except the first
 * call, which allocates the stage buffers; NS3D_ENOMEM if they do not fit). */
int ns3d_rk_step(ns3d_ctx *ctx, double *u_dev, double dt, int nsteps);

/* Statistics of u_dev copied into *out_host; synchronises the stream.  Returns
 * NS3D_ENONPHYSICAL (with out_host->status set) if the sticky status word was
 * set by any earlier call or by this one, and clears it. */
int ns3d_stats(ns3d_ctx *ctx, const double *u_dev, ns3d_stats_t *out_host);

/* Same statistics written to out_dev[NS3D_STATS_NDOUBLE] on the device without
 * synchronising (for logging every step inside a captured or timed loop).  The
 * status slot holds the sticky status word at that point (not cleared). */
int ns3d_stats_async(ns3d_ctx *ctx, const double *u_dev, double *out_dev);

/* Statistics of u_dev without any device allocation (the paper has no
 * counterpart; this serves callers that must not let a library allocate device
 * memory, e.g. a host code that owns all GPU memory through its own pool and
 * budget, or an in-situ monitoring hook inside another solver's time loop:
 * creating a context allocates scratch, and cudaMalloc/cudaFree bypass such a
 * pool, can fail under memory pressure and synchronise the device).
 *  - p: grid and gas parameters (nx, ny, nz >= 1, lx, ly, lz > 0, gamma > 1;
 *    the other fields are ignored).  No context is needed.
 *  - u_dev: the state, layout as above; out_dev: NS3D_STATS_NDOUBLE doubles on
 *    the device, written in the order of ns3d_stats_async, with the status slot
 *    1.0 if this state is non-physical (rho <= 0, p <= 0, non-finite), else 0.
 *  - Work is enqueued on cuda_stream (a cudaStream_t; NULL = legacy default
 *    stream); the call does not synchronise.
 *  - Scratch: a fixed 96 KB array of per-block partial sums (1024 slots) held in
 *    device memory by every GPU that loads the library, until the process
 *    exits.  The kernel strides over the grid, so every grid up to 2^32 points
 *    fits; larger grids return NS3D_EINVAL.  Every call overwrites the slots it
 *    uses before reading them, so no state carries over between calls, but all
 *    calls share the array: calls that overlap on the GPU (other streams,
 *    other host threads) race and must be serialised by the caller.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any stream
 *    capture.
 *  - Returns NS3D_OK, NS3D_EINVAL (null pointer, bad size) or NS3D_ECUDA.
 *    Calls no cudaMalloc, cudaFree or other allocating routine. */
int ns3d_stats_noalloc(const ns3d_params *p, const double *u_dev, double *out_dev, void *cuda_stream);

/* Time step from a CFL number (Sec. 2.3 reading: CFL = dt * max over grid points and
 * directions d of (|u_d| + c)/dx_d, c the speed of sound): *dt_out = cfl / that maximum
 * for the state u_dev, computed by the statistics kernels (synchronises the stream, and
 * reads and clears the sticky status word as ns3d_stats does).  Returns NS3D_EINVAL for
 * a null pointer or a cfl that is not finite and > 0, NS3D_ENONPHYSICAL if the state is
 * non-physical or the maximum is not finite and > 0 (*dt_out is then unchanged). */
int ns3d_dt_from_cfl(ns3d_ctx *ctx, const double *u_dev, double cfl, double *dt_out);

/* End-to-end call with host buffers: copies u_host to library-owned device
 * memory, advances nsteps steps of size dt, computes the statistics of the
 * final state into *stats_host (may be NULL), copies the state back into
 * u_host.  Synchronises.  On grids with nz >= 64 (FP64 modes, full viscous
 * storage) the copies run in z-slabs on a library-owned second stream and
 * overlap with the first and last RK stages; the result is bitwise that of
 * ns3d_rk_step on a device copy of the state.  u_host should be pinned
 * (page-locked) for the copies to overlap; it is in use until the call
 * returns, also when it fails. */
int ns3d_step_host(ns3d_ctx *ctx, double *u_host, double dt, int nsteps, ns3d_stats_t *stats_host);

/* Read and clear the sticky status word (synchronises): NS3D_OK or NS3D_ENONPHYSICAL. */
int ns3d_check(ns3d_ctx *ctx);

/* Static description of a code. */
const char *ns3d_strerror(int code);

/* Message of the last failure of ctx (empty if none). */
const char *ns3d_last_error(const ns3d_ctx *ctx);

/* ---- ensembles of independent grids of uneven sizes ---------------------------
 * Many independent realisations (e.g. the decaying-turbulence problem of Sec. 2.3
 * with different seeds and grid sizes) advanced together on one GPU.  Each
 * instance has its own parameters (grid, box, mu_eff, ...; all instances share
 * precision, which must be NS3D_FP64 or NS3D_FP64_STRICT, and rk), its own
 * caller-owned state and its own dt.  The schedules compute bitwise identical
 * results:
 *  NS3D_BATCH_SEQUENTIAL  per-instance launches (5 per RK stage per instance), one
 *                         instance after the other on the batch's stream;
 *  NS3D_BATCH_GRAPH       the same per-instance launches for one step, captured once
 *                         in a CUDA graph whose parallel branches each advance a share
 *                         of the instances (balanced by points, largest first), so that
 *                         small instances run beside the large ones; one graph launch
 *                         per step;
 *  NS3D_BATCH_PERSISTENT  one cooperative kernel for all steps, stages, phases and
 *                         instances over a flattened (instance, tile) work list, phases
 *                         separated by grid-wide barriers (captured in a CUDA graph
 *                         when the runtime allows it). */
enum { NS3D_BATCH_SEQUENTIAL = 0, NS3D_BATCH_GRAPH = 1, NS3D_BATCH_PERSISTENT = 2 };
typedef struct ns3d_batch ns3d_batch;

/* params[count] (count 1..4096, each grid <= 2^31 points); allocates the
 * per-instance scratch (~39 doubles per point).  NS3D_EINVAL / NS3D_ENOMEM. */
int ns3d_batch_init(const ns3d_params *params, int count, void *cuda_stream, ns3d_batch **out);
void ns3d_batch_free(ns3d_batch *b);
/* u_dev[count]: host array of caller-owned device states (layout as above). */
int ns3d_batch_set_states(ns3d_batch *b, double *const *u_dev);
/* dt[count]: host array of per-instance time steps. */
int ns3d_batch_set_dt(ns3d_batch *b, const double *dt);
/* Advance every instance by nsteps steps with the given schedule (no host sync). */
int ns3d_batch_step(ns3d_batch *b, int nsteps, int schedule);
/* Statistics of every instance into out_dev[count * NS3D_STATS_NDOUBLE] (no sync). */
int ns3d_batch_stats(ns3d_batch *b, double *out_dev);
/* Per-instance time steps from one CFL number (as ns3d_dt_from_cfl, each instance from
 * its own current state) applied as by ns3d_batch_set_dt and, if dt_out is not NULL,
 * copied to dt_out[count].  Synchronises.  NS3D_EINVAL for a cfl that is not finite and
 * > 0 or before ns3d_batch_set_states; NS3D_ENONPHYSICAL if an instance has no finite
 * positive wave speed (the time steps are then unchanged). */
int ns3d_batch_set_dt_from_cfl(ns3d_batch *b, double cfl, double *dt_out);
/* Read and clear the batch's sticky status word (synchronises). */
int ns3d_batch_check(ns3d_batch *b);
/* Tile shape of the direction passes: variant 0 (24 x 4), 1 (16 x 4), 2 (40 x 2)
 * points x lines, for every instance and the persistent kernel; results do not
 * depend on it.  NS3D_FP64_STRICT batches have the one shape 0 (32 x 4). */
int ns3d_batch_set_variant(ns3d_batch *b, int variant);
/* Tile shape of instance i alone (SEQUENTIAL and GRAPH schedules; the persistent
 * kernel keeps the shape of ns3d_batch_set_variant). */
int ns3d_batch_set_instance_variant(ns3d_batch *b, int i, int variant);
/* Parallel branches of the GRAPH schedule, 1..8 (default 4). */
int ns3d_batch_set_branches(ns3d_batch *b, int branches);
/* Autotuner: for every grid size of the ensemble (instances with the same nx, ny, nz
 * and viscous or not), times one step of that size's instances with each tile shape
 * (sequential launches, on copies of the current states, which are not advanced) and
 * gives those instances the fastest; then times one GRAPH-scheduled step with 1, 2, 4
 * and 8 branches and keeps the fastest count.  Each choice is appended to the
 * JSON-lines file cache_path as {"key": ..., "variant": ... | "branches": ...,
 * "ms_per_step": [...]} (NULL: no cache); keys already in the cache are used
 * without timing.  ms_out (may be NULL) has room for 3 * count + 8 doubles:
 * ms_out[3 i + v] = the time of shape v on instance i's size, then the time with
 * 1..8 branches (-1 where not timed).  NS3D_ENOMEM if the state copies do not fit. */
int ns3d_batch_autotune(ns3d_batch *b, const char *cache_path, double *ms_out);
/* Current tile shape of the persistent kernel, its CTAs per SM (0 before its first use)
 * and whether it runs captured in a graph (1), as a direct launch (0) or not yet (-1). */
int ns3d_batch_info(const ns3d_batch *b, int *variant, int *persistent_ctas_per_sm, int *persistent_in_graph);
/* Per-instance tile shapes into variants[count] and the GRAPH schedule's branch count
 * (either pointer may be NULL). */
int ns3d_batch_schedule_info(const ns3d_batch *b, int *variants, int *branches);
const char *ns3d_batch_last_error(const ns3d_batch *b);

/* Tile shape of the direction passes of a single context (see ns3d_batch_set_variant). */
int ns3d_set_variant(ns3d_ctx *ctx, int variant);
/* Order in which the CTAs of the z pass walk the grid: 0 = the tiles along z first,
 * 1 = the line groups of one tile row first (the CTAs resident at one time stay within
 * a few z-tile rows; 2.8x faster z pass on a 1024^3 grid), -1 = by grid size (the
 * default: 1 from 2^28 points up).  Both orders compute the same bits.  Returns
 * NS3D_OK or NS3D_EINVAL (order outside -1..1). */
int ns3d_set_zorder(ns3d_ctx *ctx, int order);

/* Storage chosen by ns3d_init (NS3D_STORAGE_FULL or NS3D_STORAGE_LEAN) and the
 * library-owned device bytes the context holds now. */
int ns3d_storage_info(const ns3d_ctx *ctx, int *storage, size_t *device_bytes);

/* ---- adjoint (vector-Jacobian products) -----------------------------------------
 * Exact discrete adjoints of the operators above (the paper has none; they serve
 * gradients of statistics of the flow with respect to its initial state).
 * NS3D_FP64_STRICT contexts evaluate them all in FP64; NS3D_FP64 contexts run the
 * derivatives of the WENO5 reconstructions in double-float arithmetic (relative
 * rounding ~1e-14, data range as for the forward weights, NS3D_ERANGE beyond it) and
 * the rest in FP64; NS3D_FP32_BULK contexts return NS3D_EINVAL.
 * Derivatives follow the discretisation as written: the WENO5 weights (smooth,
 * eps > 0), the Roe average, Harten's quadratic branch, and |lambda| with the
 * subgradient sign(0) = 0 at its kink.  The first adjoint call of a context
 * allocates 46*N doubles of library-owned device scratch (NS3D_ENOMEM); the
 * trajectory calls allocate their checkpoints.  No call synchronises except
 * ns3d_functional with value_host != NULL. */
enum { NS3D_FUNC_KE = 0, NS3D_FUNC_ENSTROPHY = 1 };

/* out_dev = J(u_dev)^T lam_dev, J = dR/du of ns3d_rhs at u_dev.  5*N doubles each;
 * out_dev must not overlap u_dev or lam_dev. */
int ns3d_rhs_vjp(ns3d_ctx *ctx, const double *u_dev, const double *lam_dev, double *out_dev);

/* Reverse of one step of the context's integrator from the state u_dev (the state
 * at the start of the step, unchanged): on entry ubar_dev is the adjoint of the
 * state after the step, on return the adjoint of u_dev.  The stage states are
 * recomputed from u_dev with the forward step's own launches. */
int ns3d_rk_step_vjp(ns3d_ctx *ctx, const double *u_dev, double *ubar_dev, double dt);

/* Functional of a state: NS3D_FUNC_KE = mean of rho |v|^2 / 2, NS3D_FUNC_ENSTROPHY =
 * mean of rho |omega|^2 / 2 (as in ns3d_stats).  value_host (may be NULL) receives
 * its value (synchronises); grad_dev (may be NULL; 5*N doubles, not overlapping
 * u_dev) receives its gradient with respect to u_dev. */
int ns3d_functional(ns3d_ctx *ctx, const double *u_dev, int which, double *value_host, double *grad_dev);

/* Advance u_dev in place by nsteps steps (as ns3d_rk_step) and record the states
 * at steps 0, every, 2*every, ... (ceil(nsteps/every) checkpoints of 5*N doubles,
 * library-owned, kept until the next call or ns3d_free). */
int ns3d_traj_forward(ns3d_ctx *ctx, double *u_dev, double dt, int nsteps, int every);

/* Reverse sweep over the trajectory recorded by the last ns3d_traj_forward: on
 * entry ubar_dev is the adjoint of the final state, on return the adjoint of the
 * initial state.  Each segment of `every` steps is recomputed from its checkpoint
 * (allocating `every` states once), then reversed step by step with
 * ns3d_rk_step_vjp.  NS3D_EINVAL if no trajectory has been recorded. */
int ns3d_traj_vjp(ns3d_ctx *ctx, double *ubar_dev);

/* ---- measurement support (no counterpart in the paper) -------------------- */
/* Kernel identifiers used by the timing calls. */
enum {
  NS3D_K_PRIM = 0,       /* primitive variables */
  NS3D_K_VISC = 1,       /* velocity/temperature gradients -> viscous fluxes */
  NS3D_K_DIR_X = 2,      /* fused WENO5 + Roe + conservative difference (+ viscous divergence), x */
  NS3D_K_DIR_Y = 3,
  NS3D_K_DIR_Z = 4,      /* ... z, with the RK stage update fused in */
  NS3D_K_STATS = 5,      /* statistics partial reductions */
  NS3D_K_STATS_FINAL = 6,
  NS3D_K_ADJ_VISC = 7,   /* adjoint of the viscous terms and of the primitive variables */
  NS3D_K_ADJ_DIR = 8,    /* adjoint of the fused direction passes (x, y, z) */
  NS3D_K_ADJ_MISC = 9,   /* functional seeds and adjoint copies */
  NS3D_K_COUNT = 10
};

/* on != 0: record CUDA events around every kernel launch of ctx (on its stream)
 * and accumulate their durations; on == 0 stops recording.  Resets counters. */
int ns3d_timing_enable(ns3d_ctx *ctx, int on);

/* Synchronise and read the accumulated device time (ms_out[k], milliseconds)
 * and launch counts (launches_out[k]) per kernel id, k < n (<= NS3D_K_COUNT);
 * either pointer may be NULL. */
int ns3d_timing_read(ns3d_ctx *ctx, double *ms_out, long long *launches_out, int n);

/* FP64 / FP32 arithmetic throughput of the current device in G lane-ops/s,
 * measured with register-only kernels: out[0] DFMA, out[1] DADD, out[2] DDIV,
 * out[3] DSQRT, out[4] FFMA.  Synchronises the device; allocates 2.5 MB. */
int ns3d_alu_probe(double out[5]);

#ifdef __cplusplus
}
#endif

#endif /* NS3D_H */
