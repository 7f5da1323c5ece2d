/* resim.h -- C ABI of the GB300 (sm_103a) CPR-FGMRES reservoir solver.
 *
 * The library implements, on one GPU, the Newton/linear-solve path of the
 * fully implicit two-phase oil-water simulator of Liu, Shen, Chen, Wang,
 * Yang and Chen, "A Parallel Simulator for Massive Reservoir Models
 * Utilizing Distributed-Memory Parallel Systems" (arXiv 1701.06254):
 *   model and discretisation      Sec. "Two-phase oil-water flow model",
 *                                 eqs. (3)-(18), capillary pressure eq. (9),
 *                                 wells eq. (10) with controls eqs. (11)-(14)
 *   Newton / inexact Newton       Algorithm 1, eqs. (24)-(27)
 *   decoupling                    eq. (29), ABF and Quasi-IMPES operators
 *   local potential reordering    eqs. (30)-(32)
 *   CPR-FPF preconditioner        Algorithm 2, eqs. (34)-(35)
 *   Krylov solver                 GMRES(m) (flexible, right preconditioned)
 *
 * Conventions (every entry point):
 *  - Returns a sim_status; SIM_OK = 0.  No entry point aborts the process.
 *    sim_last_error() returns a thread-local message for the last failure.
 *    Every entry point returns SIM_ERR_ARG for a NULL handle or a NULL
 *    required pointer, SIM_ERR_CUDA when a CUDA runtime call fails,
 *    SIM_ERR_OOM when a device allocation fails and SIM_ERR_STATE for a call
 *    out of order; an entry point without an "Errors" note has only these.
 *  - Units: p in bar, t in days, lengths in m, permeability in mD,
 *    viscosity in cP, density in kg/m3, compressibility in 1/bar, well
 *    rates in standard m3/day.
 *  - Cells are numbered naturally, c = i + nx*(j + ny*k), k = 0 at the top;
 *    z is depth (positive downwards).
 *  - Inputs are copied at creation; the caller keeps ownership of every
 *    array it passes.  Pointers documented as "host or device" are
 *    accepted in either memory (the library asks the CUDA runtime).
 *  - All GPU work is issued on the stream given in sim_options.cuda_stream
 *    (NULL = the legacy default stream).  Entry points that return host
 *    values synchronise that stream.
 *  - A handle is not thread-safe; distinct handles may be used from
 *    distinct threads.
 *  - One process drives one GPU: kernel attributes (shared-memory sizes)
 *    are set once per process, on the device current at first use.  Run one
 *    process per GPU (as bench.py does under torchrun).
 */
#ifndef RESIM_H
#define RESIM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SIM_OK = 0,
  SIM_ERR_ARG = 1,           /* invalid argument (NULL, size, unsupported option)   */
  SIM_ERR_CUDA = 2,          /* a CUDA runtime call failed                           */
  SIM_ERR_OOM = 3,           /* device allocation failed                              */
  SIM_ERR_NOT_CONVERGED = 4, /* Newton did not converge within the time-step cuts    */
  SIM_ERR_NAN = 5,           /* a non-finite residual or update was produced          */
  SIM_ERR_TIMEOUT = 6,       /* a bounded device loop hit its iteration cap           */
  SIM_ERR_STATE = 7          /* call out of order (e.g. solve before assemble)        */
} sim_status;

enum { SIM_INJ = 0, SIM_PROD = 1 };                            /* well kind           */
/* well controls: BHP eq. (11), water rate eq. (12), oil rate eq. (13),
 * liquid rate eq. (14), shut in (no flow; one of the schedule stages of the
 * paper's Table 1) */
enum { SIM_BHP = 0, SIM_WRATE = 1, SIM_ORATE = 2, SIM_LRATE = 3, SIM_SHUT = 4 };
enum { SIM_DEC_NONE = 0, SIM_DEC_ABF = 1, SIM_DEC_QI = 2 };    /* eq. (29) operator   */
enum { SIM_NEWTON_STANDARD = 0, SIM_NEWTON_INEXACT = 1 };      /* Algorithm 1         */
/* preconditioner precision: FP64; FP32 (AMG, RAS factors, CPR vectors; FP64
 * coarsest solve); FP32 with the RAS factor values stored in BF16 */
enum { SIM_PREC_FP64 = 0, SIM_PREC_MIXED = 1, SIM_PREC_MIXED_BF16 = 2 };
/* Krylov method of the linear solve: flexible GMRES(restart) (the paper's
 * GMRES(50), Examples 4-5) or BiCGSTAB (Examples 3, 6, 7), both right
 * preconditioned by CPR-FPF (Algorithm 2) */
enum { SIM_KRYLOV_FGMRES = 0, SIM_KRYLOV_BICGSTAB = 1 };
/* AMG interpolation on the pressure block: direct, or extended+i (distance-
 * two interpolation through the strong F neighbours' strong C points) */
enum { SIM_INTERP_DIRECT = 0, SIM_INTERP_EXTI = 1 };

typedef struct { int nx, ny, nz; double dx, dy, dz, top_depth; } sim_grid;

/* Rock: n = nx*ny*nz values each, host or device; permeability in mD. */
typedef struct { const double *kx, *ky, *kz, *phi; } sim_rock;

/* Fluid: index 0 = water, 1 = oil.  eqs. (4), (6), (7) and Corey relative
 * permeabilities kr_w = krw_max s^nw, kr_o = kro_max (1-s)^no with
 * s = (s_w - swc)/(1 - swc - sor) clipped to [0, 1]; g in m/s^2.
 * Capillary pressure (eq. 9, p_w = p_o - p_c(s_w)): pc_n points (0 = none,
 * at most 16) of a table, pc_sw strictly increasing, pc_val in bar (host
 * arrays, copied at creation), joined by straight lines and constant beyond
 * the first and last points.  The water phase pressure sets the water
 * density, viscosity, potential and perforation drawdown; porosity follows
 * p_o. */
typedef struct {
  double rho_ref[2], c_f[2], mu_ref[2], c_mu[2];
  double p_ref, c_r, swc, sor, nw, no, krw_max, kro_max, g;
  int pc_n;
  const double *pc_sw, *pc_val;
} sim_fluid;

/* A well (eq. 10): perforated cells (host array, n_perf entries), well
 * index per perforation (host, or NULL for Peaceman's formula with r_w and
 * skin), reference depth z_ref of p_b.  Controls: SIM_BHP (target in bar)
 * and SIM_WRATE for any well, SIM_ORATE and SIM_LRATE for producers
 * (injectors inject water), SIM_SHUT for any well.  Rate targets are
 * surface volumes in sm3/day (the phase mass rates of eq. 10 over each
 * phase's reference density; a producer's production counts positive; the
 * liquid rate is oil plus water).  bhp_limit (rate controls only; 0 = none)
 * is an injector's maximum or a producer's minimum p_b: when a Newton update
 * takes p_b past it the well goes on BHP control at the limit, and at the
 * start of a later time step it returns to its rate when, at the limit, it
 * would deliver more than the rate. */
typedef struct {
  int kind, control;
  double target, r_w, skin, z_ref;
  int n_perf;
  const int *perf_cell;
  const double *wi;
  double bhp_limit;
} sim_well;

typedef struct {
  int precision;       /* SIM_PREC_FP64, SIM_PREC_MIXED or SIM_PREC_MIXED_BF16      */
  int decoupling;      /* SIM_DEC_*                                                */
  int reorder;         /* 1: local potential reordering in each RAS subdomain     */
  int newton;          /* SIM_NEWTON_*                                             */
  double newton_tol;   /* scaled max-residual tolerance                            */
  double lin_tol;      /* relative linear residual (standard Newton)               */
  int max_newton, restart, max_lin; /* restart, max_lin <= 0: default; restart <= 63 */
  int tile_x, tile_y;  /* RAS subdomain = tile_x x tile_y cell columns (<= 0: 4)  */
  double amg_theta;
  int amg_max_levels, amg_coarse_max;
  uint64_t seed;       /* PMIS hash seed                                           */
  int max_cuts;        /* time-step halvings allowed per step                      */
  double dt;           /* time step, days                                          */
  void *cuda_stream;   /* cudaStream_t or NULL                                     */
  double sat_chop;     /* max |ds_w| applied per Newton update, 0 = full step      */
  int krylov;          /* SIM_KRYLOV_FGMRES or SIM_KRYLOV_BICGSTAB                 */
  int overlap;         /* RAS overlap in the matrix graph: 1 or 2 (Table 9)        */
  int interp;          /* SIM_INTERP_DIRECT or SIM_INTERP_EXTI                     */
  int fp64_basis;      /* mixed precision only: 1 keeps the FGMRES basis, w = A z
                          and Gram-Schmidt in FP64; 0 (default) holds them in
                          double-float (hi + lo FP32, ~48-bit significand)     */
} sim_options;

/* Statistics, cumulative since creation. */
typedef struct {
  long long steps, newton, linear_its, cuts, linear_solves;
  double last_relres, last_norm, t;
  int last_its, last_newton;
  double ms_assemble, ms_setup, ms_solve;   /* CUDA-event time, cumulative */
  long long ws_used, ws_fallback;           /* warm starts with / without the network's term */
  double ws_r0;                             /* sum over warm-started solves of ||b - A x0|| / ||b|| */
  long long switches;                       /* wells put on BHP control at their limit */
} sim_stats;

typedef struct sim_s *sim_t;
typedef struct sim_ls_s *sim_ls_t;

/* Fill *o with the defaults: FP64, ABF, reordering on, standard Newton,
 * newton_tol 1e-8, lin_tol 1e-8, max_newton 20, restart 50, max_lin 100,
 * 4x4 tiles, theta 0.25, 25 levels, coarsest <= 128 rows, 6 cuts, dt 1,
 * no saturation chop, FGMRES, overlap 1, direct interpolation, double-float
 * basis in mixed precision. */
void sim_default_options(sim_options *o);

/* Create a simulator (copies everything).  Builds transmissibilities,
 * well indices, the 2x2 block sparsity pattern (cells, then one padded
 * block row per well) and the RAS partition; allocates device memory.
 * Grids of at most 50M cells (the solver setup keeps 32-bit counts).
 * Errors: SIM_ERR_ARG for bad sizes/controls or option values (an unknown
 * precision, decoupling, reorder or Newton code; a tolerance that is
 * negative or not finite; amg_theta outside [0, 1]; a negative max_newton,
 * max_cuts or amg_coarse_max; dt not finite and > 0), all checked before any
 * device work; SIM_ERR_OOM, SIM_ERR_CUDA. */
sim_status sim_create(sim_t *out, const sim_grid *g, const sim_rock *r, const sim_fluid *f,
                      const sim_well *wells, int n_wells, const sim_options *o);
void sim_destroy(sim_t h);

/* Equilibrium start: each cell gets the oil potential (eq. 5) of p_datum at
 * the top depth, s_w = sw0; BHP wells start at target, rate wells 10 bar
 * above the oil pressure of their first perforated cell; t = 0. */
sim_status sim_init_hydrostatic(sim_t h, double p_datum, double sw0);

/* State in caller buffers: p, sw (n each), pb (n_wells); host or device.
 * sim_get_state skips any output passed as NULL. */
sim_status sim_set_state(sim_t h, const double *p, const double *sw, const double *pb, double t);
sim_status sim_get_state(sim_t h, double *p, double *sw, double *pb, double *t);

/* Store the accumulation of the current state as the old time level
 * (eq. 15) and set the step length used by sim_assemble. */
sim_status sim_begin_step(sim_t h, double dt);

/* Residual and Jacobian at the current iterate (eq. 17 with eq. 18
 * upstreaming and eq. 10 wells), b = -F, plus the scaled residual norm
 * (max over cells of |R| dt / (rho_ref V phi) and over wells of |R|). */
sim_status sim_assemble(sim_t h, double *scaled_norm);

/* Solve J y = b for the assembled system: decouple (eq. 29), reorder
 * (eqs. 30-32), build RAS and AMG, run FGMRES(restart) with CPR-FPF
 * (Algorithm 2) to ||b - J y|| <= tol ||b|| on the decoupled system or
 * max_lin iterations.  y stays on the device (read it with sim_ls_export,
 * SIM_X_SOLUTION, on sim_linear_system(h)).
 * SIM_ERR_ARG when tol is negative or not finite. */
sim_status sim_linear_solve(sim_t h, double tol, int *iters, double *relres);

/* One Newton iteration of Algorithm 1 at the current step length:
 * assemble, test, solve, x += y.  *converged = 1 when the test passed
 * (then nothing is solved). */
sim_status sim_newton_step(sim_t h, int *converged, sim_stats *st);

/* Advance n_steps time steps of options.dt: Newton per step, halving the
 * step on failure (max_cuts per step).  SIM_ERR_NOT_CONVERGED / SIM_ERR_NAN
 * when a step could not be completed (the state is the last good one). */
sim_status sim_advance(sim_t h, int n_steps, sim_stats *st);

sim_status sim_get_stats(sim_t h, sim_stats *st);

/* A schedule change ("various operation constraints ... at different time
 * stage"): from the next step on, well w has this control, target and BHP
 * limit (as in sim_well).  A well put on BHP gets p_b = target; a well put
 * on a rate starts 10 bar above (injector) or below (producer) the oil
 * pressure of its first perforated cell; a shut well keeps p_b.
 * Errors: SIM_ERR_ARG for a bad well index or a control the well's kind
 * does not allow. */
sim_status sim_set_well(sim_t h, int w, int control, double target, double bhp_limit);

/* Current control and target of every well (n_wells entries each, host
 * arrays; either may be NULL): after a switch to the BHP limit, SIM_BHP and
 * the limit. */
sim_status sim_get_well_controls(sim_t h, int *control, double *target);

/* The simulator's linear system (borrowed handle, valid until sim_destroy). */
sim_ls_t sim_linear_system(sim_t h);

/* ---- linear-system level (used by sim_*, exposed for callers that bring
 *      their own Jacobian, and for testing each stage) ---- */

/* A 2x2-block system over n = nx*ny*nz cells plus n_wells padded well rows.
 * rowptr (n+n_wells+1), cols (nnzb): host arrays, columns sorted per row;
 * well_cell0[w] = first perforated cell of well w (fixes its subdomain).
 * The pattern must be structurally symmetric.  Errors: SIM_ERR_ARG for
 * NULL arrays, sizes < 1 or above sim_create's 50M cells, and the option
 * values sim_create rejects (dt is not used here), SIM_ERR_OOM,
 * SIM_ERR_CUDA. */
sim_status sim_ls_create(sim_ls_t *out, int nx, int ny, int nz, int n_wells,
                         const int *rowptr, const int *cols, const int *well_cell0,
                         const sim_options *o);
void sim_ls_destroy(sim_ls_t ls);

/* Values (4 per block, row-major: [dR_oil/dp, dR_oil/ds; dR_w/dp, dR_w/ds]),
 * right-hand side (2 per block row) and reordering key (oil potential, n):
 * host or device. */
sim_status sim_ls_set(sim_ls_t ls, const double *vals, const double *b, const double *key);

/* Decoupling, reordering, RAS factorisation and AMG hierarchy. */
sim_status sim_ls_setup(sim_ls_t ls);

/* FGMRES from y = 0 on the (decoupled) system; y: 2 per block row, host
 * or device.  SIM_ERR_NOT_CONVERGED is NOT returned for an iteration cap:
 * check *relres.  SIM_ERR_ARG when tol is negative or not finite. */
sim_status sim_ls_solve(sim_ls_t ls, double tol, double *y, int *iters, double *relres);

/* Apply one operator of the set-up system to x (2 per block row; for
 * SIM_OP_VCYCLE n pressure values), host or device:
 * SIM_OP_SPMV y = A x, SIM_OP_RAS y = R(A)^{-1} x, SIM_OP_VCYCLE one V-cycle
 * on A_pp, SIM_OP_CPR Algorithm 2.  A is the decoupled matrix. */
enum { SIM_OP_SPMV = 0, SIM_OP_RAS = 1, SIM_OP_VCYCLE = 2, SIM_OP_CPR = 3 };
sim_status sim_ls_apply(sim_ls_t ls, int op, const double *x, double *y);

/* ||b - A x||_2 for the current system (the decoupled one after
 * sim_ls_setup): x is 2 values per block row, host or device; the norm is
 * returned in host memory.  Uses device scratch that the library allocates
 * (the residual vector and per-block partial sums); synchronises the
 * stream.  The sum is deterministic (fixed order).  Errors: SIM_ERR_ARG for
 * NULL arguments, SIM_ERR_CUDA / SIM_ERR_OOM from the runtime. */
sim_status sim_ls_residual_norm(sim_ls_t ls, const double *x, double *norm);

/* The same norm as sim_ls_residual_norm for callers that must not allocate
 * memory: code that runs under another allocator's budget (for example a
 * framework whose caching allocator already holds the device memory, where a
 * fresh cudaMalloc can fail), and latency-sensitive loops in which the
 * device-wide synchronisation of cudaMalloc / cudaFree is unacceptable.
 * There is no counterpart of this entry point in the paper.
 *
 * Nothing is allocated: the per-block partial sums use a fixed device array
 * inside the library (4096 doubles, 32 KB, held by every GPU that loads the
 * library until the process exits).  Limit: n + n_wells <= 4096 * 4096
 * block rows; larger systems get SIM_ERR_ARG.  The handle, x (2 per block
 * row) and norm (one double) must all be on the current device, and x and
 * norm must be device memory (SIM_ERR_ARG otherwise, before any launch); the
 * result is written to *norm on the handle's stream and the call does not
 * synchronise.  The first call on a handle looks up the array's device
 * address (with the handle's device current) and keeps it in the handle;
 * make that first call before capturing the stream into a CUDA graph.  All
 * calls share the array: calls whose work overlaps on the GPU (another
 * stream, another thread, another handle) race on it and must be ordered by
 * the caller.  Each call overwrites every partial it reads, so no clearing
 * is needed. */
sim_status sim_ls_residual_norm_noalloc(sim_ls_t ls, const double *x_dev, double *norm_dev);

/* Copy internal arrays to host memory for inspection.  what / index:
 *  SIM_X_VALS, 0      decoupled block values (4*nnzb doubles)
 *  SIM_X_RHS, 0       decoupled right-hand side (2*nb doubles)
 *  SIM_X_SOLUTION, 0  last solution y (2*nb doubles)
 *  SIM_X_ROWPTR, 0    block row pointers (nb+1 ints)
 *  SIM_X_COLS, 0      block columns (nnzb ints)
 *  SIM_X_KEY, 0       reordering key (n doubles)
 *  SIM_X_AMG_SIZES, l int[6]: n, nnz, nnzP, nc, pmis_rounds, coarsest_dense
 *                     (index -1: int[1] = number of levels)
 *  SIM_X_AMG_RP/CI/V, l   level-l CSR of A (int, int, double)
 *  SIM_X_AMG_CF, l        C/F marks (int8: 1 = C, -1 = F)
 *  SIM_X_AMG_PRP/PCI/PV, l  interpolation P of level l
 *  SIM_X_RAS_SIZES, s int[3]: owned rows, extended rows, local nnzb
 *                     (index -1: int[1] = number of subdomains)
 *  SIM_X_RAS_EXT, s   global rows of subdomain s in local (reordered) order
 *  SIM_X_RAS_LEVELS, s int[2*next+2]: number of L levels, number of U
 *                     levels, then the L level and the U level of each row
 * *needed receives the byte size; dst may be NULL to query it. */
enum {
  SIM_X_VALS = 0, SIM_X_RHS = 1, SIM_X_SOLUTION = 2, SIM_X_ROWPTR = 3, SIM_X_COLS = 4, SIM_X_KEY = 5,
  SIM_X_AMG_SIZES = 10, SIM_X_AMG_RP = 11, SIM_X_AMG_CI = 12, SIM_X_AMG_V = 13,
  SIM_X_AMG_CF = 14, SIM_X_AMG_PRP = 15, SIM_X_AMG_PCI = 16, SIM_X_AMG_PV = 17,
  SIM_X_RAS_SIZES = 20, SIM_X_RAS_EXT = 21, SIM_X_RAS_LEVELS = 22
};
sim_status sim_ls_export(sim_ls_t ls, int what, int index, void *dst, size_t bytes, size_t *needed);

/* Per-kernel-family timing with CUDA events recorded on the library stream
 * around each launch of the enabled families.  mask: bit (1 << SIM_T_*) per
 * family, 0 = off; enabling resets the counters.  sim_kernel_time returns,
 * for one family, the number of timed launches and their summed
 * milliseconds. */
enum { SIM_T_NONE = 0, SIM_T_SPMV64 = 1, SIM_T_SPMV_PREC = 2, SIM_T_RAS = 3, SIM_T_VCYCLE = 4,
       SIM_T_ORTHO = 5, SIM_T_ASSEMBLE = 6, SIM_T_AMG_SETUP = 7, SIM_T_RAS_SETUP = 8, SIM_T_DECOUPLE = 9,
       SIM_T_WARMSTART = 10 /* the whole learned initial guess */, SIM_T_NETWORK = 11 /* its network forward */,
       SIM_T_NFAMILIES = 12 };
sim_status sim_kernel_timer(sim_ls_t ls, unsigned mask);
sim_status sim_kernel_time(sim_ls_t ls, int which, long long *launches, double *ms);

/* Launch mode of the FGMRES Arnoldi step (Algorithm 1's inner loop: CPR
 * application, SpMV, Gram-Schmidt, Givens update).  The paper has no
 * counterpart: it concerns only how the kernels are issued.
 *   mode = 2: a whole restart cycle runs from one launch of a CUDA graph
 *     whose WHILE node replays the recorded step and, after each step,
 *     decides on the device whether to go on (residual estimate above
 *     tol * ||b||, h_{j+1,j} nonzero and finite, steps left in the cycle and
 *     in max_lin); the host waits once per cycle.
 *   mode = 1 (the default): each step is one replay of a CUDA graph
 *     recorded at the first solve after a setup, whose kernels read the step
 *     index from device memory; the host waits after every step and takes
 *     the same decision.
 *   mode = 0: every kernel is launched on its own.
 * All modes issue the same kernels on the same data, so results are
 * bit-identical.  Kernel timers work in modes 0 and 1 (graph brackets are
 * event nodes); with timers on, mode 2 runs as mode 1.  Subdomains too large
 * for the shared-memory RAS kernel always use separate launches; a driver
 * that cannot record the WHILE node leaves mode 1 in use.  The mode the last
 * FGMRES solve actually used is returned by sim_ls_graph_mode (-1 before the
 * first solve).  On the 1M-cell channelised case mode 2 measured about 1%
 * slower per time step than mode 1 (the body relaunch inside the WHILE node
 * costs more than the host's wait and relaunch), hence the default.
 * Errors: SIM_ERR_ARG for a NULL handle or a mode outside 0..2. */
sim_status sim_ls_step_graph(sim_ls_t ls, int mode);
sim_status sim_ls_graph_mode(sim_ls_t ls, int *mode);

/* ---- ensembles: many independent models advanced together ----
 *
 * Not in the paper, whose experiments run one model at a time.  A batch
 * holds n_members simulators (each created as by sim_create from grids[k],
 * rocks[k], fluids[k], wells[k][0..n_wells[k]) and opts[k]; opts[k].cuda_stream
 * is ignored: every member gets a non-blocking stream of its own).  Members
 * share no data, so a member's results are those of the same model run
 * alone.  The batch owns the members; sim_batch_member lends one (valid until
 * sim_batch_destroy) for sim_init_hydrostatic, sim_set_state, sim_get_state,
 * sim_get_stats and the rest of the single-model calls.  n_workers host
 * threads (0 = 8) advance the members concurrently, largest grids first.
 * Errors: SIM_ERR_ARG, SIM_ERR_OOM, SIM_ERR_CUDA; a member that fails to be
 * created fails the whole call (nothing is left allocated). */
typedef struct sim_batch_s *sim_batch_t;
sim_status sim_batch_create(sim_batch_t *out, int n_members, const sim_grid *grids, const sim_rock *rocks,
                            const sim_fluid *fluids, const sim_well *const *wells, const int *n_wells,
                            const sim_options *opts, int n_workers);
void sim_batch_destroy(sim_batch_t b);
sim_status sim_batch_member(sim_batch_t b, int k, sim_t *member);
sim_status sim_batch_size(sim_batch_t b, int *n_members, int *n_workers);

/* Advance every member by n_steps time steps (sim_advance on each).  stats
 * (n_members, may be NULL) receives each member's cumulative statistics and
 * status (n_members, may be NULL) each member's return code.  Returns the
 * first failing member's code (in member order) with its message, after all
 * members have run; SIM_OK when every member completed its steps. */
sim_status sim_batch_advance(sim_batch_t b, int n_steps, sim_stats *stats, sim_status *status);

/* Pick the worker count: for each of candidates[0..n_candidates) advance the
 * `sample` largest members (sample < 1: twice the largest candidate) by one
 * time step, timing it on the host (seconds[c], may be NULL), then restore
 * those members' states and statistics exactly.  The fastest count becomes
 * the batch's worker count and is returned in *chosen. */
sim_status sim_batch_autotune(sim_batch_t b, const int *candidates, int n_candidates, int sample, int *chosen,
                              double *seconds);

/* ---- learned warm start: a 3D convolutional network that predicts the
 *      Newton update, used as the FGMRES initial guess ----
 *
 * Not in the paper.  The network is a U-Net over 4 resolution levels
 * (3x3x3 convolutions, 32 channels, ReLU, average-pool down, nearest up,
 * skip concatenation) on the simulator's grid; all its contractions run
 * as BF16 tensor-core MMAs with FP32 accumulation (mma.sync, or tcgen05
 * with TMEM accumulators for the forward and data-gradient convolutions, see
 * sim_ws_use_tcgen05), for inference and for training (Adam with FP32 master
 * weights).  It is grid-size agnostic: weights trained on one grid apply to
 * any other.  Inputs per cell (8 channels): the Newton residual, i.e. the
 * decoupled right-hand side b (pressure and saturation rows, each over its
 * rms over the cells), (ln k - 4) / 2, 4 (s_w - 0.5), the previous solve's
 * update (each component over its rms; zero before the first solve) and two
 * zero channels.  Output: the shape of the update, each component (pressure,
 * saturation) with unit rms over the cells; well rows are not predicted (0).
 * The two components enter the initial guess as separate candidates whose
 * scales a least-squares fit sets (sim_ws_attach).  The head layer starts at
 * zero: an untrained network predicts nothing.  A handle is used by one caller at a time (calls
 * on it are serialised internally). */
typedef struct sim_ws_s *sim_ws_t;
sim_status sim_ws_create(sim_ws_t *out, unsigned long long seed);   /* He-normal weights from seed, zero head */
void sim_ws_destroy(sim_ws_t ws);
/* Convolution kernels: on = tcgen05 MMAs with TMEM accumulators for the
 * forward and data-gradient passes; off (default, faster with the current
 * per-tap staging) = the mma.sync kernels.  The head layer and the weight
 * gradients always use mma.sync.  Both compute the same contraction in BF16
 * with FP32 accumulation. */
sim_status sim_ws_use_tcgen05(sim_ws_t ws, int on);

/* Parameters in layer order (c00 c01 c10 c11 c20 c21 c30 c31 d20 d21 d10 d11
 * d00 d01 h), each as W[27][Co][Ci] (tap t = (dx+1) + 3 (dy+1) + 9 (dz+1))
 * then b[Co].  which = 0: the FP32 master weights; 1: the accumulated
 * gradients divided by the number of samples accumulated.  dst == NULL
 * returns the count in *needed. */
sim_status sim_ws_params(sim_ws_t ws, int which, float *dst, size_t n, size_t *needed);
/* Replace the weights (same layout, exactly the count) and reset Adam. */
sim_status sim_ws_set_params(sim_ws_t ws, const float *src, size_t n);

/* Network output for one grid: feat [nz][ny][nx][8] FP32 (rounded to BF16 on
 * the device), y [nz][ny][nx][8] FP32 (channels 0-1 are the prediction).
 * Host or device pointers. */
sim_status sim_ws_forward(sim_ws_t ws, int nx, int ny, int nz, const float *feat, float *y);
/* Forward, loss 0.5/n sum over cells of |y[0:2] - target|^2 (target
 * [n][2]), and backward: gradients are added to the accumulated ones. */
sim_status sim_ws_backward(sim_ws_t ws, int nx, int ny, int nz, const float *feat, const float *target,
                           double *loss);
sim_status sim_ws_zero_grad(sim_ws_t ws);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with the mean accumulated
 * gradient, then the gradients are cleared. */
sim_status sim_ws_adam(sim_ws_t ws, double lr);

/* Record: every linear solve of h appends its (features, target) pair, the
 * target being the solved update with each component over its rms, to ws's
 * dataset (device memory).  NULL stops recording. */
sim_status sim_ws_record(sim_t h, sim_ws_t ws);
sim_status sim_ws_dataset(sim_ws_t ws, int *n_samples);
/* Train on the dataset: `epochs` passes in a seeded random order, an Adam
 * step every `batch` samples; *mean_loss = mean loss of the last epoch.
 * SIM_ERR_STATE when nothing was recorded. */
sim_status sim_ws_train(sim_ws_t ws, int epochs, int batch, double lr, unsigned long long seed, double *mean_loss);
sim_status sim_ws_eval(sim_ws_t ws, double *mean_loss);

/* Attach a network to a simulator (NULL detaches).  Every linear solve then
 * starts from the least-squares combination, on the decoupled system, of
 * the network's predicted update (its pressure and saturation parts as two
 * candidates) and (at the first Newton iteration of a time step) the
 * previous step's first update: the x0 in their span with the
 * smallest ||b - J x0||.  The network's term is kept only when it lowers that
 * residual (ws_used), else it is dropped (ws_fallback: the previous step's
 * first update alone where there is one, else zero); the guess is never
 * worse than zero.  The stopping test stays
 * ||b - J y|| <= tol ||b||, so the converged update meets the same
 * tolerance either way.  sim_init_hydrostatic clears the history. */
sim_status sim_ws_attach(sim_t h, sim_ws_t ws);

/* Number of this library's kernel launches issued so far (all handles). */
long long sim_launch_count(void);

const char *sim_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
