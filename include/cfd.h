/*
 * cfd.h -- C-ABI of the GB300 (sm_103a) lid-driven-cavity projection path.
 *
 * The operation is the time step of a 3D lid-driven cavity on a staggered
 * (MAC) grid, advanced by the fractional-step method of arXiv 2504.03697
 * ("cfdSCOPE"), Sec. 3 and 3.1: external forces, semi-Lagrangian advection,
 * a pressure Poisson solve by (preconditioned) conjugate gradients, and the
 * pressure correction; Table 1 names the same phases (applyForces,
 * solveAdvection, solvePressureCorrection / pcg, applyPressureCorrection).
 * A backward-Euler viscosity substep (not in the paper's inviscid model) runs
 * between advection and projection when nu > 0.
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid: nx * ny * nz cubic cells of edge h = length / nx.  Arrays are
 * float64, x fastest, then y, then z:
 *   U: (nx+1) * ny * nz   V: nx * (ny+1) * nz   W: nx * ny * (nz+1)
 *   P: nx * ny * nz       (cell centres)
 * The lid is the y = ny*h wall, moving in +x at lid_u; every other wall is
 * at rest.  Normal velocity on the walls is zero.
 *
 * Memory ownership: the caller owns all device memory.  It asks for the
 * workspace size with cfd_workspace_bytes, allocates one device buffer of at
 * least that many bytes (256-byte aligned), and passes it to cfd_create; the
 * library never allocates device memory.  The handle itself lives in host
 * memory (malloc) and is freed by cfd_destroy, which does not touch the
 * workspace.
 *
 * Streams: every call enqueues its work on the stream given to cfd_create
 * (or cfd_set_stream).  Calls that return statistics or copy to host memory
 * synchronise that stream before returning; the others are asynchronous.
 *
 * Errors: every int-returning call returns one of the CFD_* codes below;
 * cfd_last_error(h) returns a static, human-readable description of the
 * last failure on that handle (h may be NULL for failures before a handle
 * exists).  Solver outcomes (not converged, breakdown, device-wait timeout)
 * leave the fields holding the last iterate.
 */
#ifndef CFD_GB300_H
#define CFD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t (a CUstream_st pointer); pass torch.cuda.current_stream().cuda_stream */
typedef struct CUstream_st *cfd_stream_t;
typedef struct cfd_handle cfd_handle;

enum {
  CFD_OK = 0,
  CFD_ERR_INVALID_ARG = -1,
  CFD_ERR_CUDA = -2,
  CFD_ERR_NOT_CONVERGED = -3,      /* iteration cap reached; fields hold the last iterate */
  CFD_ERR_BREAKDOWN = -4,          /* NaN/Inf or p^T A p <= 0 inside CG */
  CFD_ERR_TIMEOUT = -5,            /* a bounded device-side wait gave up */
  CFD_ERR_WORKSPACE_TOO_SMALL = -6
};

enum { CFD_FIELD_U = 0, CFD_FIELD_V = 1, CFD_FIELD_W = 2, CFD_FIELD_P = 3 };

/* Pressure solver (Sec. 3.1: PCG with an optional preconditioner).
 *   CG      unpreconditioned conjugate gradients, FP64
 *   JACOBI  Jacobi-preconditioned CG, FP64 (the paper's optimised variant)
 *   IR      FP32 CG (vectors and stencil in FP32, partial sums reduced and
 *           CG scalars formed in FP64) with FP64 iterative refinement:
 *           each time the FP32 residual has fallen by ir_delta, x gathers
 *           the FP32 correction in FP64 and the FP64 true residual
 *           b - A x replaces the FP32 one, keeping the search direction.
 *           Convergence is judged on the FP64 true residual only.  Stats:
 *           iters = FP32 iterations, outer_iters = FP64 refinements.  The
 *           diffusion solves of the step (nu > 0) run the same way on the
 *           velocity matrices I + c L (no mean removal; refinement every
 *           ir_delta, default 1e-4).
 *   DIC     CG preconditioned by the simplified diagonal-based incomplete
 *           Cholesky factorisation (the paper's default): pivots d_c = n_c
 *           - sum of 1/d over the x-1, y-1, z-1 neighbours, M = (D + L)
 *           D^-1 (D + L^T), applied by two hyperplane-wavefront triangular
 *           sweeps (exactly the sequential recurrences).  FP64, host-driven
 *           iteration; calls using it synchronise the stream.  Pressure only
 *           (the diffusion solves use CG); not available in batches.
 *   FPCG    flexible PCG with the learned U-Net preconditioner attached by
 *           cfd_attach_preconditioner; pressure only; not available in
 *           batches.  Two forms (cfd_set_fpcg_form):
 *             GRAPH (default) flexible CG with FP32 vectors and FP64
 *                   reliable-update refinement, as the IR solver, with
 *                   z = M(r) from the network in every FP32 iteration, the
 *                   Polak-Ribiere beta, and the switch to plain CG (after
 *                   50 iterations without halving the residual norm, or a
 *                   breakdown) decided on the device: one CUDA graph per
 *                   solve, no host round trip per iteration.  Convergence
 *                   on the FP64 true residual.  Stats: iters = FP32
 *                   iterations, outer_iters = FP64 refinements, restarts =
 *                   iterations run as plain CG.  The diffusion solves of
 *                   the step then run as in IR (mixed precision).  Needs
 *                   nx % 4 == 0 (the network's grids do).
 *             HOST  the FP64 flexible PCG of cfd_unet_fpcg_solve (cold
 *                   start, host-driven; stats as documented there); the
 *                   diffusion solves run in FP64 CG.                      */
enum { CFD_SOLVER_CG = 0, CFD_SOLVER_JACOBI = 1, CFD_SOLVER_IR = 2, CFD_SOLVER_DIC = 3, CFD_SOLVER_FPCG = 4 };

/* Substeps for cfd_substep (kernel-level access to one phase of the step). */
enum {
  CFD_SUBSTEP_FORCES = 0,   /* applyForces: top-layer faces += dt * g            */
  CFD_SUBSTEP_ADVECT = 1,   /* solveAdvection: semi-Lagrangian, old -> new field  */
  CFD_SUBSTEP_DIFFUSE = 2,  /* backward-Euler viscosity (three CG solves)         */
  CFD_SUBSTEP_PROJECT = 3   /* divergence, pressure solve, correction, gauge      */
};

typedef struct {
  int32_t nx, ny, nz;       /* cells per axis, each >= 1                          */
  double length;            /* box edge along x (h = length / nx), > 0            */
  double dt;                /* time step, > 0                                     */
  double rho;               /* density, > 0                                       */
  double nu;                /* kinematic viscosity, >= 0 (0: no diffusion step)   */
  double lid_u;             /* lid speed along +x                                 */
  double g[3];              /* forcing offset per unit time on the top cell layer */
  int32_t solver;           /* CFD_SOLVER_*                                       */
  double rtol;              /* ||b - A x||_2 <= rtol ||b||_2 (true FP64 residual)  */
  int32_t max_iters;        /* CG iteration cap per solve; 0 -> 20 * max(n)       */
  int32_t warm_start;       /* 1: start the pressure solve from the previous p    */
  double ir_delta;          /* IR: refine in FP64 each time the FP32 residual has
                               fallen by this factor, in (0, 1); 0 -> 0.01 for
                               the pressure solve (the FP32 recurrence keeps the
                               iteration count of FP64 CG over two decades, not
                               over three), 1e-4 for the diffusion solves
                               (well-conditioned systems)                        */
  int32_t advect_order;     /* backtrace: 0 or 1 explicit Euler x - dt v(x); 2 the
                               explicit midpoint rule x - dt v(x - dt/2 v(x))     */
  int32_t learned_guess;    /* 1 (solver IR, with a U-Net attached by
                               cfd_attach_preconditioner): every pressure solve
                               starts from x0 = alpha M(b), M the network
                               (cfd_unet_apply) and alpha = M(b).b / M(b).A M(b),
                               the multiple of M(b) of least energy-norm error;
                               with warm_start = 1 the network corrects the
                               warm start instead: x0 = x + alpha M(r), r =
                               b - A x, alpha = M(r).r / M(r).A M(r); graph form
                               of the IR solve only; 0: cold (or warm) start    */
  int32_t reserved[6];      /* must be zero                                       */
} cfd_params;

typedef struct {
  int32_t iters;            /* pressure CG iterations (IR: inner, summed)         */
  int32_t outer_iters;      /* IR refinement steps (0 for CG / JACOBI)            */
  int32_t restarts;         /* restarts from the true residual                   */
  int32_t status;           /* CFD_OK or the solver code of this solve            */
  int32_t diff_iters[3];    /* diffusion CG iterations for u, v, w (0 if nu = 0)  */
  int32_t diff_status;      /* worst status of the three diffusion solves         */
  double rel_resid;         /* true ||b - A x|| / ||b|| of the pressure solve     */
  double b_norm;            /* ||b||_2 of the pressure right-hand side            */
} cfd_solve_stats;

/* Size in bytes of the device workspace cfd_create needs for these params.
 * Returns CFD_ERR_INVALID_ARG for an invalid parameter set. */
int cfd_workspace_bytes(const cfd_params *params, size_t *bytes);

/* Create a cavity on the given workspace (device pointer, >= the size from
 * cfd_workspace_bytes, 256-byte aligned).  The initial state is v = 0,
 * p = 1 (Sec. 3, eq. 3).  On success *out holds a new handle. */
int cfd_create(const cfd_params *params, void *dev_ws, size_t bytes, cfd_stream_t stream,
               cfd_handle **out);

/* Free the host-side handle.  The workspace stays the caller's. */
void cfd_destroy(cfd_handle *h);

/* Static description of the last failure on h (or of the last failure
 * without a handle when h is NULL).  Never returns NULL. */
const char *cfd_last_error(const cfd_handle *h);

/* Change the stream subsequent calls enqueue on. */
int cfd_set_stream(cfd_handle *h, cfd_stream_t stream);

/* Copy a whole field (layout above) into the cavity.  src is a device
 * pointer when src_on_device != 0, else a host pointer (pinned memory gives
 * an asynchronous copy).  Wall-normal velocity faces are forced to zero. */
int cfd_set_field(cfd_handle *h, int field, const double *src, int src_on_device);

/* Copy a whole field out; dims_out (nullable) receives its (x, y, z) sizes.
 * A host destination synchronises the stream. */
int cfd_read_field(cfd_handle *h, int field, double *dst, int dst_on_device, int64_t dims_out[3]);

/* Advance nsteps fractional steps (Sec. 3.1).  per_step (nullable) receives
 * nsteps entries; when given, the call synchronises and returns the worst
 * solver status seen; otherwise it returns after enqueueing. */
int cfd_step(cfd_handle *h, int nsteps, cfd_solve_stats *per_step);

/* Statistics of the last n steps taken by cfd_step (oldest first; n at
 * most 1024 and at most the number of steps taken).  Synchronises the
 * stream; returns the worst solver status among them.  Lets a caller run
 * steps asynchronously (per_step = NULL) and inspect them afterwards. */
int cfd_recent_stats(cfd_handle *h, int n, cfd_solve_stats *out);

/* Run one substep (CFD_SUBSTEP_*) of the step on the current state.
 * stats (nullable) as for cfd_step. */
int cfd_substep(cfd_handle *h, int which, cfd_solve_stats *stats);

/* Standalone Neumann-Poisson solve A x = b with the handle's solver, rtol
 * and grid (the pressure system of Sec. 3.1; A = -h^2 * 7-point Laplacian).
 * b_dev, x_dev: device arrays of nx*ny*nz float64.  b is read only; the
 * mean of b is removed internally.  x is overwritten (cold start from 0,
 * or from its contents when warm_start = 1); no gauge shift is applied.
 * stats (nullable) receives iterations and the true residual; the call
 * synchronises when stats is given. */
int cfd_solve_pressure(cfd_handle *h, const double *b_dev, double *x_dev, cfd_solve_stats *stats);

/* y = A x for the Neumann pressure matrix A (scaled by h^2: row c has
 * n_c on the diagonal and -1 for each of its n_c neighbours).  x_dev and
 * y_dev: device arrays of nx*ny*nz float64, not overlapping.  This is the
 * paper's SpMV (Sec. 3.1, Table 1 "spmv"), matrix-free. */
int cfd_apply_poisson(cfd_handle *h, const double *x_dev, double *y_dev);

/* Number of kernels this handle has run since creation (for launch
 * accounting in benchmarks).  Kernels inside the graph form of the
 * mixed-precision solve are counted on the device; when that form has run,
 * the call synchronises the handle's stream to read the count. */
int64_t cfd_launch_count(const cfd_handle *h);

/* Launch shape of the persistent CG solves (the knobs the autotuner
 * searches): blocks per SM (1..the co-resident maximum) and stencil tile
 * depth (cells per thread along z: 1, 2, 4 or 8).  0 selects the built-in
 * heuristic, which prefers the register path on small grids (each block
 * keeps its cells' search direction and operator output in registers
 * between the two phases of an iteration).  Applies to later solves.
 * Results are bitwise reproducible for a fixed shape; different shapes sum
 * the reductions in different orders. */
int cfd_set_solver_shape(cfd_handle *h, int blocks_per_sm, int tile_depth);

/* Form of the unpreconditioned FP64 CG solves (CFD_SOLVER_CG pressure
 * solves and the diffusion solves); both give the same iterates in exact
 * arithmetic (Sec. 3.1 CG):
 *   SINGLE_REDUCTION  (default) Chronopoulos-Gear form: w = A r and s = A p
 *                     carried by recurrence, r.r and w.r reduced together,
 *                     one grid-wide reduction per iteration;
 *   TWO_REDUCTIONS    textbook form, p.q then r.r (two per iteration).
 * Jacobi-preconditioned and batched solves always use the textbook form. */
enum { CFD_CG_SINGLE_REDUCTION = 0, CFD_CG_TWO_REDUCTIONS = 1 };
int cfd_set_cg_variant(cfd_handle *h, int variant);

/* Execution form of the CFD_SOLVER_IR pressure solve (same method, same
 * stopping rule):
 *   PERSISTENT  one cooperative kernel per solve, two grid-wide reductions
 *               per FP32 iteration (any grid);
 *   GRAPH       one CUDA graph per solve whose device-side while loops run
 *               the FP32 iterations as two streaming kernels (direction +
 *               operator, update) and the FP64 refinements as separate
 *               kernels; each kernel's last block updates the solver scalars
 *               and the loop conditions.  Needs nx % 4 == 0.
 *   AUTO        (default) GRAPH when nx % 4 == 0, PERSISTENT otherwise
 *               (the graph form measured faster at every size from 64^3 to
 *               384^3).
 * The diffusion solves of the step follow the same form (in the GRAPH form
 * on float4 lanes over FP32 rows padded to a multiple of 4 cells, any
 * width).
 * Errors: unknown form; GRAPH with nx % 4 != 0.  Batches run the batched
 * graph form: each cavity's solve inside one persistent cooperative launch. */
enum { CFD_IR_AUTO = 0, CFD_IR_PERSISTENT = 1, CFD_IR_GRAPH = 2 };
int cfd_set_ir_form(cfd_handle *h, int form);

/* Form of the CFD_SOLVER_FPCG pressure solve (see CFD_SOLVER_FPCG).
 * Errors: unknown form; a handle whose solver is not FPCG. */
enum { CFD_FPCG_GRAPH = 0, CFD_FPCG_HOST = 1 };
int cfd_set_fpcg_form(cfd_handle *h, int form);

/* Run the three diffusion solves of a step (nu > 0) at once (on = 1): u on
 * the handle's stream, v and w on two internal streams forked from and
 * joined back to it, each solve with its own solver vectors and a third of
 * the co-resident blocks.  Same method, results within rounding of the
 * sequential solves (their reductions run over other block counts).
 * Available on grids of at most 2^21 cells with nu > 0 (the workspace then
 * holds the two extra vector sets), where it is on from cfd_create; not
 * used with CFD_SOLVER_IR (its solves share one set of FP32 vectors) nor
 * inside batches.  Errors: on not 0/1; on = 1 without that workspace. */
int cfd_set_concurrent_diffusion(cfd_handle *h, int on);

/* Autotuner of the solver shape for this handle's grid and solver: times
 * fixed-length pressure solves (iters iterations, a deterministic hashed
 * right-hand side) with the automatic shape and with every blocks_per_sm in
 * {1, 2, 3, 4} x tile_depth in {1, 2, 4, 8} -- for CFD_SOLVER_CG under both
 * CG forms (cfd_set_cg_variant); for CFD_SOLVER_IR these shapes in the
 * persistent form plus the graph form when nx % 4 == 0 -- keeps the fastest
 * (as by cfd_set_solver_shape, cfd_set_cg_variant and cfd_set_ir_form;
 * shape 0 / 0 when the automatic one wins) and reports it.  Uses the intermediate-velocity
 * scratch; the state (u, v, w, p) is not touched.  Call between steps;
 * synchronises the stream. */
typedef struct {
  int32_t blocks_per_sm;    /* chosen (0: automatic)                            */
  int32_t tile_depth;       /* chosen (0: automatic)                            */
  int32_t candidates;       /* configurations timed                             */
  float ms_auto;            /* ms per fixed-length solve, automatic shape       */
  float ms_best;            /* ms per fixed-length solve, chosen configuration  */
  int32_t cg_variant;       /* chosen CFD_CG_* form                             */
  int32_t ir_form;          /* chosen CFD_IR_* form (CFD_SOLVER_IR handles)     */
} cfd_tune_report;
int cfd_autotune_solver(cfd_handle *h, int32_t iters, cfd_tune_report *rep);

/* The shape the next solve of `kind` (0 pressure, 1..3 diffusion of u, v,
 * w) would use: grid size, tile depth, and the path: *register_path is 0
 * for the memory path, 1 for the register path, 2 for the tile-resident
 * single-reduction FP64 CG (one block of 256 threads per 32 x 8 x 8 tile,
 * every CG vector of the tile in registers; taken by unpreconditioned
 * single-reduction CG solves with the automatic shape when the tiles number
 * more than half of the SMs and at most one per SM, e.g. 64^3, and not by
 * the diffusion solves while cfd_set_concurrent_diffusion runs them at
 * once).  Each output pointer may be NULL. */
int cfd_get_solver_shape(cfd_handle *h, int kind, int *blocks, int *tile_depth, int *register_path);

/* Phase timers, mirroring the call tree of the paper's Table 1
 * (applyForces, solveAdvection, solvePressureCorrection -> pcg,
 * applyPressureCorrection) plus the diffusion substep.  CFD_PHASE_PCG
 * brackets exactly the pressure-solve kernel launch. */
enum {
  CFD_PHASE_FORCES = 0,
  CFD_PHASE_ADVECT = 1,
  CFD_PHASE_DIFFUSE = 2,
  CFD_PHASE_DIVERGENCE = 3,
  CFD_PHASE_PCG = 4,
  CFD_PHASE_CORRECT = 5,
  CFD_PHASE_COUNT = 6
};

/* on != 0: record a CUDA event pair on the handle's stream around every
 * phase of later calls (host-side event objects; no device allocation).
 * on == 0: stop recording (pending pairs stay until queried). */
int cfd_enable_timing(cfd_handle *h, int on);

/* Synchronise the stream, write the summed device time (ms) and the number
 * of recorded calls of each phase since the last query into ms_out /
 * calls_out (CFD_PHASE_COUNT entries each, nullable), and reset them. */
int cfd_phase_times(cfd_handle *h, double *ms_out, int64_t *calls_out);

/* ---------------------------------------------------------------------------
 * Batches of independent cavities (uneven sizes allowed) advanced together.
 * Each cavity is a full cfd_handle living in its own slice of the batch
 * workspace (set / read its fields through cfd_batch_cavity).  Per step the
 * sweeps run per cavity, and each family of solves (diffusion of u, v, w;
 * the pressure) is ONE cooperative persistent launch in which every cavity
 * owns a contiguous range of blocks sized in proportion to cells^(4/3) and
 * runs its own CG with its own reductions (cavities never wait on each
 * other).  All cavities of a batch use the same solver.  The number of
 * cavities is limited by the co-resident blocks of one launch (one block per
 * cavity at least).  Ownership and errors as for single cavities; errors
 * are described by cfd_batch_last_error. */
typedef struct cfd_batch cfd_batch;

int cfd_batch_workspace_bytes(int n, const cfd_params *per_cavity, size_t *bytes);
int cfd_batch_create(int n, const cfd_params *per_cavity, void *dev_ws, size_t bytes, cfd_stream_t stream,
                     cfd_batch **out);
void cfd_batch_destroy(cfd_batch *b);
const char *cfd_batch_last_error(const cfd_batch *b);

/* The handle of cavity i (owned by the batch; do not destroy it). */
cfd_handle *cfd_batch_cavity(cfd_batch *b, int i);

/* Advance every cavity nsteps steps.  per_cavity (nullable, n entries)
 * receives each cavity's solver statistics of the LAST step; when given the
 * call synchronises and returns the worst status. */
int cfd_batch_step(cfd_batch *b, int nsteps, cfd_solve_stats *per_cavity);

/* on != 0: capture one whole batch step into a CUDA graph at the next
 * cfd_batch_step and replay it for every later step (falls back to direct
 * launches if the capture is not possible; see cfd_batch_graph_active). */
int cfd_batch_use_graph(cfd_batch *b, int on);
int cfd_batch_graph_active(const cfd_batch *b);

/* Blocks of the batched launch `kind` (0..2 diffusion u, v, w; 3 pressure
 * CG; 4 pressure IR) and kernel launches issued so far. */
int cfd_batch_blocks(const cfd_batch *b, int kind, int *total_blocks);
int64_t cfd_batch_launch_count(const cfd_batch *b);

/* ---------------------------------------------------------------------------
 * Allocation-free standalone pressure solve.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory
 * at all (plug-ins whose host application owns every allocation, runtimes
 * that reserve all device memory up front), so they cannot provide the
 * workspace cfd_create needs.  It still calls the CUDA runtime (copies, a
 * memset, a kernel launch, a stream synchronisation when stats is given),
 * so it must not be called from inside a CUDA stream callback
 * (cudaLaunchHostFunc), where no CUDA call is allowed.
 *
 * Solves the same Neumann system as cfd_solve_pressure with plain FP64 CG
 * (cold start, mean of b removed, no gauge shift), in the two-reduction
 * (textbook) form: its fixed scratch has no room for the extra vectors of
 * the single-reduction form, so its rounding and iteration count can differ
 * slightly from cfd_solve_pressure's default form.  b_dev and x_dev are
 * device arrays of nx*ny*nz doubles (x fastest), b is read only, x is
 * overwritten.  rtol in (0, 1); max_iters = 0 means 20 * max(n).  stats
 * (nullable) as for cfd_solve_pressure; when given, the call synchronises
 * the stream.
 *
 * Its scratch vectors live in one fixed-size __device__ array inside this
 * library instead of a workspace, so it never calls an allocator.  Limits:
 *  - at most CFD_NOALLOC_MAX_CELLS cells (e.g. 64^3); larger grids return
 *    CFD_ERR_INVALID_ARG with a message from cfd_last_error(NULL);
 *  - every GPU that loads the library holds that array (about 11 MB)
 *    until the process exits;
 *  - all calls on a device share the array and it keeps the last call's
 *    contents, so calls whose GPU work overlaps (other streams, other host
 *    threads) race: serialise them on one stream;
 *  - the first call on each device looks up the array's device address
 *    (with that device current); make that first call before any stream
 *    capture.  A failed lookup is not remembered: the next call retries.
 * Errors are reported through cfd_last_error(NULL). */
#define CFD_NOALLOC_MAX_CELLS 262144
int cfd_poisson_solve_noalloc(int32_t nx, int32_t ny, int32_t nz, const double *b_dev, double *x_dev,
                              double rtol, int32_t max_iters, cfd_stream_t stream, cfd_solve_stats *stats);

/* Snapshot output (Sec. 3.2: the proxy app writes a CSV file of the state
 * each step for ParaView).  cfd_snapshot enqueues device->host copies of
 * u, v, w, p into a pinned host buffer owned by the handle (allocated on
 * first use, freed by cfd_destroy) on the handle's stream and returns; the
 * caller may enqueue the next cfd_step at once, so the copy and the
 * formatting below overlap the GPU work.  cfd_snapshot_write_csv waits for
 * that copy and writes the file: a header "x,y,z,u,v,w,p", then one line per
 * cell (x fastest): the cell centre ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h),
 * the cell-centred velocity (the mean of the two faces along each axis) and
 * p, each printed with 17 significant digits (exact round trip).  nthreads
 * host threads format z-slabs in parallel (<= 0: all hardware threads).
 * Returns CFD_ERR_INVALID_ARG without a pending snapshot or if the file
 * cannot be written. */
int cfd_snapshot(cfd_handle *h);
int cfd_snapshot_write_csv(cfd_handle *h, const char *path, int nthreads);

/* Pressure right-hand side of the projection (Sec. 3.1 "Projection"): the
 * scaled divergence -(rho h / dt) * sum of face differences of the current
 * velocity (u, v, w), one value per cell, written to b_dev (nx*ny*nz float64,
 * device).  The mean is NOT removed (the solvers remove it).  Asynchronous on
 * the handle's stream.  Used to harvest pressure systems from a run. */
int cfd_pressure_rhs(cfd_handle *h, double *b_dev);

/* One training pair of the learned preconditioner from a pressure system:
 * with b' = b - mean(b), r = b' - A xk is the residual of the iterate xk and
 * e = (xs - xk) - mean(xs - xk) its error against the converged solution xs
 * (the Neumann system fixes x only up to a constant), A the operator of
 * cfd_apply_poisson (Sec. 3.1).  All five are device arrays of nx*ny*nz
 * float64; r and e must not alias the inputs or each other.  Asynchronous on
 * the handle's stream (it uses the handle's partial-sum scratch, so it must
 * not overlap a solve of the same handle). */
int cfd_harvest_pair(cfd_handle *h, const double *b_dev, const double *xs_dev, const double *xk_dev, double *r_dev,
                     double *e_dev);

/* Time limit of each grid-wide wait inside the persistent solve kernels of
 * this handle (the all-reduce barrier of the CG and mixed-precision
 * kernels; default 2 s; UINT64_MAX restores the default).  A block that
 * waits longer records CFD_ERR_TIMEOUT, every other block leaves at its
 * next wait, and the solve returns CFD_ERR_TIMEOUT with the fields holding
 * whatever the kernel had written; the handle stays usable.  0 gives up at
 * the first wait that is not already satisfied (for tests of that path).
 * Waits for the tensor-memory copies keep their own fixed limits.  Applies
 * to later calls; batch cavities keep the default. */
int cfd_set_wait_limit(cfd_handle *h, uint64_t limit_ns);

/* Assembled-matrix path (Sec. 3.1: the paper assembles the pressure matrix
 * in CSR and multiplies with it), beside the matrix-free operator of
 * cfd_apply_poisson for comparison.  One caller-owned device buffer holds
 * row_ptr (int32, n + 1), col (int32, nnz, ascending per row) and val
 * (float64, nnz), each piece 16-byte aligned; nnz = 7 n - 2 (nx ny + ny nz
 * + nz nx).  cfd_csr_bytes sizes it (and returns nnz, nullable); the grid
 * must have 7 n < 2^31.  cfd_csr_assemble fills it (asynchronous);
 * cfd_csr_spmv computes y = A x, one row per thread in stored order
 * (asynchronous).  Errors through cfd_last_error(NULL). */
int cfd_csr_bytes(int32_t nx, int32_t ny, int32_t nz, size_t *bytes, int64_t *nnz);
int cfd_csr_assemble(int32_t nx, int32_t ny, int32_t nz, void *dev_buf, cfd_stream_t stream);
int cfd_csr_spmv(int32_t nx, int32_t ny, int32_t nz, const void *dev_buf, const double *x_dev, double *y_dev,
                 cfd_stream_t stream);

/* ------------------------------------------------------------------------
 * Stand-alone Krylov building blocks (Sec. 3.1, Table 1: spmv, the vector
 * add / scale operators and dot), for measurement one kernel at a time; the
 * solvers above fuse the same arithmetic into their persistent kernels.
 * All calls are asynchronous on `stream` and report argument errors through
 * the return code and cfd_last_error(NULL).
 * ------------------------------------------------------------------------ */

/* y = A x in FP32 for the Neumann pressure matrix of an nx x ny x nz grid
 * (x fastest; row c: n_c x_c minus the in-box neighbours, n_c their count),
 * the operator of the mixed-precision inner solve.  x, y: device, V floats,
 * must not overlap.  Errors: empty grid, NULL, ny > 524280 or nz > 131070. */
int cfd_apply_poisson_f32(int32_t nx, int32_t ny, int32_t nz, const float *x_dev, float *y_dev,
                          cfd_stream_t stream);

/* Bytes of the caller-owned device scratch of cfd_cg_update_*.  It must be
 * zero-filled once before its first use; every call leaves it zero-filled
 * again.  One scratch serves one call at a time (one stream). */
size_t cfd_cg_update_scratch_bytes(void);

/* The CG update of Algorithm-1 form (Sec. 3.1):  x += alpha p,
 * r -= alpha q, then *rr_dev = r.r of the updated r (summed in FP64 in an
 * order fixed by n alone, so repeated calls give identical bits).
 * p, q, x, r: device vectors of n elements, 16-byte aligned, x and r not
 * overlapping p, q or each other; rr_dev: one device double.
 * Errors: n = 0, NULL, misaligned pointers. */
int cfd_cg_update_f64(size_t n, double alpha, const double *p_dev, const double *q_dev, double *x_dev,
                      double *r_dev, double *rr_dev, void *scratch_dev, cfd_stream_t stream);
/* The same in FP32 (the vector arithmetic rounds to FP32; r.r accumulates in
 * FP64 from FP32 partial sums of four squares). */
int cfd_cg_update_f32(size_t n, float alpha, const float *p_dev, const float *q_dev, float *x_dev, float *r_dev,
                      double *rr_dev, void *scratch_dev, cfd_stream_t stream);

/* FP64 FMA throughput probe, the peak the FP64 kernels are measured
 * against (GB300's FP64 rate, not HBM, bounds the FP64 stencil): blocks x
 * 256 threads, each running 8 independent chains of `iters` fused
 * multiply-adds, 2 * 8 * iters * 256 * blocks flop in all.  out_dev: device
 * doubles, one per thread (blocks * 256).  Asynchronous on stream; the
 * caller times it (CUDA events). */
int cfd_probe_fp64_fma(int blocks, int iters, double *out_dev, cfd_stream_t stream);

/* ------------------------------------------------------------------------
 * Learned preconditioner (flexible PCG with a U-Net, Sec. 5 "other
 * preconditioners"; the paper itself uses DIC / Jacobi, Sec. 3.1).
 * ------------------------------------------------------------------------ */

/* One stride-1 3D convolution on the tensor cores (BF16 operands, FP32
 * accumulation), the U-Net's building block, exposed for direct checks.
 * Grid nx x ny x nz (x fastest, V cells), zero padding.  Activations are
 * BF16 "channel-octet planes": a tensor of C channels is ceil(C / W) planes
 * of [V][W], W = min(C, 8), so channel c of cell v is element
 * (c / W) V W + v W + c % W.  src0: c0 channels; src1: c1 channels
 * concatenated after src0 (c1 = 0: unused; c1 > 0 needs c0 % 16 == 0).  ks = 3 or 1.  weights: device BF16
 * [ks^3][nout_pad][cin_pad] (cin_pad = c0 + c1 rounded up to 16, tap index
 * kx + 3 ky + 9 kz, zero-filled padding), or for c0 = 1, c1 = 0, ks = 3 the
 * tap-packed [nout_pad][32] (taps 0..26, zeros after).  bias: device FP32
 * [cout] or NULL.  cout <= nout_pad in {16, 32, 64}.  Output: dst_bf16
 * (cout channels, octet planes), or dst_f32 [V][cout] FP32 when dst_f32
 * is non-NULL.  All pointers 16-byte aligned.
 * err_dev: device int set to 1 if a bounded device-side wait timed out.
 * Asynchronous on stream; returns a negative code on invalid arguments. */
int cfd_conv3d_bf16(int nx, int ny, int nz, const void *src0, int c0, const void *src1, int c1, int ks,
                    const void *weights, const float *bias, int cout, int nout_pad, void *dst_bf16,
                    float *dst_f32, int *err_dev, void *stream);

typedef struct cfd_unet cfd_unet;

/* Workspace of a U-Net preconditioner for an nx x ny x nz grid (each a
 * multiple of 4): parameters, Adam moments, BF16 activations and their
 * gradients, and the flexible-CG vectors (about 450 bytes per cell). */
int cfd_unet_workspace_bytes(int nx, int ny, int nz, size_t *bytes);

/* Create on a caller-owned device workspace (256-byte aligned, at least
 * cfd_unet_workspace_bytes); parameters are initialised from seed
 * (uniform +-sqrt(3 / fan_in), zero biases).  All work runs on stream. */
int cfd_unet_create(int nx, int ny, int nz, void *dev_ws, size_t bytes, cfd_stream_t stream, uint64_t seed,
                    cfd_unet **out);
void cfd_unet_destroy(cfd_unet *u);

/* Number of FP32 parameters (u may be NULL: the count is grid independent).
 * Layout: for each layer in order L0a, L0b, L1a, L1b, L2a, L2b, L1c, L0c,
 * head: weights [taps][cout][cin] (tap = kx + 3 ky + 9 kz), then bias
 * [cout]. */
int64_t cfd_unet_param_count(const cfd_unet *u);
/* The network's grid (as given to cfd_unet_create). */
int cfd_unet_grid(const cfd_unet *u, int *nx, int *ny, int *nz);
int cfd_unet_get_params(cfd_unet *u, float *host, int64_t n);
int cfd_unet_set_params(cfd_unet *u, const float *host, int64_t n);

/* z = M(r) = U(s r) / s - mean, s = sqrt(V) / ||r||: r_dev, z_dev device
 * float64 [V].  Asynchronous. */
int cfd_unet_apply(cfd_unet *u, const double *r_dev, double *z_dev);

/* One Adam step (lr, beta 0.9 / 0.999, eps 1e-8) on the mean over npairs
 * pairs of the loss (cfd_unet_set_loss; default |U(s r) - s e|^2 / V), with
 * s = sqrt(V) / ||r|| per pair; r_dev and e_dev device float64
 * [npairs][V].  *loss (nullable) receives the mean loss before the step.
 * Synchronises the stream. */
int cfd_unet_train_step(cfd_unet *u, const double *r_dev, const double *e_dev, int npairs, float lr, float *loss);

/* Training loss of cfd_unet_train_step (per pair, with d = U(s r) - s e):
 *   MSE    |d|^2 / V                 (the default)
 *   ANORM  d.(A d) / V, A the operator of cfd_apply_poisson (the error
 *          measured in the energy norm CG minimises)
 *   COS    1 - (z.A t) / sqrt((z.A z)(t.A t)), z = U(s r), t = s e: one
 *          minus the energy-norm cosine, invariant to a positive scale of
 *          z (as flexible CG is)                                         */
enum { CFD_UNET_LOSS_MSE = 0, CFD_UNET_LOSS_ANORM = 1, CFD_UNET_LOSS_COS = 2 };
int cfd_unet_set_loss(cfd_unet *u, int kind);

/* How the tiled 3x3x3 convolutions stage each 16-channel block (all modes
 * issue the same MMAs in the same order, so results are bitwise equal):
 *   REGISTERS  one stage; all threads copy the weights through registers
 *   BULK       one stage; one thread issues the TMA input copies and one bulk
 *              copy of the weights (kept in shared-memory order), then the
 *              MMAs (default)
 *   TWO_STAGE  as BULK with two stages: block cb + 1 is copied while the
 *              MMAs of block cb run (halves the tile and the occupancy)
 *   PERSISTENT one CTA per SM walks many tiles: one warp streams (tile,
 *              block) units into two stages, one issues the MMAs into two
 *              TMEM accumulators (tiles alternate), four store the finished
 *              tile, so copies, MMAs and stores overlap */
enum { CFD_UNET_CONV_REGISTERS = 0, CFD_UNET_CONV_BULK = 1, CFD_UNET_CONV_TWO_STAGE = 2, CFD_UNET_CONV_PERSISTENT = 3 };
int cfd_unet_set_conv_mode(cfd_unet *u, int mode);

/* Where the weight gradients of cfd_unet_train_step run:
 *   TENSOR      (default) the 3x3x3 layers L0b..L0c on the tensor cores (BF16
 *               operands, FP32 accumulation in tensor memory): per tap a
 *               contraction over the voxels, each CTA summing its boxes,
 *               then a fixed-order sum over the CTAs (bitwise repeatable);
 *               the first layer (one input channel) and the head (one output
 *               channel) on the CUDA cores;
 *   CUDA_CORES  every layer as FP32 sums on the CUDA cores (for comparison). */
enum { CFD_UNET_WGRAD_TENSOR = 0, CFD_UNET_WGRAD_CUDA_CORES = 1 };
int cfd_unet_set_wgrad_mode(cfd_unet *u, int mode);

/* Tensor read-back for checks (synchronous).  which in 0..25: the BF16
 * tensors (octet planes) xin, a0, s0, p0, a1, s1, p1, a2, s2, u1, d1, u0, d0
 * (activations of the last forward pass) and gz, g_d0, g_s0, g_u0, g_d1,
 * g_s1, g_u1, g_s2, g_a2, g_p1, g_a1, g_p0, g_a0 (their gradients from the
 * last backward pass); or one of the CFD_UNET_T_* below.  count must equal
 * the tensor's element count. */
enum {
  CFD_UNET_T_OUT = 100,     /* FP32 [V] head output of the last forward pass  */
  CFD_UNET_T_TARGET = 101,  /* FP32 [V] scaled target s e of the last pair     */
  CFD_UNET_T_GRAD = 102,    /* FP32 [params] accumulated gradient (last step)  */
  CFD_UNET_T_ADAM_M = 103,  /* FP32 [params] Adam first moment                 */
  CFD_UNET_T_ADAM_V = 104   /* FP32 [params] Adam second moment                */
};
int cfd_unet_read_tensor(cfd_unet *u, int which, void *host, int64_t count);

/* Flexible PCG on the Neumann pressure system of the U-Net's grid (the
 * operator of cfd_apply_poisson) with z = M(r) and the Polak-Ribiere beta
 * z_{k+1}.(r_{k+1} - r_k) / (z_k.r_k).  Cold start x = 0; the mean of b is
 * removed; no gauge shift.  Converged when the FP64 TRUE residual satisfies
 * ||b - A x|| <= rtol ||b||.  z.r < 0 is allowed (alpha = z.r / p.q is
 * then negative, still the exact line search along p).  On breakdown (p.q
 * <= 0, z.r = 0, a non-finite value) or stagnation (50 iterations without
 * the residual norm halving) it continues as plain CG from the current
 * iterate.  max_iters = 0 means
 * 20 * max(n).  stats (nullable): iters (all iterations), outer_iters (the
 * plain-CG ones), restarts, status, rel_resid, b_norm.  Synchronises the
 * stream; returns the status (CFD_OK, CFD_ERR_NOT_CONVERGED, ...). */
int cfd_unet_fpcg_solve(cfd_unet *u, const double *b_dev, double *x_dev, double rtol, int32_t max_iters,
                        cfd_solve_stats *stats);

/* Attach the U-Net u (same grid as h; NULL detaches) to a cavity created
 * with solver CFD_SOLVER_FPCG (the network preconditions flexible CG) or
 * with solver CFD_SOLVER_IR and learned_guess = 1 (the network gives the
 * initial guess).  Its pressure solves (cfd_step, cfd_substep,
 * cfd_solve_pressure) then use it with the handle's rtol and iteration
 * cap; the step's gauge follows.  In the graph forms the network's forward
 * pass is captured into the solve's graph and runs on the handle's stream,
 * reading the network's workspace (input, activations, output): do not use
 * the network on another stream while such a solve may run.  Changing the
 * network's parameters between solves is fine (the graph reads them from
 * its workspace); its convolution mode is captured, and a change rebuilds
 * the graph.  The HOST form of FPCG synchronises the handle's stream
 * before each solve (the network runs on its own stream).  u must outlive
 * its attachment; a pressure solve that needs a network without one
 * attached returns CFD_ERR_INVALID_ARG. */
int cfd_attach_preconditioner(cfd_handle *h, cfd_unet *u);

/* The learned initial guess alone: x = alpha (z - mean z) with z = U(s b'),
 * b' = b - mean(b), s = sqrt(V) / |b'| (the network of cfd_unet_apply on
 * the attached U-Net) and alpha = z~.b' / z~.A z~ (z~ = z - mean z): the
 * multiple of the network's answer closest to A^+ b' in the energy norm
 * (alpha = 0 when the network returns a constant or its wait timed out).
 * b_dev, x_dev: distinct device arrays of nx*ny*nz float64.  Needs a handle
 * with solver IR or FPCG, nx % 4 == 0 and a network attached.
 * Asynchronous on the handle's stream; uses the network's workspace. */
int cfd_learned_guess(cfd_handle *h, const double *b_dev, double *x_dev);

int64_t cfd_unet_launch_count(const cfd_unet *u);
const char *cfd_unet_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CFD_GB300_H */
