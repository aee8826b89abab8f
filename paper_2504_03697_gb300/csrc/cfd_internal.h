// Host-side interface between the C-ABI layer and the kernel translation
// units.  Not part of the public ABI (include/cfd.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "cfd_common.cuh"

struct cfd_unet;  // the learned preconditioner (include/cfd.h)

namespace cfd {

// Operator kinds of the stencil solves.
enum OpKind : int {
  kOpPressure = 0,  // Neumann 7-point, A = -h^2 Laplacian (scaled), singular
  kOpVelU = 1,      // I + c L for the u faces (x walls are known rows)
  kOpVelV = 2,      // ... v faces
  kOpVelW = 3       // ... w faces
};

struct GridDims {
  int mx, my, mz;
  size_t count() const { return size_t(mx) * my * mz; }
};

// Geometry of one persistent solve launch.
struct LaunchGeom {
  int blocks;       // maximum co-resident blocks of the cooperative launch
  int tz;           // unused (kept for layout compatibility)
  int num_sms;
  int bps_req;      // requested blocks per SM (0: automatic)
  int tz_req;       // requested tile depth (0: automatic)
  int no_tma;       // 1: never take the TMA stencil path
  int cg_variant;   // CgArgs::variant for the handle's FP64 solves
  int shared;       // 1: other cooperative grids run at the same time (blocks is this grid's share)
};

// Launch shape picked for one solve.
struct SolveShape {
  int blocks;       // grid size
  int tz;           // tile depth (cells per thread along z)
  int rtz;          // > 0: register path with this depth; 0: memory path
};

SolveShape pick_solve_shape(GridDims g, int max_blocks, int bps_req, int tz_req);

// Arguments of the persistent FP64 CG solve.
struct CgArgs {
  GridDims g;
  int kind;              // OpKind
  int precond;           // 0 none, 1 Jacobi (pressure only)
  double c;              // Helmholtz coefficient nu*dt/h^2 (velocity kinds)
  double* x;             // solution, in/out
  double* b;             // right-hand side, modified in place (mean removal)
  double* r;
  double* d0;
  double* d1;
  double* q;
  double* e0;            // extra vectors of the single-reduction variant
  double* e1;            // (all three non-null to allow it)
  double* e2;
  int variant;           // 0: single-reduction CG when allowed, 1: two all-reduces per iteration
  int zero_x0;           // 1: x0 = 0
  int remove_mean;       // 1: b -= mean(b) first
  int gauge;             // 1: after the solve, x += gauge_value - mean(x)
  double gauge_value;
  double rtol;
  int max_iters;
  int max_restarts;
  unsigned long long timeout_ns;
  SolveCtrl* ctrl;       // zeroed by the host before the launch
  double* partials;      // 2 * blocks * kMaxPartials doubles (double-buffered)
  DevSolveStats* stats;  // written by block 0 at exit
  int tz;
};

// Arguments of the FP32-inner / FP64-outer iterative-refinement solve.
struct IrArgs {
  GridDims g;
  int kind;        // kOp* operator (the TMA stencil ring serves kOpPressure only)
  double c;        // nu dt / h^2 of the velocity operators
  double* x;       // FP64 solution (out)
  double* b;       // FP64 rhs (mean removed in place)
  double* r;       // FP64 outer residual
  float* r32;      // FP32 inner vectors
  float* d32;      // inner solution increment
  float* p0_32;
  float* p1_32;
  float* q32;
  int zero_x0;
  int remove_mean;
  int gauge;
  double gauge_value;
  double rtol;
  double delta;     // refine when the FP32 residual fell by this factor
  int max_iters;   // cap on the FP32 CG iterations
  int max_outer;   // cap on the FP64 refinements
  unsigned long long timeout_ns;
  SolveCtrl* ctrl;
  double* partials;
  DevSolveStats* stats;
  int tz;
  // TMA path of the FP32 stencil phase (use_tma != 0): 3D tensor maps over
  // r32, p0_32, p1_32 with a (kTmaBoxW x kTmaBoxH x 1) box, z-chunk depth.
  int use_tma;
  int tma_zl;
  // graph form only (ir_graph.cu): the learned preconditioner.  With net
  // set, flexible = 1 runs flexible CG with z = M(r32) from the network in
  // every FP32 iteration (falling back to plain CG after `stagnation`
  // iterations without halving the residual norm, or on a breakdown), and
  // guess = 1 starts from x0 = alpha M(b) (alpha the energy line search).
  cfd_unet* net;
  int net_mode;     // the network's convolution mode when the graph was built
  int flexible;
  int guess;
  int guess_warm;   // guess: correct the starting x (warm start) instead of replacing it
  int stagnation;
  CUtensorMap map_r32;
  CUtensorMap map_p0;
  CUtensorMap map_p1;
};

// TMA slab box of the FP32 stencil: a 32 x 8 tile plus a 4-float-aligned x
// halo (x from x0-4, 40 floats = 160 B) and a one-row y halo.
constexpr int kTmaBoxW = 40;
constexpr int kTmaBoxH = 10;

// Encode a 3D FP32 tensor map (mx, my, mz; x fastest) for the FP32 stencil
// box.  Returns false when the grid does not meet TMA's stride rules (mx a
// multiple of 4) or the driver entry point is unavailable.
bool encode_f32_grid_map(CUtensorMap* map, const float* base, int mx, int my, int mz);

struct PhysArgs {
  int nx, ny, nz;
  double h, inv_h, dt, rho, nu, lid_u;
  double g[3];
  double* u; double* v; double* w;       // current velocity
  double* ua; double* va; double* wa;    // intermediate velocity
  double* p;                             // pressure (cells)
  double* b;                             // solver rhs scratch
  int rk2;                               // 1: explicit-midpoint backtrace
};

// Kernel launchers (return the CUDA error of the launch).  Each adds the
// number of kernels it launched to *launches.
cudaError_t launch_cg(const CgArgs& a, const LaunchGeom& lg, cudaStream_t s, int64_t* launches);
// Grid of the tile-resident single-reduction FP64 CG for this grid and
// launch geometry (one block per tile), 0 when the automatic shape does not
// take it; it runs for unpreconditioned single-reduction CG solves.
int cgt_blocks_for(GridDims g, const LaunchGeom& lg);
constexpr int kCgtTileDepth = 8;  // its tile depth along z
cudaError_t launch_ir(const IrArgs& a, const LaunchGeom& lg, cudaStream_t s, int64_t* launches);
cudaError_t launch_apply_poisson(GridDims g, const double* x, double* y, int tz, cudaStream_t s,
                                 int64_t* launches);
cudaError_t launch_forces(const PhysArgs& a, cudaStream_t s, int64_t* launches);
cudaError_t launch_advect(const PhysArgs& a, cudaStream_t s, int64_t* launches);
cudaError_t launch_diffusion_rhs(const PhysArgs& a, int comp, cudaStream_t s, int64_t* launches);
cudaError_t launch_divergence(const PhysArgs& a, cudaStream_t s, int64_t* launches);
cudaError_t launch_correct(const PhysArgs& a, cudaStream_t s, int64_t* launches);
cudaError_t launch_zero_wall_faces(const PhysArgs& a, cudaStream_t s, int64_t* launches);
// Batched sweeps (one launch for many cavities): cavity k of the device
// table d_tab works on the blocks [d_starts[k], d_starts[k+1]); its block
// count is sweep_blocks_for(its args, op, comp), the single-cavity grid.
enum SweepOp { kSweepAdvect = 0, kSweepForces = 1, kSweepDiffusionRhs = 2, kSweepDivergence = 3, kSweepCorrect = 4 };
size_t sweep_elems(const PhysArgs& a, int op, int comp);
int sweep_blocks_for(const PhysArgs& a, int op, int comp);
cudaError_t launch_sweep_multi(int op, const PhysArgs* d_tab, const int* d_starts, int nprob, int total_blocks,
                               int comp, cudaStream_t s, int64_t* launches);
cudaError_t launch_fill(double* p, size_t n, double value, cudaStream_t s, int64_t* launches);
// Training pair of the learned preconditioner: r = (b - mean b) - A xk and
// e = (xs - xk) - mean(xs - xk), with the FP64 pressure operator A.  r must
// not overlap xk.  scratch: harvest_scratch_doubles() device doubles.
cudaError_t launch_harvest_pair(GridDims g, const double* b, const double* xs, const double* xk, double* r, double* e,
                                double* scratch, cudaStream_t s, int64_t* launches);
size_t harvest_scratch_doubles();

// Co-resident block count for the persistent solve kernels on this device.
int cg_max_coresident_blocks(int kind_is_ir);

// Multi-problem persistent solves: problem p owns blocks d_starts[p] ..
// d_starts[p+1] of a cooperative grid of total_blocks = d_starts[nprob]
// blocks; problems never synchronise with each other.  Tables live in device
// memory.  Memory path only (per-problem runtime tile depth), no TMA.
cudaError_t launch_cg_multi(const CgArgs* d_table, const int* d_starts, int nprob, int total_blocks, int precond,
                            cudaStream_t s, int64_t* launches);
int batch_blocks_per_sm();
int batch_num_sms();
// Deepest tile depth that still gives `blocks` blocks two tiles each.
int solve_tile_depth_for(GridDims g, int blocks);

// Stencil tile depth (cells per thread along z) used for a grid of mz planes.
int solve_tile_depth(int mz);

// Record a printf-style message as cfd_last_error(NULL) and return code.
int cfd_internal_error(int code, const char* fmt, ...);

constexpr int kTileX = 32;
constexpr int kTileY = 8;
constexpr int kSolveThreads = kTileX * kTileY;

}  // namespace cfd
