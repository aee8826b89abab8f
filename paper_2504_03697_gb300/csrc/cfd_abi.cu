// C-ABI of the cavity projection path: handle, workspace layout, step
// driver.  Declared in include/cfd.h; the functions below follow the
// paper's statement of the problem (Sec. 3 / 3.1 of arXiv 2504.03697):
// parameters and initial state (v0 = 0, p0 = 1), the fractional step
// (forces, advection, pressure correction), and reading the fields.
//
// The library never allocates device memory: every array lives in the
// caller's workspace, carved up by ws_layout below (256-byte aligned).

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <queue>
#include <vector>

#include "../../include/cfd.h"
#include "cfd_internal.h"
#include "dic.h"
#include "ir_graph.h"
#include "unet.h"

using namespace cfd;

namespace {

constexpr int kStatsCap = 1024;   // per-step statistics slots in the workspace
constexpr int kMaxRestarts = 8;
constexpr unsigned long long kTimeoutNs = 2000000000ull;  // 2 s per device wait

thread_local char g_last_error[256] = "no error";

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t u, v, w, ua, va, wa, p;
  size_t b, r, d0, d1, q;
  size_t e0, e1, e2;
  size_t dicd;
  size_t r32, d32, p0_32, p1_32, q32;
  size_t irg;  // state of the graph-driven mixed-precision solve
  size_t partials, ctrl, stats;
  // concurrent diffusion solves (small grids): solver vectors b, r, d0, d1,
  // q, e0, e1, e2, partial sums and a control block for the v and w solves
  size_t cset[2][8], cpartials[2], cctrl[2];
  bool conc;
  size_t total;
};

size_t face_count(const cfd_params& p, int comp) {
  return size_t(p.nx + (comp == 0)) * size_t(p.ny + (comp == 1)) * size_t(p.nz + (comp == 2));
}

// Grids up to this many cells get workspace for running the three diffusion
// solves of a step concurrently (they are latency-bound there).
constexpr size_t kConcDiffusionCells = size_t(1) << 21;

Layout ws_layout(const cfd_params& p, int max_blocks, bool standalone = true) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t cells = size_t(p.nx) * p.ny * p.nz;
  size_t vec = cells;
  for (int c = 0; c < 3; ++c) vec = vec > face_count(p, c) ? vec : face_count(p, c);
  L.u = take(face_count(p, 0) * 8);
  L.v = take(face_count(p, 1) * 8);
  L.w = take(face_count(p, 2) * 8);
  L.ua = take(face_count(p, 0) * 8);
  L.va = take(face_count(p, 1) * 8);
  L.wa = take(face_count(p, 2) * 8);
  L.p = take(cells * 8);
  L.b = take(vec * 8);
  L.r = take(vec * 8);
  L.d0 = take(vec * 8);
  L.d1 = take(vec * 8);
  L.q = take(vec * 8);
  // extra vectors of the single-reduction CG (double-buffered r and s, p)
  L.e0 = take(vec * 8);
  L.e1 = take(vec * 8);
  L.e2 = take(vec * 8);
  if (p.solver == CFD_SOLVER_DIC) L.dicd = take(cells * 8);  // reciprocal DIC pivots of the pressure matrix
  if (p.solver == CFD_SOLVER_IR || p.solver == CFD_SOLVER_FPCG) {
    // sized to the largest face grid: the graph form also runs the
    // diffusion solves in FP32 with FP64 refinement (and the flexible CG
    // with the learned preconditioner uses the same FP32 vectors)
    const size_t vec32 = std::max(vec, ir_fp32_vector_cells(p.nx, p.ny, p.nz));
    L.r32 = take(vec32 * 4);
    L.d32 = take(vec32 * 4);
    L.p0_32 = take(vec32 * 4);
    L.p1_32 = take(vec32 * 4);
    L.q32 = take(vec32 * 4);
    L.irg = take(ir_graph_state_bytes());
  }
  L.partials = take(partials_doubles(max_blocks) * 8);  // double-buffered block + group partials
  L.ctrl = take(sizeof(SolveCtrl));
  L.stats = take(size_t(kStatsCap + 1) * sizeof(DevStepStats));  // ring + one slot for substep/solve calls
  // batch members run their diffusion solves in the batch's multi-problem launch
  L.conc = standalone && p.nu > 0.0 && cells <= kConcDiffusionCells;
  if (L.conc)
    for (int c = 0; c < 2; ++c) {
      for (int v = 0; v < 8; ++v) L.cset[c][v] = take(vec * 8);
      L.cpartials[c] = take(partials_doubles(max_blocks) * 8);
      L.cctrl[c] = take(sizeof(SolveCtrl));
    }
  L.total = off;
  return L;
}

// Upper bound on the co-resident block count used for sizing partials; the
// real count is capped by the device at create time.
constexpr int kMaxBlocksBound = 4096;

}  // namespace

struct cfd_handle {
  cfd_params prm;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  Layout L;
  double *u, *v, *w, *ua, *va, *wa, *p;
  double *b, *r, *d0, *d1, *q;
  double *e0, *e1, *e2;
  double* dicd = nullptr;
  bool dic_ready = false;
  cfd_unet* precond_net = nullptr;  // CFD_SOLVER_FPCG
  float *r32, *d32, *p0_32, *p1_32, *q32;
  void* irg_state = nullptr;     // graph solve state (CFD_SOLVER_IR)
  cfd::IrGraph* irg = nullptr;   // its cached, instantiated graph (pressure)
  cfd::IrGraph* irg_diff[3] = {nullptr, nullptr, nullptr};  // diffusion of u, v, w
  int ir_form = CFD_IR_AUTO;
  int fpcg_form = CFD_FPCG_GRAPH;
  unsigned long long wait_ns = kTimeoutNs;  // limit of each grid-wide wait (cfd_set_wait_limit)
  double* partials;
  SolveCtrl* ctrl;
  DevStepStats* stats;
  // concurrent diffusion solves of v and w (workspace slots, two streams)
  double* cset[2][8] = {};
  double* cpartials[2] = {nullptr, nullptr};
  SolveCtrl* cctrl[2] = {nullptr, nullptr};
  cudaStream_t aux[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  bool conc_diffusion = false;   // enabled (cfd_set_concurrent_diffusion)
  LaunchGeom lg;
  int64_t launches;
  char err[256];
  // phase timers (host-side CUDA events)
  bool timing;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_next;
  struct Pending { int phase; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  int64_t ring;  // steps taken so far (statistics ring position)
  // host snapshot of u, v, w, p for CSV output (pinned host memory)
  double* snap = nullptr;
  cudaEvent_t snap_ev = nullptr;
  bool snap_pending = false;
};

namespace {

int set_err(cfd_handle* h, int code, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) std::memcpy(h->err, buf, sizeof(buf));
  std::memcpy(g_last_error, buf, sizeof(buf));
  return code;
}

int cuda_check(cfd_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CFD_OK;
  return set_err(h, CFD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Event pair around one phase when timing is on (begin returns the pair index).
int phase_begin(cfd_handle* h, int phase) {
  if (!h->timing) return -1;
  if (h->ev_next + 2 > h->ev_pool.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      h->ev_pool.push_back(e);
    }
  }
  cudaEvent_t a = h->ev_pool[h->ev_next], b = h->ev_pool[h->ev_next + 1];
  h->ev_next += 2;
  cudaEventRecord(a, h->stream);
  h->pending.push_back({phase, a, b});
  return int(h->pending.size()) - 1;
}

void phase_end(cfd_handle* h, int slot) {
  if (slot < 0) return;
  cudaEventRecord(h->pending[size_t(slot)].b, h->stream);
}

int validate(const cfd_params* p) {
  if (!p) return set_err(nullptr, CFD_ERR_INVALID_ARG, "params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return set_err(nullptr, CFD_ERR_INVALID_ARG, "grid sizes must be >= 1");
  if (double(p->nx + 1) * p->ny * p->nz > 2.0e9 || double(p->nx) * (p->ny + 1) * p->nz > 2.0e9 ||
      double(p->nx) * p->ny * (p->nz + 1) > 2.0e9)
    return set_err(nullptr, CFD_ERR_INVALID_ARG, "grid too large");
  if (!(p->length > 0) || !(p->dt > 0) || !(p->rho > 0) || !(p->nu >= 0))
    return set_err(nullptr, CFD_ERR_INVALID_ARG, "length, dt, rho must be > 0 and nu >= 0");
  if (!std::isfinite(p->lid_u) || !std::isfinite(p->g[0]) || !std::isfinite(p->g[1]) || !std::isfinite(p->g[2]))
    return set_err(nullptr, CFD_ERR_INVALID_ARG, "lid_u and g must be finite");
  if (p->solver < CFD_SOLVER_CG || p->solver > CFD_SOLVER_FPCG)
    return set_err(nullptr, CFD_ERR_INVALID_ARG, "unknown solver %d", p->solver);
  if (!(p->rtol > 0) || p->rtol >= 1) return set_err(nullptr, CFD_ERR_INVALID_ARG, "rtol must be in (0, 1)");
  if (p->max_iters < 0) return set_err(nullptr, CFD_ERR_INVALID_ARG, "max_iters must be >= 0");
  if (p->ir_delta < 0 || p->ir_delta >= 1) return set_err(nullptr, CFD_ERR_INVALID_ARG, "ir_delta must be in [0, 1)");
  if (p->advect_order < 0 || p->advect_order > 2) return set_err(nullptr, CFD_ERR_INVALID_ARG, "advect_order in {0, 1, 2}");
  if (p->learned_guess != 0 && p->learned_guess != 1)
    return set_err(nullptr, CFD_ERR_INVALID_ARG, "learned_guess must be 0 or 1");
  if (p->learned_guess && p->solver != CFD_SOLVER_IR)
    return set_err(nullptr, CFD_ERR_INVALID_ARG, "learned_guess needs the IR solver");
  if (p->learned_guess && p->nx % 4 != 0)
    return set_err(nullptr, CFD_ERR_INVALID_ARG, "learned_guess needs nx %% 4 == 0 (graph form)");
  for (int i = 0; i < 6; ++i)
    if (p->reserved[i] != 0) return set_err(nullptr, CFD_ERR_INVALID_ARG, "reserved fields must be zero");
  return CFD_OK;
}

int iter_cap(const cfd_params& p) {
  if (p.max_iters > 0) return p.max_iters;
  int m = p.nx > p.ny ? p.nx : p.ny;
  m = m > p.nz ? m : p.nz;
  return 20 * m;
}

PhysArgs phys(const cfd_handle* h) {
  PhysArgs a{};
  a.nx = h->prm.nx; a.ny = h->prm.ny; a.nz = h->prm.nz;
  a.h = h->prm.length / h->prm.nx;
  a.inv_h = 1.0 / a.h;
  a.dt = h->prm.dt; a.rho = h->prm.rho; a.nu = h->prm.nu; a.lid_u = h->prm.lid_u;
  a.g[0] = h->prm.g[0]; a.g[1] = h->prm.g[1]; a.g[2] = h->prm.g[2];
  a.u = h->u; a.v = h->v; a.w = h->w; a.ua = h->ua; a.va = h->va; a.wa = h->wa;
  a.p = h->p; a.b = h->b;
  a.rk2 = h->prm.advect_order == 2 ? 1 : 0;
  return a;
}

int tz_for(int mz) {
  // cells per thread along z in the stencil tiles: 0 lets the solver pick
  // the deepest tile that still spreads over every SM
  (void)mz;
  return 0;
}

// The FP64 solver vectors (and partial-sum scratch) one CG solve works on.
struct SolveVectors {
  double *b, *r, *d0, *d1, *q, *e0, *e1, *e2, *partials;
};

SolveVectors main_vectors(const cfd_handle* h) {
  return SolveVectors{h->b, h->r, h->d0, h->d1, h->q, h->e0, h->e1, h->e2, h->partials};
}

// The extra set k (0: v, 1: w) of the concurrent diffusion solves.
SolveVectors extra_vectors(const cfd_handle* h, int k) {
  double* const* v = h->cset[k];
  return SolveVectors{v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], h->cpartials[k]};
}

CgArgs diffusion_args(const cfd_handle* h, int comp, DevSolveStats* st, SolveCtrl* ctrl, const SolveVectors& vs);

// Arguments of the backward-Euler diffusion solve of component comp on the
// intermediate velocity (x0 = the advected field, b from diffusion_rhs).
CgArgs diffusion_args(const cfd_handle* h, int comp, DevSolveStats* st, SolveCtrl* ctrl) {
  return diffusion_args(h, comp, st, ctrl, main_vectors(h));
}

CgArgs diffusion_args(const cfd_handle* h, int comp, DevSolveStats* st, SolveCtrl* ctrl, const SolveVectors& vs) {
  const double hh = h->prm.length / h->prm.nx;
  CgArgs a{};
  a.g = GridDims{h->prm.nx + (comp == 0), h->prm.ny + (comp == 1), h->prm.nz + (comp == 2)};
  a.kind = kOpVelU + comp;
  a.precond = 0;
  a.c = h->prm.nu * h->prm.dt / (hh * hh);
  a.x = comp == 0 ? h->ua : (comp == 1 ? h->va : h->wa);
  a.b = vs.b; a.r = vs.r; a.d0 = vs.d0; a.d1 = vs.d1; a.q = vs.q;
  a.e0 = vs.e0; a.e1 = vs.e1; a.e2 = vs.e2;
  a.variant = h->lg.cg_variant;
  a.zero_x0 = 0; a.remove_mean = 0; a.gauge = 0; a.gauge_value = 0.0;
  a.rtol = h->prm.rtol;
  a.max_iters = iter_cap(h->prm);
  a.max_restarts = kMaxRestarts;
  a.timeout_ns = h->wait_ns;
  a.ctrl = ctrl; a.partials = vs.partials; a.stats = st;
  a.tz = tz_for(a.g.mz);
  return a;
}

// Arguments of the FP64 pressure CG (or Jacobi PCG) on the workspace b.
CgArgs pressure_cg_args(const cfd_handle* h, double* x, int zero_x0, int gauge, DevSolveStats* st, SolveCtrl* ctrl) {
  CgArgs a{};
  a.g = GridDims{h->prm.nx, h->prm.ny, h->prm.nz};
  a.kind = kOpPressure;
  a.precond = h->prm.solver == CFD_SOLVER_JACOBI ? 1 : 0;
  a.c = 0.0;
  a.x = x; a.b = h->b; a.r = h->r; a.d0 = h->d0; a.d1 = h->d1; a.q = h->q;
  a.e0 = h->e0; a.e1 = h->e1; a.e2 = h->e2;
  a.variant = h->lg.cg_variant;
  a.zero_x0 = zero_x0; a.remove_mean = 1; a.gauge = gauge; a.gauge_value = 1.0;
  a.rtol = h->prm.rtol;
  a.max_iters = iter_cap(h->prm);
  a.max_restarts = kMaxRestarts;
  a.timeout_ns = h->wait_ns;
  a.ctrl = ctrl; a.partials = h->partials; a.stats = st;
  a.tz = tz_for(a.g.mz);
  return a;
}

// Arguments of the FP32-CG / FP64-refinement pressure solve.
IrArgs pressure_ir_args(const cfd_handle* h, double* x, int zero_x0, int gauge, DevSolveStats* st, SolveCtrl* ctrl) {
  IrArgs a{};
  a.g = GridDims{h->prm.nx, h->prm.ny, h->prm.nz};
  a.x = x; a.b = h->b; a.r = h->r;
  a.r32 = h->r32; a.d32 = h->d32; a.p0_32 = h->p0_32; a.p1_32 = h->p1_32; a.q32 = h->q32;
  a.zero_x0 = zero_x0; a.remove_mean = 1; a.gauge = gauge; a.gauge_value = 1.0;
  a.rtol = h->prm.rtol;
  // two decades per FP32 recurrence: at 256^3 and 384^3 the same FP32
  // iterations as with 0.1 and 4 refinements instead of 7; 1e-3 adds 3-17 %
  // iterations, 1e-4 stagnates
  a.delta = h->prm.ir_delta > 0 ? h->prm.ir_delta : 0.01;
  a.max_iters = iter_cap(h->prm);
  a.max_outer = 1000;
  a.timeout_ns = h->wait_ns;
  a.ctrl = ctrl; a.partials = h->partials; a.stats = st;
  a.tz = tz_for(a.g.mz);
  return a;
}

// Graph form of the mixed-precision solve wherever it applies (the pressure
// matrix needs nx % 4 == 0), unless the persistent form is requested: a
// cavity step at 64^3 / 128^3 / 192^3 takes 6.0 / 17.7 / 56.4 ms with it
// against 11.0 / 26.9 / 91.1 ms with the persistent kernel.
bool use_ir_graph(const cfd_handle* h, const IrArgs& a) {
  return h->irg_state && ir_graph_eligible(a) && h->ir_form != CFD_IR_PERSISTENT;
}

// The diffusion solve of component comp as FP32 CG with FP64 refinement
// (CFD_SOLVER_IR, any form): x0 = the advected field, b from diffusion_rhs,
// the velocity matrix I + c L; no mean removal or gauge.  The persistent and
// batch launches add their control block and partial sums.
IrArgs diffusion_ir_args(const cfd_handle* h, int comp, DevSolveStats* st) {
  const double hh = h->prm.length / h->prm.nx;
  IrArgs a{};
  a.g = GridDims{h->prm.nx + (comp == 0), h->prm.ny + (comp == 1), h->prm.nz + (comp == 2)};
  a.kind = kOpVelU + comp;
  a.c = h->prm.nu * h->prm.dt / (hh * hh);
  a.x = comp == 0 ? h->ua : (comp == 1 ? h->va : h->wa);
  a.b = h->b; a.r = h->r;
  a.r32 = h->r32; a.d32 = h->d32; a.p0_32 = h->p0_32; a.p1_32 = h->p1_32; a.q32 = h->q32;
  a.zero_x0 = 0; a.remove_mean = 0; a.gauge = 0; a.gauge_value = 0.0;
  a.rtol = h->prm.rtol;
  // I + c L is well conditioned (eigenvalues in [1, 1 + 12 c]): the FP32
  // recurrence may run four decades between refinements
  a.delta = h->prm.ir_delta > 0 ? h->prm.ir_delta : 1e-4;
  a.max_iters = iter_cap(h->prm);
  a.max_outer = 1000;
  a.timeout_ns = h->wait_ns;
  a.stats = st;
  return a;
}

// The diffusion solves run in mixed precision (FP32 CG with FP64
// refinement) for the IR solver and the graph form of FPCG.
bool ir_diffusion(const cfd_handle* h) {
  return h->prm.solver == CFD_SOLVER_IR || (h->prm.solver == CFD_SOLVER_FPCG && h->fpcg_form == CFD_FPCG_GRAPH);
}

// Velocity diffusion solve for component comp (x = intermediate velocity).
int run_diffusion(cfd_handle* h, int comp, DevSolveStats* st) {
  PhysArgs pa = phys(h);
  int rc = cuda_check(h, launch_diffusion_rhs(pa, comp, h->stream, &h->launches), "diffusion rhs");
  if (rc) return rc;
  if (ir_diffusion(h)) {
    IrArgs ia = diffusion_ir_args(h, comp, st);
    if (use_ir_graph(h, ia))
      return cuda_check(h, launch_ir_graph(ia, h->irg_state, &h->irg_diff[comp], h->stream), "IR diffusion graph");
    ia.ctrl = h->ctrl;
    ia.partials = h->partials;
    rc = cuda_check(h, cudaMemsetAsync(h->ctrl, 0, sizeof(SolveCtrl), h->stream), "memset ctrl");
    if (rc) return rc;
    return cuda_check(h, launch_ir(ia, h->lg, h->stream, &h->launches), "IR diffusion launch");
  }
  const CgArgs a = diffusion_args(h, comp, st, h->ctrl);
  rc = cuda_check(h, cudaMemsetAsync(h->ctrl, 0, sizeof(SolveCtrl), h->stream), "memset ctrl");
  if (rc) return rc;
  return cuda_check(h, launch_cg(a, h->lg, h->stream, &h->launches), "diffusion CG launch");
}

// The three diffusion solves of a step at once: u on the handle's stream,
// v and w on two auxiliary streams forked from and joined back to it, each
// with its own solver vectors, partial sums and control block, each grid a
// third of the co-resident blocks (so that the three cooperative grids fit
// together).  The solves are independent (component c reads and writes only
// its own intermediate field).
int run_diffusion_concurrent(cfd_handle* h, DevStepStats* st) {
  int rc = cuda_check(h, cudaEventRecord(h->ev_fork, h->stream), "fork event");
  for (int k = 0; k < 2 && !rc; ++k) rc = cuda_check(h, cudaStreamWaitEvent(h->aux[k], h->ev_fork, 0), "fork wait");
  LaunchGeom lg = h->lg;
  lg.blocks = std::max(1, h->lg.blocks / 3);
  lg.shared = 1;
  lg.bps_req = 0;  // a tuned shape is for the whole device
  lg.tz_req = 0;
  for (int c = 0; c < 3 && !rc; ++c) {
    cudaStream_t s = c == 0 ? h->stream : h->aux[c - 1];
    const SolveVectors vs = c == 0 ? main_vectors(h) : extra_vectors(h, c - 1);
    SolveCtrl* ctrl = c == 0 ? h->ctrl : h->cctrl[c - 1];
    PhysArgs pa = phys(h);
    pa.b = vs.b;
    rc = cuda_check(h, launch_diffusion_rhs(pa, c, s, &h->launches), "diffusion rhs");
    if (!rc) rc = cuda_check(h, cudaMemsetAsync(ctrl, 0, sizeof(SolveCtrl), s), "memset ctrl");
    if (!rc) rc = cuda_check(h, launch_cg(diffusion_args(h, c, &st->d[c], ctrl, vs), lg, s, &h->launches), "diffusion CG");
  }
  // join even after a failure, so that nothing launched runs past the step
  for (int k = 0; k < 2; ++k) {
    const int r1 = cuda_check(h, cudaEventRecord(h->ev_join[k], h->aux[k]), "join event");
    const int r2 = cuda_check(h, cudaStreamWaitEvent(h->stream, h->ev_join[k], 0), "join wait");
    if (!rc) rc = r1 ? r1 : r2;
  }
  return rc;
}

bool diffusion_concurrent(const cfd_handle* h) {
  // the mixed-precision solves share one set of FP32 vectors
  return h->conc_diffusion && h->aux[0] && h->cset[0][0] && !ir_diffusion(h);
}

// Pressure solve A x = b on the handle's workspace b (already filled).
int run_pressure(cfd_handle* h, double* x, int zero_x0, int gauge, DevSolveStats* st) {
  int rc = cuda_check(h, cudaMemsetAsync(h->ctrl, 0, sizeof(SolveCtrl), h->stream), "memset ctrl");
  if (rc) return rc;
  if (h->prm.solver == CFD_SOLVER_FPCG && h->fpcg_form == CFD_FPCG_GRAPH) {
    // flexible CG with FP32 vectors and FP64 refinement, one graph per solve
    if (!h->precond_net) return set_err(h, CFD_ERR_INVALID_ARG, "FPCG solver without an attached preconditioner");
    IrArgs a = pressure_ir_args(h, x, zero_x0, gauge, st, h->ctrl);
    UNetView nv{};
    unet_view(h->precond_net, &nv);
    a.net = h->precond_net;
    a.net_mode = nv.conv_mode;
    a.flexible = 1;
    a.stagnation = 50;
    if (!ir_graph_eligible(a)) return set_err(h, CFD_ERR_INVALID_ARG, "the FPCG graph form needs nx %% 4 == 0");
    const int t = phase_begin(h, CFD_PHASE_PCG);
    rc = cuda_check(h, launch_ir_graph(a, h->irg_state, &h->irg, h->stream), "FPCG graph launch");
    phase_end(h, t);
    return rc;
  }
  if (h->prm.solver == CFD_SOLVER_FPCG) {
    if (!h->precond_net) return set_err(h, CFD_ERR_INVALID_ARG, "FPCG solver without an attached preconditioner");
    rc = cuda_check(h, cudaStreamSynchronize(h->stream), "synchronize");
    if (rc) return rc;
    // FPCG is cold-started; warm_start does not apply
    (void)zero_x0;
    cfd_solve_stats cs{};
    const int t = phase_begin(h, CFD_PHASE_PCG);
    const int frc = cfd_unet_fpcg_solve(h->precond_net, h->b, x, h->prm.rtol, iter_cap(h->prm), &cs);
    phase_end(h, t);
    if (frc != CFD_OK && frc != CFD_ERR_NOT_CONVERGED && frc != CFD_ERR_BREAKDOWN && frc != CFD_ERR_TIMEOUT)
      return set_err(h, frc, "FPCG: %s", cfd_unet_last_error());
    if (gauge) {
      rc = cuda_check(h, launch_gauge(GridDims{h->prm.nx, h->prm.ny, h->prm.nz}, x, 1.0, h->partials, h->stream,
                                      &h->launches), "gauge");
      if (rc) return rc;
    }
    DevSolveStats ds{};
    ds.iters = cs.iters;
    ds.outer_iters = cs.outer_iters;
    ds.restarts = cs.restarts;
    ds.status = cs.status;
    ds.rel_resid = cs.rel_resid;
    ds.b_norm = cs.b_norm;
    rc = cuda_check(h, cudaMemcpyAsync(st, &ds, sizeof(ds), cudaMemcpyHostToDevice, h->stream), "FPCG stats");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "synchronize");
    return rc;
  }
  if (h->prm.solver == CFD_SOLVER_DIC) {
    DicArgs a{};
    a.g = GridDims{h->prm.nx, h->prm.ny, h->prm.nz};
    a.x = x; a.b = h->b; a.r = h->r; a.z = h->d0; a.p = h->d1; a.q = h->q; a.t = h->e0; a.d = h->dicd;
    a.scratch = h->partials;
    a.setup = h->dic_ready ? 0 : 1;
    a.zero_x0 = zero_x0; a.remove_mean = 1; a.gauge = gauge; a.gauge_value = 1.0;
    a.rtol = h->prm.rtol;
    a.max_iters = iter_cap(h->prm);
    a.max_restarts = kMaxRestarts;
    DicResult res{};
    const int t = phase_begin(h, CFD_PHASE_PCG);
    rc = cuda_check(h, run_dic_pcg(a, h->stream, &h->launches, &res), "DIC-PCG");
    phase_end(h, t);
    if (rc) return rc;
    h->dic_ready = true;
    DevSolveStats ds{};
    ds.iters = res.iters;
    ds.outer_iters = 0;
    ds.restarts = res.restarts;
    ds.status = res.status;
    ds.rel_resid = res.rel_resid;
    ds.b_norm = res.b_norm;
    rc = cuda_check(h, cudaMemcpyAsync(st, &ds, sizeof(ds), cudaMemcpyHostToDevice, h->stream), "DIC stats");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "synchronize");
    return rc;
  }
  if (h->prm.solver == CFD_SOLVER_IR && h->prm.learned_guess) {
    // x0 = alpha M(b) from the attached network, then the graph-form solve
    if (!h->precond_net) return set_err(h, CFD_ERR_INVALID_ARG, "learned_guess without an attached network");
    IrArgs a = pressure_ir_args(h, x, 0, gauge, st, h->ctrl);
    UNetView nv{};
    unet_view(h->precond_net, &nv);
    a.net = h->precond_net;
    a.net_mode = nv.conv_mode;
    a.guess = 1;
    a.guess_warm = zero_x0 ? 0 : 1;  // warm start: the network corrects the starting x
    if (!ir_graph_eligible(a)) return set_err(h, CFD_ERR_INVALID_ARG, "learned_guess needs nx %% 4 == 0");
    const int t = phase_begin(h, CFD_PHASE_PCG);
    rc = cuda_check(h, launch_ir_graph(a, h->irg_state, &h->irg, h->stream), "IR graph launch");
    phase_end(h, t);
    return rc;
  }
  if (h->prm.solver == CFD_SOLVER_IR) {
    const IrArgs a = pressure_ir_args(h, x, zero_x0, gauge, st, h->ctrl);
    const int t = phase_begin(h, CFD_PHASE_PCG);
    if (use_ir_graph(h, a))
      rc = cuda_check(h, launch_ir_graph(a, h->irg_state, &h->irg, h->stream), "IR graph launch");
    else
      rc = cuda_check(h, launch_ir(a, h->lg, h->stream, &h->launches), "IR launch");
    phase_end(h, t);
    return rc;
  }
  const CgArgs a = pressure_cg_args(h, x, zero_x0, gauge, st, h->ctrl);
  const int t = phase_begin(h, CFD_PHASE_PCG);
  rc = cuda_check(h, launch_cg(a, h->lg, h->stream, &h->launches), "pressure CG launch");
  phase_end(h, t);
  return rc;
}

int run_substep(cfd_handle* h, int which, DevStepStats* st) {
  PhysArgs pa = phys(h);
  int rc = CFD_OK;
  switch (which) {
    case CFD_SUBSTEP_FORCES:
      if (h->prm.g[0] != 0.0 || h->prm.g[1] != 0.0 || h->prm.g[2] != 0.0) {
        const int t = phase_begin(h, CFD_PHASE_FORCES);
        rc = cuda_check(h, launch_forces(pa, h->stream, &h->launches), "forces");
        phase_end(h, t);
      }
      return rc;
    case CFD_SUBSTEP_ADVECT: {
      // (u, v, w) -> (ua, va, wa)
      const int t = phase_begin(h, CFD_PHASE_ADVECT);
      rc = cuda_check(h, launch_advect(pa, h->stream, &h->launches), "advect");
      phase_end(h, t);
      return rc;
    }
    case CFD_SUBSTEP_DIFFUSE:
      if (h->prm.nu > 0.0) {
        const int t = phase_begin(h, CFD_PHASE_DIFFUSE);
        if (diffusion_concurrent(h))
          rc = run_diffusion_concurrent(h, st);
        else
          for (int c = 0; c < 3 && !rc; ++c) rc = run_diffusion(h, c, &st->d[c]);
        phase_end(h, t);
      }
      return rc;
    case CFD_SUBSTEP_PROJECT: {
      int t = phase_begin(h, CFD_PHASE_DIVERGENCE);
      rc = cuda_check(h, launch_divergence(pa, h->stream, &h->launches), "divergence");
      phase_end(h, t);
      if (rc) return rc;
      rc = run_pressure(h, h->p, h->prm.warm_start ? 0 : 1, 1, &st->p);
      if (rc) return rc;
      t = phase_begin(h, CFD_PHASE_CORRECT);
      rc = cuda_check(h, launch_correct(pa, h->stream, &h->launches), "correct");
      phase_end(h, t);
      return rc;
    }
  }
  return set_err(h, CFD_ERR_INVALID_ARG, "unknown substep %d", which);
}

// Clear a stats slot so that skipped solves read as zero iterations / OK.
int clear_stats(cfd_handle* h, DevStepStats* st, int n) {
  return cuda_check(h, cudaMemsetAsync(st, 0, sizeof(DevStepStats) * size_t(n), h->stream), "memset stats");
}

int worst(int a, int b) {
  // more negative codes are not "worse" in general; prefer the first failure
  return a != CFD_OK ? a : b;
}

void to_public(const DevStepStats& d, cfd_solve_stats* o) {
  std::memset(o, 0, sizeof(*o));
  o->iters = d.p.iters;
  o->outer_iters = d.p.outer_iters;
  o->restarts = d.p.restarts;
  o->status = d.p.status;
  for (int c = 0; c < 3; ++c) o->diff_iters[c] = d.d[c].iters;
  int ds = CFD_OK;
  for (int c = 0; c < 3; ++c) ds = worst(ds, d.d[c].status);
  o->diff_status = ds;
  o->rel_resid = d.p.rel_resid;
  o->b_norm = d.p.b_norm;
}

// Copy n stats slots back (synchronising), convert, and return the worst status.
int gather_stats(cfd_handle* h, const DevStepStats* src, int n, cfd_solve_stats* out) {
  DevStepStats* host = static_cast<DevStepStats*>(std::malloc(sizeof(DevStepStats) * size_t(n > 0 ? n : 1)));
  if (!host) return set_err(h, CFD_ERR_INVALID_ARG, "out of host memory");
  int rc = cuda_check(h, cudaMemcpyAsync(host, src, sizeof(DevStepStats) * size_t(n), cudaMemcpyDeviceToHost, h->stream),
                      "copy stats");
  if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "synchronize");
  SolveCtrl ctrl{};
  if (!rc) rc = cuda_check(h, cudaMemcpyAsync(&ctrl, h->ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, h->stream), "copy ctrl");
  if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "synchronize");
  int status = CFD_OK;
  if (!rc) {
    for (int i = 0; i < n; ++i) {
      if (out) to_public(host[i], &out[i]);
      status = worst(status, host[i].p.status);
      for (int c = 0; c < 3; ++c) status = worst(status, host[i].d[c].status);
    }
    if (ctrl.error != 0) status = worst(status, ctrl.error);
  }
  std::free(host);
  if (rc) return rc;
  if (status != CFD_OK)
    set_err(h, status, "solver status %d (%s)", status,
            status == CFD_ERR_NOT_CONVERGED ? "not converged"
            : status == CFD_ERR_BREAKDOWN ? "CG breakdown"
            : status == CFD_ERR_TIMEOUT ? "device wait timed out" : "error");
  return status;
}

}  // namespace

extern "C" {

int cfd_workspace_bytes(const cfd_params* params, size_t* bytes) {
  int rc = validate(params);
  if (rc) return rc;
  if (!bytes) return set_err(nullptr, CFD_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = ws_layout(*params, kMaxBlocksBound).total;
  return CFD_OK;
}

namespace {
int create_handle(const cfd_params* params, void* dev_ws, size_t bytes, cfd_stream_t stream, cfd_handle** out,
                  bool standalone);
}  // namespace

int cfd_create(const cfd_params* params, void* dev_ws, size_t bytes, cfd_stream_t stream, cfd_handle** out) {
  return create_handle(params, dev_ws, bytes, stream, out, true);
}

namespace {
int create_handle(const cfd_params* params, void* dev_ws, size_t bytes, cfd_stream_t stream, cfd_handle** out,
                  bool standalone) {
  int rc = validate(params);
  if (rc) return rc;
  if (!out) return set_err(nullptr, CFD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!dev_ws) return set_err(nullptr, CFD_ERR_INVALID_ARG, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(dev_ws) & 255) return set_err(nullptr, CFD_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  Layout L = ws_layout(*params, kMaxBlocksBound, standalone);
  if (bytes < L.total)
    return set_err(nullptr, CFD_ERR_WORKSPACE_TOO_SMALL, "workspace %zu bytes < required %zu", bytes, L.total);
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, dev_ws) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return set_err(nullptr, CFD_ERR_INVALID_ARG, "workspace is not device memory");
  }
  cfd_handle* h = new (std::nothrow) cfd_handle();
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "out of host memory");
  h->prm = *params;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->ws = static_cast<char*>(dev_ws);
  h->ws_bytes = bytes;
  h->L = L;
  auto D = [&](size_t o) { return reinterpret_cast<double*>(h->ws + o); };
  auto F = [&](size_t o) { return reinterpret_cast<float*>(h->ws + o); };
  h->u = D(L.u); h->v = D(L.v); h->w = D(L.w);
  h->ua = D(L.ua); h->va = D(L.va); h->wa = D(L.wa); h->p = D(L.p);
  h->b = D(L.b); h->r = D(L.r); h->d0 = D(L.d0); h->d1 = D(L.d1); h->q = D(L.q);
  h->e0 = D(L.e0); h->e1 = D(L.e1); h->e2 = D(L.e2);
  if (params->solver == CFD_SOLVER_DIC) h->dicd = D(L.dicd);
  if (params->solver == CFD_SOLVER_IR || params->solver == CFD_SOLVER_FPCG) {
    h->r32 = F(L.r32); h->d32 = F(L.d32); h->p0_32 = F(L.p0_32); h->p1_32 = F(L.p1_32); h->q32 = F(L.q32);
    h->irg_state = h->ws + L.irg;
  }
  h->partials = D(L.partials);
  h->ctrl = reinterpret_cast<SolveCtrl*>(h->ws + L.ctrl);
  h->stats = reinterpret_cast<DevStepStats*>(h->ws + L.stats);
  if (L.conc)
    for (int c = 0; c < 2; ++c) {
      for (int v = 0; v < 8; ++v) h->cset[c][v] = D(L.cset[c][v]);
      h->cpartials[c] = D(L.cpartials[c]);
      h->cctrl[c] = reinterpret_cast<SolveCtrl*>(h->ws + L.cctrl[c]);
    }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->lg.num_sms, cudaDevAttrMultiProcessorCount, dev);
  h->lg.blocks = cg_max_coresident_blocks(params->solver == CFD_SOLVER_IR);
  if (h->lg.blocks > kMaxBlocksBound) h->lg.blocks = kMaxBlocksBound;
  if (h->lg.blocks < 1) {
    delete h;
    return set_err(nullptr, CFD_ERR_CUDA, "cannot place the solve kernel on this device");
  }
  std::snprintf(h->err, sizeof(h->err), "no error");
  // initial state (Sec. 3, eq. 3): v0 = 0, p0 = 1
  rc = cuda_check(h, cudaMemsetAsync(h->ws, 0, L.total, h->stream), "memset workspace");
  if (!rc) rc = cuda_check(h, launch_fill(h->p, size_t(params->nx) * params->ny * params->nz, 1.0, h->stream, &h->launches),
                          "fill p");
  // standalone cavities on small grids run their diffusion solves at once
  if (!rc && L.conc) rc = cfd_set_concurrent_diffusion(h, 1);
  if (rc) {
    cfd_destroy(h);
    return rc;
  }
  *out = h;
  return CFD_OK;
}
}  // namespace

void cfd_destroy(cfd_handle* h) {
  if (!h) return;
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->snap_ev) {
    cudaEventSynchronize(h->snap_ev);
    cudaEventDestroy(h->snap_ev);
  }
  if (h->snap) cudaFreeHost(h->snap);
  destroy_ir_graph(h->irg);
  for (cfd::IrGraph* g : h->irg_diff) destroy_ir_graph(g);
  for (int k = 0; k < 2; ++k) {
    if (h->aux[k]) {
      cudaStreamSynchronize(h->aux[k]);
      cudaStreamDestroy(h->aux[k]);
    }
    if (h->ev_join[k]) cudaEventDestroy(h->ev_join[k]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  delete h;
}

int cfd_snapshot(cfd_handle* h) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  const size_t nu = face_count(h->prm, 0), nv = face_count(h->prm, 1), nw = face_count(h->prm, 2);
  const size_t nc = size_t(h->prm.nx) * h->prm.ny * h->prm.nz;
  if (!h->snap) {
    void* p = nullptr;
    int rc = cuda_check(h, cudaMallocHost(&p, (nu + nv + nw + nc) * 8), "snapshot host buffer");
    if (rc) return rc;
    h->snap = static_cast<double*>(p);
  }
  if (!h->snap_ev) {
    int rc = cuda_check(h, cudaEventCreateWithFlags(&h->snap_ev, cudaEventDisableTiming), "snapshot event");
    if (rc) return rc;
  }
  if (h->snap_pending) {
    // the previous snapshot's copies may still be reading into the buffer
    int rc = cuda_check(h, cudaEventSynchronize(h->snap_ev), "snapshot wait");
    if (rc) return rc;
  }
  double* dst = h->snap;
  const double* src[4] = {h->u, h->v, h->w, h->p};
  const size_t cnt[4] = {nu, nv, nw, nc};
  for (int f = 0; f < 4; ++f) {
    int rc = cuda_check(h, cudaMemcpyAsync(dst, src[f], cnt[f] * 8, cudaMemcpyDeviceToHost, h->stream), "snapshot copy");
    if (rc) return rc;
    dst += cnt[f];
  }
  int rc = cuda_check(h, cudaEventRecord(h->snap_ev, h->stream), "snapshot record");
  if (rc) return rc;
  h->snap_pending = true;
  return CFD_OK;
}

int cfd_snapshot_write_csv(cfd_handle* h, const char* path, int nthreads) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (!path) return set_err(h, CFD_ERR_INVALID_ARG, "path is NULL");
  if (!h->snap_pending) return set_err(h, CFD_ERR_INVALID_ARG, "no snapshot taken (cfd_snapshot)");
  int rc = cuda_check(h, cudaEventSynchronize(h->snap_ev), "snapshot wait");
  if (rc) return rc;
  const int nx = h->prm.nx, ny = h->prm.ny, nz = h->prm.nz;
  const double hh = h->prm.length / nx;
  const size_t nu = face_count(h->prm, 0), nv = face_count(h->prm, 1), nw = face_count(h->prm, 2);
  const double* u = h->snap;
  const double* v = u + nu;
  const double* w = v + nv;
  const double* p = w + nw;
  if (nthreads <= 0) nthreads = int(std::thread::hardware_concurrency());
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nz) nthreads = nz;
  // each thread formats a contiguous range of z-planes into its own buffer
  std::vector<std::string> parts = std::vector<std::string>(size_t(nthreads));
  auto format = [&](int t) {
    const int k0 = int(int64_t(nz) * t / nthreads), k1 = int(int64_t(nz) * (t + 1) / nthreads);
    std::string& out = parts[size_t(t)];
    out.reserve(size_t(k1 - k0) * size_t(nx) * ny * 120);
    char line[256];
    for (int k = k0; k < k1; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          // cell-centred velocity: mean of the two faces along each axis
          const double uc = 0.5 * (u[(size_t(k) * ny + j) * (nx + 1) + i] + u[(size_t(k) * ny + j) * (nx + 1) + i + 1]);
          const double vc = 0.5 * (v[(size_t(k) * (ny + 1) + j) * nx + i] + v[(size_t(k) * (ny + 1) + j + 1) * nx + i]);
          const double wc = 0.5 * (w[(size_t(k) * ny + j) * nx + i] + w[(size_t(k + 1) * ny + j) * nx + i]);
          const double pc = p[(size_t(k) * ny + j) * nx + i];
          const int len = std::snprintf(line, sizeof(line), "%.17g,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g\n",
                                        (i + 0.5) * hh, (j + 0.5) * hh, (k + 0.5) * hh, uc, vc, wc, pc);
          out.append(line, size_t(len));
        }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nthreads; ++t) pool.emplace_back(format, t);
  format(0);
  for (auto& th : pool) th.join();
  std::FILE* f = std::fopen(path, "wb");
  if (!f) return set_err(h, CFD_ERR_INVALID_ARG, "cannot open %s for writing", path);
  static const char header[] = "x,y,z,u,v,w,p\n";
  bool ok = std::fwrite(header, 1, sizeof(header) - 1, f) == sizeof(header) - 1;
  for (const auto& s2 : parts) ok = ok && std::fwrite(s2.data(), 1, s2.size(), f) == s2.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return set_err(h, CFD_ERR_INVALID_ARG, "writing %s failed", path);
  return CFD_OK;
}

const char* cfd_last_error(const cfd_handle* h) { return h ? h->err : g_last_error; }

int cfd_set_stream(cfd_handle* h, cfd_stream_t stream) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return CFD_OK;
}

static int field_ptr(cfd_handle* h, int field, double** ptr, size_t* count, int64_t dims[3]) {
  const cfd_params& p = h->prm;
  switch (field) {
    case CFD_FIELD_U: *ptr = h->u; dims[0] = p.nx + 1; dims[1] = p.ny; dims[2] = p.nz; break;
    case CFD_FIELD_V: *ptr = h->v; dims[0] = p.nx; dims[1] = p.ny + 1; dims[2] = p.nz; break;
    case CFD_FIELD_W: *ptr = h->w; dims[0] = p.nx; dims[1] = p.ny; dims[2] = p.nz + 1; break;
    case CFD_FIELD_P: *ptr = h->p; dims[0] = p.nx; dims[1] = p.ny; dims[2] = p.nz; break;
    default: return set_err(h, CFD_ERR_INVALID_ARG, "unknown field %d", field);
  }
  *count = size_t(dims[0]) * dims[1] * dims[2];
  return CFD_OK;
}

int cfd_set_field(cfd_handle* h, int field, const double* src, int src_on_device) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (!src) return set_err(h, CFD_ERR_INVALID_ARG, "src is NULL");
  double* dst;
  size_t n;
  int64_t dims[3];
  int rc = field_ptr(h, field, &dst, &n, dims);
  if (rc) return rc;
  rc = cuda_check(h, cudaMemcpyAsync(dst, src, n * 8, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream),
                  "set_field copy");
  if (rc) return rc;
  if (field != CFD_FIELD_P) rc = cuda_check(h, launch_zero_wall_faces(phys(h), h->stream, &h->launches), "zero wall faces");
  return rc;
}

int cfd_read_field(cfd_handle* h, int field, double* dst, int dst_on_device, int64_t dims_out[3]) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  double* src;
  size_t n;
  int64_t dims[3];
  int rc = field_ptr(h, field, &src, &n, dims);
  if (rc) return rc;
  if (dims_out) { dims_out[0] = dims[0]; dims_out[1] = dims[1]; dims_out[2] = dims[2]; }
  if (!dst) return dims_out ? CFD_OK : set_err(h, CFD_ERR_INVALID_ARG, "dst is NULL");
  rc = cuda_check(h, cudaMemcpyAsync(dst, src, n * 8, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream),
                  "read_field copy");
  if (rc) return rc;
  if (!dst_on_device) rc = cuda_check(h, cudaStreamSynchronize(h->stream), "synchronize");
  return rc;
}

int cfd_step(cfd_handle* h, int nsteps, cfd_solve_stats* per_step) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (nsteps < 0) return set_err(h, CFD_ERR_INVALID_ARG, "nsteps must be >= 0");
  int status = CFD_OK;
  int done = 0;
  while (done < nsteps) {
    // steps fill the statistics ring in order; a chunk never wraps past the
    // end of the ring so that it can be gathered with one copy
    const int ring_pos = int(h->ring % kStatsCap);
    int chunk = nsteps - done;
    if (chunk > kStatsCap - ring_pos) chunk = kStatsCap - ring_pos;
    DevStepStats* base = h->stats + ring_pos;
    int rc = clear_stats(h, base, chunk);
    if (rc) return rc;
    for (int s = 0; s < chunk; ++s) {
      for (int which = CFD_SUBSTEP_FORCES; which <= CFD_SUBSTEP_PROJECT; ++which) {
        rc = run_substep(h, which, base + s);
        if (rc) return rc;
      }
    }
    h->ring += chunk;
    if (per_step) {
      rc = gather_stats(h, base, chunk, per_step + done);
      if (rc != CFD_OK && rc != CFD_ERR_NOT_CONVERGED && rc != CFD_ERR_BREAKDOWN && rc != CFD_ERR_TIMEOUT) return rc;
      status = worst(status, rc);
    }
    done += chunk;
  }
  return status;
}

int cfd_recent_stats(cfd_handle* h, int n, cfd_solve_stats* out) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0 || n > kStatsCap || int64_t(n) > h->ring || !out)
    return set_err(h, CFD_ERR_INVALID_ARG, "n must be in [0, min(steps taken, %d)] and out non-NULL", kStatsCap);
  // the last n ring slots, oldest first (at most two contiguous pieces)
  const int64_t first = h->ring - n;
  int status = CFD_OK;
  int done = 0;
  while (done < n) {
    const int pos = int((first + done) % kStatsCap);
    int len = n - done;
    if (len > kStatsCap - pos) len = kStatsCap - pos;
    int rc = gather_stats(h, h->stats + pos, len, out + done);
    if (rc != CFD_OK && rc != CFD_ERR_NOT_CONVERGED && rc != CFD_ERR_BREAKDOWN && rc != CFD_ERR_TIMEOUT) return rc;
    status = worst(status, rc);
    done += len;
  }
  return status;
}

int cfd_substep(cfd_handle* h, int which, cfd_solve_stats* stats) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (which < CFD_SUBSTEP_FORCES || which > CFD_SUBSTEP_PROJECT) return set_err(h, CFD_ERR_INVALID_ARG, "unknown substep %d", which);
  int rc = clear_stats(h, h->stats + kStatsCap, 1);
  if (rc) return rc;
  // Inside a step the diffusion and projection read the intermediate
  // velocity (ua, va, wa); a standalone substep starts from and ends in the
  // current velocity (u, v, w).
  auto copy_vel = [&](bool to_intermediate) {
    int r2 = CFD_OK;
    for (int c = 0; c < 3 && !r2; ++c) {
      double* cur = c == 0 ? h->u : (c == 1 ? h->v : h->w);
      double* mid = c == 0 ? h->ua : (c == 1 ? h->va : h->wa);
      const size_t n = face_count(h->prm, c);
      r2 = cuda_check(h, cudaMemcpyAsync(to_intermediate ? mid : cur, to_intermediate ? cur : mid, n * 8,
                                         cudaMemcpyDeviceToDevice, h->stream), "substep copy");
    }
    return r2;
  };
  if (which == CFD_SUBSTEP_DIFFUSE || which == CFD_SUBSTEP_PROJECT) rc = copy_vel(true);
  if (!rc) rc = run_substep(h, which, h->stats + kStatsCap);
  if (!rc && (which == CFD_SUBSTEP_ADVECT || which == CFD_SUBSTEP_DIFFUSE)) rc = copy_vel(false);
  if (rc) return rc;
  if (stats) return gather_stats(h, h->stats + kStatsCap, 1, stats);
  return CFD_OK;
}

int cfd_solve_pressure(cfd_handle* h, const double* b_dev, double* x_dev, cfd_solve_stats* stats) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (!b_dev || !x_dev) return set_err(h, CFD_ERR_INVALID_ARG, "b or x is NULL");
  const size_t n = size_t(h->prm.nx) * h->prm.ny * h->prm.nz;
  int rc = clear_stats(h, h->stats + kStatsCap, 1);
  if (!rc) rc = cuda_check(h, cudaMemcpyAsync(h->b, b_dev, n * 8, cudaMemcpyDeviceToDevice, h->stream), "copy b");
  if (!rc) rc = run_pressure(h, x_dev, h->prm.warm_start ? 0 : 1, 0, &(h->stats + kStatsCap)->p);
  if (rc) return rc;
  if (stats) return gather_stats(h, h->stats + kStatsCap, 1, stats);
  return CFD_OK;
}

int cfd_apply_poisson(cfd_handle* h, const double* x_dev, double* y_dev) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (!x_dev || !y_dev) return set_err(h, CFD_ERR_INVALID_ARG, "x or y is NULL");
  GridDims g{h->prm.nx, h->prm.ny, h->prm.nz};
  return cuda_check(h, launch_apply_poisson(g, x_dev, y_dev, tz_for(g.mz), h->stream, &h->launches), "apply_poisson");
}

namespace {
// deterministic right-hand side for shape tuning: hashed values in [-1, 1)
__global__ void tune_rhs_kernel(double* b, size_t n) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    uint64_t z = (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    b[i] = double(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}
}  // namespace

int cfd_attach_preconditioner(cfd_handle* h, cfd_unet* u) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (u) {
    if (h->prm.solver != CFD_SOLVER_FPCG && !(h->prm.solver == CFD_SOLVER_IR && h->prm.learned_guess))
      return set_err(h, CFD_ERR_INVALID_ARG, "a network needs solver FPCG, or IR with learned_guess = 1");
    int nx = 0, ny = 0, nz = 0;
    cfd_unet_grid(u, &nx, &ny, &nz);
    if (nx != h->prm.nx || ny != h->prm.ny || nz != h->prm.nz)
      return set_err(h, CFD_ERR_INVALID_ARG, "the network's grid %dx%dx%d differs from the cavity's", nx, ny, nz);
  }
  h->precond_net = u;
  return CFD_OK;
}

int cfd_set_cg_variant(cfd_handle* h, int variant) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (variant != CFD_CG_SINGLE_REDUCTION && variant != CFD_CG_TWO_REDUCTIONS)
    return set_err(h, CFD_ERR_INVALID_ARG, "unknown CG variant %d", variant);
  h->lg.cg_variant = variant;
  return CFD_OK;
}

int cfd_autotune_solver(cfd_handle* h, int32_t iters, cfd_tune_report* rep) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (iters < 1 || iters > 100000) return set_err(h, CFD_ERR_INVALID_ARG, "iters in [1, 100000]");
  const size_t n = size_t(h->prm.nx) * h->prm.ny * h->prm.nz;
  const cfd_params saved = h->prm;
  const int bps0 = h->lg.bps_req, tz0 = h->lg.tz_req;
  // fixed-length solves: rtol far below reach, cap = iters; x in the
  // intermediate-velocity slot (scratch between steps), state untouched
  h->prm.rtol = 1e-300;
  h->prm.max_iters = iters;
  double* x = h->ua;
  DevSolveStats* st = &(h->stats + kStatsCap)->p;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cuda_check(h, cudaEventCreate(&e0), "event");
  if (!rc) rc = cuda_check(h, cudaEventCreate(&e1), "event");
  const int var0 = h->lg.cg_variant;
  const int form0 = h->ir_form;
  auto time_shape = [&](int variant, int bps, int tz, int form, float& best_ms) -> int {
    h->ir_form = form;
    h->lg.cg_variant = variant;
    h->lg.bps_req = bps;
    h->lg.tz_req = tz;
    best_ms = 1e30f;
    for (int rep_i = 0; rep_i < 3; ++rep_i) {  // first run warms up
      tune_rhs_kernel<<<1216, 256, 0, h->stream>>>(h->b, n);
      int r = cuda_check(h, cudaGetLastError(), "tune rhs");
      if (!r) r = cuda_check(h, cudaEventRecord(e0, h->stream), "event record");
      if (!r) r = run_pressure(h, x, 1, 0, st);
      if (!r) r = cuda_check(h, cudaEventRecord(e1, h->stream), "event record");
      if (!r) r = cuda_check(h, cudaEventSynchronize(e1), "event sync");
      if (r) return r;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep_i > 0 && ms < best_ms) best_ms = ms;
    }
    return CFD_OK;
  };
  // the CG form is a candidate too when the solves are unpreconditioned FP64 CG
  const int nvar = h->prm.solver == CFD_SOLVER_CG ? 2 : 1;
  // the mixed-precision solve: shapes of the persistent form, then the graph form
  const bool ir = h->prm.solver == CFD_SOLVER_IR;
  const bool graph_ok = ir && h->irg_state && h->prm.nx % 4 == 0;
  const int shape_form = ir ? CFD_IR_PERSISTENT : form0;
  float ms_auto = 0.f, ms_best = 0.f;
  int best_bps = 0, best_tz = 0, best_var = var0, best_form = form0, tried = 0;
  if (!rc) rc = time_shape(var0, 0, 0, form0, ms_auto);
  ms_best = ms_auto;
  ++tried;
  const int bps_list[4] = {1, 2, 3, 4};
  const int tz_list[4] = {1, 2, 4, 8};
  for (int v = 0; v < nvar && !rc; ++v) {
    const int variant = nvar == 1 ? var0 : v;
    for (int i = -1; i < 4 && !rc; ++i) {
      for (int j = 0; j < 4 && !rc; ++j) {
        if (i < 0 && j > 0) break;
        if (i < 0 && variant == var0 && shape_form == form0) continue;  // timed above
        const int bps = i < 0 ? 0 : bps_list[i], tz = i < 0 ? 0 : tz_list[j];
        float ms = 0.f;
        rc = time_shape(variant, bps, tz, shape_form, ms);
        ++tried;
        if (!rc && ms < ms_best) {
          ms_best = ms;
          best_bps = bps;
          best_tz = tz;
          best_var = variant;
          best_form = shape_form;
        }
      }
    }
  }
  if (graph_ok && !rc) {
    float ms = 0.f;
    rc = time_shape(var0, 0, 0, CFD_IR_GRAPH, ms);
    ++tried;
    if (!rc && ms < ms_best) {
      ms_best = ms;
      best_bps = 0;
      best_tz = 0;
      best_var = var0;
      best_form = CFD_IR_GRAPH;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->prm = saved;
  if (rc) {
    h->lg.bps_req = bps0;
    h->lg.tz_req = tz0;
    h->lg.cg_variant = var0;
    h->ir_form = form0;
    return rc;
  }
  h->lg.bps_req = best_bps;
  h->lg.tz_req = best_tz;
  h->lg.cg_variant = best_var;
  h->ir_form = best_form;
  if (rep) {
    rep->blocks_per_sm = best_bps;
    rep->tile_depth = best_tz;
    rep->candidates = tried;
    rep->ms_auto = ms_auto;
    rep->ms_best = ms_best;
    rep->cg_variant = best_var;
    rep->ir_form = best_form;
  }
  return CFD_OK;
}

int cfd_pressure_rhs(cfd_handle* h, double* b_dev) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (!b_dev) return set_err(h, CFD_ERR_INVALID_ARG, "b is NULL");
  // the divergence sweep reads the intermediate-velocity slots: point them
  // at the current velocity and its output at the caller's array
  PhysArgs pa = phys(h);
  pa.ua = h->u; pa.va = h->v; pa.wa = h->w;
  pa.b = b_dev;
  return cuda_check(h, launch_divergence(pa, h->stream, &h->launches), "divergence");
}

int cfd_harvest_pair(cfd_handle* h, const double* b_dev, const double* xs_dev, const double* xk_dev, double* r_dev,
                     double* e_dev) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (!b_dev || !xs_dev || !xk_dev || !r_dev || !e_dev) return set_err(h, CFD_ERR_INVALID_ARG, "NULL vector");
  if (r_dev == xk_dev || r_dev == b_dev || r_dev == xs_dev || e_dev == xk_dev || e_dev == xs_dev || r_dev == e_dev)
    return set_err(h, CFD_ERR_INVALID_ARG, "r and e must not alias the inputs or each other");
  static_assert(partials_doubles(kMaxBlocksBound) >= 2 * 512 + 2, "partial-sum scratch too small for the harvest");
  if (harvest_scratch_doubles() > partials_doubles(kMaxBlocksBound))
    return set_err(h, CFD_ERR_INVALID_ARG, "harvest scratch does not fit");
  return cuda_check(h, launch_harvest_pair(GridDims{h->prm.nx, h->prm.ny, h->prm.nz}, b_dev, xs_dev, xk_dev, r_dev,
                                           e_dev, h->partials, h->stream, &h->launches),
                    "harvest pair");
}

int cfd_learned_guess(cfd_handle* h, const double* b_dev, double* x_dev) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (!b_dev || !x_dev || b_dev == x_dev) return set_err(h, CFD_ERR_INVALID_ARG, "b and x must be distinct device arrays");
  if (!h->precond_net) return set_err(h, CFD_ERR_INVALID_ARG, "no network attached");
  if (!h->irg_state || h->prm.nx % 4 != 0)
    return set_err(h, CFD_ERR_INVALID_ARG, "the learned guess needs solver IR or FPCG and nx %% 4 == 0");
  IrArgs a = pressure_ir_args(h, x_dev, 0, 0, &(h->stats + kStatsCap)->p, h->ctrl);
  a.b = const_cast<double*>(b_dev);  // read only
  a.net = h->precond_net;
  return cuda_check(h, launch_learned_guess(a, h->irg_state, h->stream, &h->launches), "learned guess");
}

int cfd_set_wait_limit(cfd_handle* h, uint64_t limit_ns) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  h->wait_ns = limit_ns == UINT64_MAX ? kTimeoutNs : static_cast<unsigned long long>(limit_ns);
  return CFD_OK;
}

int64_t cfd_launch_count(const cfd_handle* h) {
  if (!h) return 0;
  // kernels of the graph form (and of the learned guess) count themselves
  // in the graph state on the device
  long long graph_kernels = 0;
  if (h->irg_state && ir_graph_kernel_count(h->irg_state, h->stream, &graph_kernels) != cudaSuccess)
    graph_kernels = 0;
  return h->launches + graph_kernels;
}

int cfd_set_concurrent_diffusion(cfd_handle* h, int on) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (on != 0 && on != 1) return set_err(h, CFD_ERR_INVALID_ARG, "on must be 0 or 1");
  if (on && !h->cset[0][0])
    return set_err(h, CFD_ERR_INVALID_ARG, "concurrent diffusion needs nu > 0 and at most 2^21 cells");
  if (on && !h->aux[0]) {
    int rc = CFD_OK;
    for (int k = 0; k < 2 && !rc; ++k) {
      rc = cuda_check(h, cudaStreamCreateWithFlags(&h->aux[k], cudaStreamNonBlocking), "stream");
      if (!rc) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_join[k], cudaEventDisableTiming), "event");
    }
    if (!rc) rc = cuda_check(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "event");
    if (rc) return rc;
  }
  h->conc_diffusion = on != 0;
  return CFD_OK;
}

int cfd_set_fpcg_form(cfd_handle* h, int form) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (form != CFD_FPCG_GRAPH && form != CFD_FPCG_HOST) return set_err(h, CFD_ERR_INVALID_ARG, "unknown FPCG form %d", form);
  if (h->prm.solver != CFD_SOLVER_FPCG) return set_err(h, CFD_ERR_INVALID_ARG, "the handle's solver is not FPCG");
  if (form == CFD_FPCG_GRAPH && h->prm.nx % 4 != 0)
    return set_err(h, CFD_ERR_INVALID_ARG, "the FPCG graph form needs nx %% 4 == 0");
  h->fpcg_form = form;
  return CFD_OK;
}

int cfd_set_ir_form(cfd_handle* h, int form) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (form != CFD_IR_AUTO && form != CFD_IR_PERSISTENT && form != CFD_IR_GRAPH)
    return set_err(h, CFD_ERR_INVALID_ARG, "unknown IR form %d", form);
  if (form == CFD_IR_GRAPH && h->prm.nx % 4 != 0)
    return set_err(h, CFD_ERR_INVALID_ARG, "the graph form needs nx %% 4 == 0");
  h->ir_form = form;
  return CFD_OK;
}

int cfd_set_solver_shape(cfd_handle* h, int blocks_per_sm, int tile_depth) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (blocks_per_sm < 0 || blocks_per_sm > 32 || tile_depth < 0 || tile_depth > 64)
    return set_err(h, CFD_ERR_INVALID_ARG, "blocks_per_sm in [0, 32] and tile_depth in [0, 64]");
  h->lg.bps_req = blocks_per_sm;
  h->lg.tz_req = tile_depth;
  return CFD_OK;
}

int cfd_get_solver_shape(cfd_handle* h, int kind, int* blocks, int* tile_depth, int* register_path) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  if (kind < 0 || kind > 3) return set_err(h, CFD_ERR_INVALID_ARG, "kind must be 0 (pressure) or 1..3 (u, v, w)");
  GridDims g{h->prm.nx + (kind == 1), h->prm.ny + (kind == 2), h->prm.nz + (kind == 3)};
  const SolveShape s = pick_solve_shape(g, h->lg.blocks, h->lg.bps_req, h->lg.tz_req);
  if (blocks) *blocks = s.blocks;
  if (tile_depth) *tile_depth = s.tz;
  if (register_path) *register_path = s.rtz > 0;
  // unpreconditioned single-reduction FP64 CG on the whole device: the
  // tile-resident kernel when the grid qualifies
  const bool fp64_cg = kind == 0 ? h->prm.solver == CFD_SOLVER_CG : !ir_diffusion(h) && !diffusion_concurrent(h);
  if (fp64_cg && h->lg.cg_variant == CFD_CG_SINGLE_REDUCTION) {
    if (const int tiles = cgt_blocks_for(g, h->lg)) {
      if (blocks) *blocks = tiles;
      if (tile_depth) *tile_depth = kCgtTileDepth;
      if (register_path) *register_path = 2;
    }
  }
  return CFD_OK;
}

int cfd_enable_timing(cfd_handle* h, int on) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  h->timing = on != 0;
  return CFD_OK;
}

int cfd_phase_times(cfd_handle* h, double* ms_out, int64_t* calls_out) {
  if (!h) return set_err(nullptr, CFD_ERR_INVALID_ARG, "handle is NULL");
  int rc = cuda_check(h, cudaStreamSynchronize(h->stream), "synchronize");
  if (rc) return rc;
  double ms[CFD_PHASE_COUNT] = {0};
  int64_t calls[CFD_PHASE_COUNT] = {0};
  for (const auto& p : h->pending) {
    float t = 0.f;
    rc = cuda_check(h, cudaEventElapsedTime(&t, p.a, p.b), "event elapsed");
    if (rc) return rc;
    ms[p.phase] += t;
    calls[p.phase] += 1;
  }
  h->pending.clear();
  h->ev_next = 0;
  for (int i = 0; i < CFD_PHASE_COUNT; ++i) {
    if (ms_out) ms_out[i] = ms[i];
    if (calls_out) calls_out[i] = calls[i];
  }
  return CFD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent cavities.
//
// Every cavity keeps its own handle and workspace slice.  The sweeps run as
// one launch per cavity; each family of solves (diffusion of u, of v, of w,
// and the pressure) runs as ONE cooperative persistent launch in which
// cavity i owns a contiguous range of blocks, sized in proportion to
// cells^(4/3) (CG work grows like cells x N), with its own control block and
// all-reduces, so cavities never wait on each other.  A whole step can be
// captured once into a CUDA graph and replayed.
// ---------------------------------------------------------------------------
struct cfd_batch {
  int n;
  cudaStream_t stream;
  char* ws;
  size_t bytes;
  std::vector<cfd_handle*> cav;
  int solver;
  // device tables inside the batch workspace
  CgArgs* d_cg;            // [4][n]: diffusion u, v, w (first nd entries), pressure CG
  IrArgs* d_ir;            // [4][n]: mixed-precision diffusion u, v, w (first nd entries), pressure
  char* d_gir;             // [4][n] entries of the batched graph-form solve (ir_batch_table), same order
  // batched sweeps: cavity tables (all cavities, those with nu > 0, those
  // with forces) and block starts per sweep slot (advect, forces, diffusion
  // rhs u / v / w, divergence, correct)
  PhysArgs* d_phys;        // [3][n]
  int* d_sweep_starts;     // [kSweepSlots][n + 1]
  int sweep_total[7];
  std::vector<int> force_idx;
  int* d_starts;           // [5][n + 1]
  SolveCtrl* d_ctrl;       // [4][n]
  DevSolveStats* d_stats;  // [4][n]
  std::vector<int> diff_idx;  // cavities with nu > 0
  int total_blocks[5];
  int precond;
  int64_t launches;
  bool use_graph;
  bool graph_ok;
  cudaGraphExec_t graph;
  int64_t graph_launches;  // kernel launches per replay
  char err[256];
};

namespace {

constexpr int kSweepSlots = 7;

struct BatchLayout {
  size_t cg, ir, gir, phys, sweep_starts, starts, ctrl, stats, cav0;
  std::vector<size_t> cav;
  size_t total;
};

BatchLayout batch_layout(int n, const cfd_params* prm) {
  BatchLayout L;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off = align256(off + b);
    return o;
  };
  L.cg = take(sizeof(CgArgs) * 4 * size_t(n));
  L.ir = take(sizeof(IrArgs) * 4 * size_t(n));  // [kind][cavity]: diffusion u, v, w, then pressure
  L.gir = take(ir_batch_table_bytes(4 * n));
  L.phys = take(sizeof(PhysArgs) * 3 * size_t(n));
  L.sweep_starts = take(sizeof(int) * kSweepSlots * size_t(n + 1));
  L.starts = take(sizeof(int) * 5 * size_t(n + 1));
  L.ctrl = take(sizeof(SolveCtrl) * 4 * size_t(n));
  L.stats = take(sizeof(DevSolveStats) * 4 * size_t(n));
  L.cav0 = off;
  for (int i = 0; i < n; ++i) L.cav.push_back(take(ws_layout(prm[i], kMaxBlocksBound, false).total));
  L.total = off;
  return L;
}

int batch_err(cfd_batch* b, int code, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) std::memcpy(b->err, buf, sizeof(buf));
  std::memcpy(g_last_error, buf, sizeof(buf));
  return code;
}

// Split `total` blocks over problems in proportion to weight (at least one
// each); returns prefix starts (size n + 1) or an empty vector if n > total.
std::vector<int> split_blocks(const std::vector<double>& w, int total) {
  const int n = int(w.size());
  std::vector<int> starts(size_t(n) + 1, 0);
  if (n == 0) return starts;
  if (n > total) return {};
  double W = 0.0;
  for (double x : w) W += x;
  std::vector<int> nb = std::vector<int>(static_cast<size_t>(n));
  int sum = 0;
  for (int i = 0; i < n; ++i) {
    nb[size_t(i)] = std::max(1, int(double(total) * w[size_t(i)] / W));
    sum += nb[size_t(i)];
  }
  while (sum > total) {  // trim the largest allocations
    int k = 0;
    for (int i = 1; i < n; ++i)
      if (nb[size_t(i)] > nb[size_t(k)]) k = i;
    if (nb[size_t(k)] <= 1) return {};
    --nb[size_t(k)];
    --sum;
  }
  for (int i = 0; i < n; ++i) starts[size_t(i) + 1] = starts[size_t(i)] + nb[size_t(i)];
  return starts;
}

// Split `total` blocks over problems whose time on nb blocks is
// extent * ceil(items / nb) (the batched graph-form solve): one block each,
// then, while blocks remain, the slowest problem gets the blocks that take
// it to its next shorter time.  Returns prefix starts (size n + 1) or an
// empty vector if n > total.
std::vector<int> split_blocks_balanced(const std::vector<int>& items, const std::vector<int>& extent, int total) {
  const int n = int(items.size());
  std::vector<int> starts(size_t(n) + 1, 0);
  if (n == 0) return starts;
  if (n > total) return {};
  std::vector<int> nb(size_t(n), 1);
  auto cost = [&](int i, int b) {
    return double(extent[size_t(i)]) * double((items[size_t(i)] + b - 1) / b);
  };
  std::priority_queue<std::pair<double, int>> q;
  for (int i = 0; i < n; ++i) q.push({cost(i, 1), i});
  int left = total - n;
  while (left > 0 && !q.empty()) {
    const int i = q.top().second;
    const int it = items[size_t(i)], b = nb[size_t(i)];
    const int per = (it + b - 1) / b;
    if (per <= 1) break;  // the slowest problem has one item per block: nothing shortens the longest time
    const int need = (it + per - 2) / (per - 1) - b;  // blocks to reach ceil(items / nb) = per - 1
    if (need > left) break;
    q.pop();
    nb[size_t(i)] = b + need;
    left -= need;
    q.push({cost(i, nb[size_t(i)]), i});
  }
  for (int i = 0; i < n; ++i) starts[size_t(i) + 1] = starts[size_t(i)] + nb[size_t(i)];
  return starts;
}

// Enqueue one step of every cavity.
int batch_enqueue_step(cfd_batch* b) {
  const int n = b->n;
  int rc = CFD_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == CFD_OK) rc = batch_err(b, CFD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return rc == CFD_OK;
  };
  auto sweep = [&](int slot, int table, int count, int op, int comp, const char* what) {
    ck(launch_sweep_multi(op, b->d_phys + size_t(table) * n, b->d_sweep_starts + size_t(slot) * (n + 1), count,
                          b->sweep_total[slot], comp, b->stream, &b->launches),
       what);
  };
  if (!b->force_idx.empty()) sweep(1, 2, int(b->force_idx.size()), kSweepForces, 0, "forces");
  sweep(0, 0, n, kSweepAdvect, 0, "advect");
  const int nd = int(b->diff_idx.size());
  for (int c = 0; c < 3 && nd > 0 && rc == CFD_OK; ++c) {
    sweep(2 + c, 1, nd, kSweepDiffusionRhs, c, "diffusion rhs");
    ck(cudaMemsetAsync(b->d_ctrl + size_t(c) * n, 0, sizeof(SolveCtrl) * size_t(nd), b->stream), "memset ctrl");
    if (b->solver == CFD_SOLVER_IR)
      ck(launch_ir_batch(b->d_gir + size_t(c) * n * ir_batch_table_bytes(1), b->d_starts + size_t(c) * (n + 1), nd,
                         b->total_blocks[c], kOpVelU + c, b->stream, &b->launches),
         "batched mixed-precision diffusion launch");
    else
      ck(launch_cg_multi(b->d_cg + size_t(c) * n, b->d_starts + size_t(c) * (n + 1), nd, b->total_blocks[c], 0,
                         b->stream, &b->launches),
         "batched diffusion launch");
  }
  sweep(5, 0, n, kSweepDivergence, 0, "divergence");
  ck(cudaMemsetAsync(b->d_ctrl + size_t(3) * n, 0, sizeof(SolveCtrl) * size_t(n), b->stream), "memset ctrl");
  if (b->solver == CFD_SOLVER_IR)
    ck(launch_ir_batch(b->d_gir + size_t(3) * n * ir_batch_table_bytes(1), b->d_starts + size_t(4) * (n + 1), n,
                       b->total_blocks[4], kOpPressure, b->stream, &b->launches),
       "batched pressure launch");
  else
    ck(launch_cg_multi(b->d_cg + size_t(3) * n, b->d_starts + size_t(3) * (n + 1), n, b->total_blocks[3], b->precond,
                       b->stream, &b->launches),
       "batched pressure launch");
  sweep(6, 0, n, kSweepCorrect, 0, "correct");
  return rc;
}

}  // namespace

extern "C" {

int cfd_batch_workspace_bytes(int n, const cfd_params* per_cavity, size_t* bytes) {
  if (n < 1 || !per_cavity || !bytes) return batch_err(nullptr, CFD_ERR_INVALID_ARG, "n >= 1, params and bytes required");
  for (int i = 0; i < n; ++i) {
    int rc = validate(&per_cavity[i]);
    if (rc) return rc;
  }
  *bytes = batch_layout(n, per_cavity).total;
  return CFD_OK;
}

int cfd_batch_create(int n, const cfd_params* per_cavity, void* dev_ws, size_t bytes, cfd_stream_t stream,
                     cfd_batch** out) {
  if (!out) return batch_err(nullptr, CFD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  size_t need = 0;
  int rc = cfd_batch_workspace_bytes(n, per_cavity, &need);
  if (rc) return rc;
  if (!dev_ws || (reinterpret_cast<uintptr_t>(dev_ws) & 255))
    return batch_err(nullptr, CFD_ERR_INVALID_ARG, "workspace NULL or not 256-byte aligned");
  if (bytes < need) return batch_err(nullptr, CFD_ERR_WORKSPACE_TOO_SMALL, "batch workspace %zu < %zu", bytes, need);
  const int solver = per_cavity[0].solver;
  if (solver == CFD_SOLVER_DIC || solver == CFD_SOLVER_FPCG)
    return batch_err(nullptr, CFD_ERR_INVALID_ARG, "batches do not support the DIC or FPCG solvers");
  for (int i = 1; i < n; ++i)
    if (per_cavity[i].solver != solver) return batch_err(nullptr, CFD_ERR_INVALID_ARG, "all cavities of a batch use one solver");
  for (int i = 0; i < n; ++i)
    if (per_cavity[i].learned_guess)
      return batch_err(nullptr, CFD_ERR_INVALID_ARG, "batches do not support the learned initial guess");
  const BatchLayout L = batch_layout(n, per_cavity);
  cfd_batch* b = new (std::nothrow) cfd_batch();
  if (!b) return batch_err(nullptr, CFD_ERR_INVALID_ARG, "out of host memory");
  b->n = n;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->ws = static_cast<char*>(dev_ws);
  b->bytes = bytes;
  b->solver = solver;
  b->precond = solver == CFD_SOLVER_JACOBI ? 1 : 0;
  b->d_cg = reinterpret_cast<CgArgs*>(b->ws + L.cg);
  b->d_ir = reinterpret_cast<IrArgs*>(b->ws + L.ir);
  b->d_gir = b->ws + L.gir;
  b->d_phys = reinterpret_cast<PhysArgs*>(b->ws + L.phys);
  b->d_sweep_starts = reinterpret_cast<int*>(b->ws + L.sweep_starts);
  b->d_starts = reinterpret_cast<int*>(b->ws + L.starts);
  b->d_ctrl = reinterpret_cast<SolveCtrl*>(b->ws + L.ctrl);
  b->d_stats = reinterpret_cast<DevSolveStats*>(b->ws + L.stats);
  std::snprintf(b->err, sizeof(b->err), "no error");
  auto fail = [&](int code) {
    for (cfd_handle* h : b->cav) cfd_destroy(h);
    delete b;
    return code;
  };
  for (int i = 0; i < n; ++i) {
    cfd_handle* h = nullptr;
    rc = create_handle(&per_cavity[i], b->ws + L.cav[size_t(i)],
                       L.cav.size() > size_t(i) + 1 ? L.cav[size_t(i) + 1] - L.cav[size_t(i)] : L.total - L.cav[size_t(i)],
                       stream, &h, false);
    if (rc) return fail(rc);
    b->cav.push_back(h);
    if (per_cavity[i].nu > 0.0) b->diff_idx.push_back(i);
    if (per_cavity[i].g[0] != 0.0 || per_cavity[i].g[1] != 0.0 || per_cavity[i].g[2] != 0.0) b->force_idx.push_back(i);
  }
  // block split and solve tables
  const int sms = batch_num_sms();
  std::vector<CgArgs> cg(4 * size_t(n));
  std::vector<IrArgs> ir = std::vector<IrArgs>(4 * static_cast<size_t>(n));
  const bool mixed = solver == CFD_SOLVER_IR;
  std::vector<int> starts(5 * size_t(n + 1), 0);
  auto weights = [&](const std::vector<int>& idx, int comp) {
    std::vector<double> w;
    for (int i : idx) {
      const cfd_params& p = per_cavity[i];
      const double cells = double(p.nx + (comp == 0)) * double(p.ny + (comp == 1)) * double(p.nz + (comp == 2));
      w.push_back(std::pow(cells, 4.0 / 3.0));
    }
    return w;
  };
  std::vector<int> all = std::vector<int>(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i) all[size_t(i)] = i;
  for (int kind = 0; kind < 5; ++kind) {
    const bool is_ir = kind == 4;
    const std::vector<int>& idx = kind < 3 ? b->diff_idx : all;
    // the mixed-precision solves (diffusion kinds 0-2 and pressure kind 4)
    // run the batched graph-form kernel (one wave, at most 4 blocks per SM)
    const int bps = (kind < 3 && mixed) || is_ir ? std::min(4, ir_batch_blocks_per_sm(kind < 3 ? kOpVelU + kind : kOpPressure))
                                                 : batch_blocks_per_sm();
    const int total = bps * sms;
    const bool ir_kind = (kind < 3 && mixed) || is_ir;
    std::vector<int> st;
    if (ir_kind) {
      // the batched graph-form solve: blocks in proportion to each
      // cavity's (row, plane) steps times its iteration count
      std::vector<int> items, extent;
      for (int i : idx) {
        cfd_handle* h = b->cav[size_t(i)];
        int it = 1, ex = 1;
        ir_batch_work(kind < 3 ? diffusion_ir_args(h, kind, nullptr) : pressure_ir_args(h, h->p, 0, 1, nullptr, nullptr),
                      &it, &ex);
        items.push_back(it);
        extent.push_back(ex);
      }
      st = split_blocks_balanced(items, extent, total);
    } else {
      st = split_blocks(weights(idx, kind < 3 ? kind : 3), total);
    }
    if (st.empty()) {
      rc = batch_err(nullptr, CFD_ERR_INVALID_ARG, "%zu cavities exceed the %d co-resident blocks of one launch", idx.size(), total);
      return fail(rc);
    }
    b->total_blocks[kind] = st.back();
    for (size_t k = 0; k < st.size(); ++k) starts[size_t(kind) * (n + 1) + k] = st[k];
    for (size_t k = 0; k < idx.size(); ++k) {
      cfd_handle* h = b->cav[size_t(idx[k])];
      const int nbk = st[k + 1] - st[k];
      if (kind < 3) {
        CgArgs a = diffusion_args(h, kind, b->d_stats + size_t(kind) * n + size_t(idx[k]), b->d_ctrl + size_t(kind) * n + k);
        a.tz = solve_tile_depth_for(a.g, nbk);
        cg[size_t(kind) * n + k] = a;
        if (mixed) {
          IrArgs d = diffusion_ir_args(h, kind, b->d_stats + size_t(kind) * n + size_t(idx[k]));
          d.ctrl = b->d_ctrl + size_t(kind) * n + k;
          d.partials = h->partials;
          d.tz = a.tz;
          d.use_tma = 0;
          ir[size_t(kind) * n + k] = d;
        }
      } else if (kind == 3) {
        CgArgs a = pressure_cg_args(h, h->p, h->prm.warm_start ? 0 : 1, 1, b->d_stats + size_t(3) * n + k, b->d_ctrl + size_t(3) * n + k);
        a.tz = solve_tile_depth_for(a.g, nbk);
        cg[size_t(3) * n + k] = a;
      } else {
        IrArgs a = pressure_ir_args(h, h->p, h->prm.warm_start ? 0 : 1, 1, b->d_stats + size_t(3) * n + k, b->d_ctrl + size_t(3) * n + k);
        a.tz = solve_tile_depth_for(a.g, nbk);
        a.use_tma = 0;
        ir[size_t(3) * n + k] = a;
      }
    }
  }
  if (mixed) {
    // entries of the batched graph-form solve: diffusion kinds over the
    // cavities with nu > 0, the pressure over all; partial sums in each
    // cavity's graph state
    const size_t entry = ir_batch_table_bytes(1);
    for (int kind = 0; kind < 4 && !rc; ++kind) {
      const std::vector<int>& idx = kind < 3 ? b->diff_idx : all;
      if (idx.empty()) continue;
      std::vector<void*> states;
      for (int i : idx) states.push_back(b->cav[size_t(i)]->irg_state);
      rc = cuda_check(nullptr, ir_batch_table(&ir[size_t(kind) * n], states.data(), int(idx.size()),
                                               b->d_gir + size_t(kind) * n * entry, b->stream),
                      "batched solve table");
    }
    if (rc) return fail(rc);
  }
  {
    // batched sweeps: per slot, each cavity gets the grid its single-cavity
    // sweep launches
    std::vector<PhysArgs> ph(3 * size_t(n));
    const std::vector<int>* subsets[3] = {&all, &b->diff_idx, &b->force_idx};
    for (int t = 0; t < 3; ++t)
      for (size_t k = 0; k < subsets[t]->size(); ++k) ph[size_t(t) * n + k] = phys(b->cav[size_t((*subsets[t])[k])]);
    const int slot_table[kSweepSlots] = {0, 2, 1, 1, 1, 0, 0};
    const int slot_op[kSweepSlots] = {kSweepAdvect, kSweepForces, kSweepDiffusionRhs, kSweepDiffusionRhs,
                                      kSweepDiffusionRhs, kSweepDivergence, kSweepCorrect};
    std::vector<int> sst(size_t(kSweepSlots) * (n + 1), 0);
    for (int slot = 0; slot < kSweepSlots; ++slot) {
      const int t = slot_table[slot];
      const int comp = slot >= 2 && slot <= 4 ? slot - 2 : 0;
      int acc = 0;
      for (size_t k = 0; k < subsets[t]->size(); ++k) {
        sst[size_t(slot) * (n + 1) + k] = acc;
        acc += sweep_blocks_for(ph[size_t(t) * n + k], slot_op[slot], comp);
      }
      sst[size_t(slot) * (n + 1) + subsets[t]->size()] = acc;
      b->sweep_total[slot] = acc;
    }
    rc = cuda_check(nullptr, cudaMemcpyAsync(b->d_phys, ph.data(), sizeof(PhysArgs) * ph.size(), cudaMemcpyHostToDevice,
                                             b->stream), "copy tables");
    if (!rc)
      rc = cuda_check(nullptr, cudaMemcpyAsync(b->d_sweep_starts, sst.data(), sizeof(int) * sst.size(),
                                               cudaMemcpyHostToDevice, b->stream), "copy tables");
    if (!rc) rc = cuda_check(nullptr, cudaStreamSynchronize(b->stream), "synchronize");  // ph, sst are released
    if (rc) return fail(rc);
  }
  rc = cuda_check(nullptr, cudaMemcpyAsync(b->d_cg, cg.data(), sizeof(CgArgs) * cg.size(), cudaMemcpyHostToDevice, b->stream), "copy tables");
  if (!rc) rc = cuda_check(nullptr, cudaMemcpyAsync(b->d_ir, ir.data(), sizeof(IrArgs) * ir.size(), cudaMemcpyHostToDevice, b->stream), "copy tables");
  if (!rc) rc = cuda_check(nullptr, cudaMemcpyAsync(b->d_starts, starts.data(), sizeof(int) * starts.size(), cudaMemcpyHostToDevice, b->stream), "copy tables");
  if (!rc) rc = cuda_check(nullptr, cudaMemsetAsync(b->d_stats, 0, sizeof(DevSolveStats) * 4 * size_t(n), b->stream), "memset stats");
  if (!rc) rc = cuda_check(nullptr, cudaStreamSynchronize(b->stream), "synchronize");
  if (rc) return fail(rc);
  *out = b;
  return CFD_OK;
}

void cfd_batch_destroy(cfd_batch* b) {
  if (!b) return;
  if (b->graph_ok) cudaGraphExecDestroy(b->graph);
  for (cfd_handle* h : b->cav) cfd_destroy(h);
  delete b;
}

const char* cfd_batch_last_error(const cfd_batch* b) { return b ? b->err : g_last_error; }

cfd_handle* cfd_batch_cavity(cfd_batch* b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->cav[size_t(i)];
}

int cfd_batch_blocks(const cfd_batch* b, int kind, int* total_blocks) {
  if (!b || kind < 0 || kind > 4 || !total_blocks) return batch_err(nullptr, CFD_ERR_INVALID_ARG, "bad arguments");
  *total_blocks = b->total_blocks[kind];
  return CFD_OK;
}

int cfd_batch_use_graph(cfd_batch* b, int on) {
  if (!b) return batch_err(nullptr, CFD_ERR_INVALID_ARG, "batch is NULL");
  b->use_graph = on != 0;
  return CFD_OK;
}

int cfd_batch_step(cfd_batch* b, int nsteps, cfd_solve_stats* per_cavity) {
  if (!b) return batch_err(nullptr, CFD_ERR_INVALID_ARG, "batch is NULL");
  if (nsteps < 0) return batch_err(b, CFD_ERR_INVALID_ARG, "nsteps must be >= 0");
  int rc = CFD_OK;
  if (b->use_graph && !b->graph_ok && nsteps > 0) {
    // capture one step once; replay it afterwards
    // (captured on a private stream: the caller's may be the legacy default
    // stream, which cannot be captured; the graph is launched on the caller's)
    cudaGraph_t g = nullptr;
    const int64_t l0 = b->launches;
    cudaStream_t user = b->stream, cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      b->stream = cs;
      const int erc = batch_enqueue_step(b);
      b->stream = user;
      e = cudaStreamEndCapture(cs, &g);
      if (erc == CFD_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&b->graph, g, 0);
      if (erc == CFD_OK && e == cudaSuccess && g) {
        b->graph_ok = true;
        b->graph_launches = b->launches - l0;
      }
      if (g) cudaGraphDestroy(g);
    }
    if (cs) cudaStreamDestroy(cs);
    b->launches = l0;
    if (!b->graph_ok) {
      batch_err(b, CFD_OK, "graph capture not possible (%s); using direct launches", cudaGetErrorString(e));
      b->use_graph = false;
    }
    cudaGetLastError();
  }
  for (int s = 0; s < nsteps && rc == CFD_OK; ++s) {
    if (b->graph_ok) {
      const cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
      if (e != cudaSuccess) rc = batch_err(b, CFD_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
      b->launches += b->graph_launches;
    } else {
      rc = batch_enqueue_step(b);
    }
  }
  if (rc || !per_cavity) return rc;
  std::vector<DevSolveStats> st(4 * size_t(b->n));
  rc = cuda_check(nullptr, cudaMemcpyAsync(st.data(), b->d_stats, sizeof(DevSolveStats) * st.size(), cudaMemcpyDeviceToHost, b->stream), "copy stats");
  if (!rc) rc = cuda_check(nullptr, cudaStreamSynchronize(b->stream), "synchronize");
  if (rc) return batch_err(b, rc, "%s", g_last_error);
  int status = CFD_OK;
  for (int i = 0; i < b->n; ++i) {
    DevStepStats d{};
    d.p = st[size_t(3) * b->n + size_t(i)];
    for (int c = 0; c < 3; ++c) d.d[c] = st[size_t(c) * b->n + size_t(i)];
    to_public(d, &per_cavity[i]);
    status = worst(status, d.p.status);
    for (int c = 0; c < 3; ++c) status = worst(status, d.d[c].status);
  }
  if (status != CFD_OK) batch_err(b, status, "solver status %d in the batch", status);
  return status;
}

int64_t cfd_batch_launch_count(const cfd_batch* b) { return b ? b->launches : 0; }

int cfd_batch_graph_active(const cfd_batch* b) { return b && b->graph_ok ? 1 : 0; }

}  // extern "C"

namespace cfd {

int solve_tile_depth(int mz) { return tz_for(mz); }

int cfd_internal_error(int code, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  std::memcpy(g_last_error, buf, sizeof(buf));
  return code;
}

}  // namespace cfd
