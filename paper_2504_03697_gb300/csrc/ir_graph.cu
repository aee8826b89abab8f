// Mixed-precision pressure solve (FP32 CG with FP64 reliable-update
// refinement, Sec. 3.1's PCG in the precision split of the persistent
// ir_kernel) as one CUDA graph with device-side loops, for large grids.
//
// The method is that of ir_kernel: the FP32 recurrence p = r32 + beta p,
// q = A p, alpha = r32.r32 / p.q, x32 += alpha p, r32 -= alpha q (in the
// plain loop x32 takes these terms two at a time, see below; r32, p and the
// scalars are the same operations in the same order); FP64
// refinement x += x32, r = b - A x whenever |r32|^2 has fallen by delta^2
// since the last refinement (or below the tolerance); the search direction
// is kept across a refinement; convergence only on the FP64 true residual.
// What differs is the execution: instead of one cooperative kernel with two
// grid barriers per iteration, every phase is its own streaming kernel
// (float4 accesses, x neighbours by warp shuffles) and the loop control runs
// on the device.  The FP32 iteration moves 28 B per cell on average: the
// direction kernel reads r32 and the previous p and writes p (forming p on
// the fly at the +x, +y, +z neighbours too, for p.Ap as a sum of squared
// differences over the grid's edges); the update kernel forms q = A p from
// the stored p and reads and writes r32, and x32 every other iteration: one
// iteration defers its term alpha p, the next adds both, the deferred one as
// (alpha_deferred / beta)(p - r) since p - r = beta p_deferred (until then
// the passes that read x32 add the deferred term themselves).  q is never
// stored.
//
//   memset(counter) -> pro_sum -> pro_resid ->
//   while (outer) { prep -> while (inner) { (dir -> upd) x kItersPerPass } -> refine } ->
//   epi_resid -> finish -> shift
//
// `outer` and `inner` are conditional graph nodes of type while.  Each
// kernel reduces its partial sums in FP64 through a last-block pass (blocks
// add their sums to a fixed slot, the block that arrives last sums the slots
// in block order), and that block's thread 0 updates the solver scalars in
// GState and sets the loop conditions; once an update kernel has left the
// inner loop, the kernels after it in the same pass of the body return at
// once.  Nothing waits on another block: the graph's node order is the only
// synchronisation.  Every loop ends: each update raises `iters` by one and
// the outer body stops the loops once iters >= max_iters or refinements >
// max_outer.
//
// The batched form (irb_kernel, below) runs the same passes for many
// independent systems inside one persistent cooperative launch, with the
// loop control in registers and a problem-wide reduction per phase.
//
// Operators: the pressure matrix (float4 kernels, mx % 4 == 0) and the
// velocity matrices of the diffusion substep (float4 kernels on FP32 rows
// padded to a multiple of 4 cells; p.Hp in the edge form too; no mean
// removal, their matrices being nonsingular).
//
// The learned preconditioner (pressure matrix only; the paper's "other
// preconditioners", Sec. 5) enters the same graph in two ways:
//
// * flexible CG (a.flexible): each FP32 iteration applies the U-Net to the
//   recurrence residual, z = U(s r32) (its forward pass captured once as
//   the body of a conditional IF node), and takes the Polak-Ribiere step
//       z~ = z - mean(z),  beta = z~.(r_new - r_old) / (z~.r)_old
//          = -alpha_old z~.(A p_old) / (z~.r)_old,
//       p = z~ + beta p_old,  alpha = z~.r / p.A p,
//   with x32, r32 updated as in CG.  The inner loop body is
//       f_norm -> IF(network) { U-Net } -> f_beta -> f_dir -> f_upd
//   and the outer loop refines in FP64 exactly as above (the direction is
//   kept; beta after a refinement uses the new z and the recurrence form of
//   r_new - r_old).  A breakdown of the network's step (z~.r = 0 or not
//   finite) or `stagnation` iterations without the residual norm halving
//   switch the solve to plain CG (z = r32), restarted along the residual
//   (after a refinement to the true residual on stagnation), all decided
//   on the device.  z~.r < 0 is allowed: alpha is then negative and still
//   the exact line search along p.
// * learned initial guess (a.guess): before the prologue, x0 = alpha z~
//   with z = U(s (b - mean b)), z~ = z - mean(z) and alpha = z~.b / z~.A z~,
//   the x0 along z~ of least energy-norm error; then the solve starts from
//   x0 (its prologue computes r = b - A x0 in FP64).

#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "cfd_common.cuh"
#include "cfd_internal.h"
#include "ir_graph.h"
#include "operator_rows.cuh"
#include "unet.h"

namespace cfd {
namespace {

constexpr int kGThreads = 256;  // every kernel: 256 threads (32 x 8 for the stencils)
// Resident blocks per SM of the FP32 iteration kernels (g_dir, g_upd): with
// 5 (at most 48 registers a thread, no spills) an iteration at 384^3 takes
// 323 us against 334 us with 4 (64 registers); 6 spills.
constexpr int kIterBlocks = 5;
// FP32 iterations per pass of the inner while body (its loop test and node
// launches are paid once per pass; after the loop is left inside a pass the
// remaining kernels of the pass return at once): 4 measured 24.2 against
// 27.5 us per iteration at 128^3 and 329 against 334 us at 384^3.
constexpr int kItersPerPass = 4;
constexpr int kGMax = 1024;     // blocks per kernel (partial-sum slots per value)
// z planes per FP32 stencil work item (2, 8 and 16 measured no faster at
// 384^3; 16 slower)
constexpr int kZ32 = 4;
constexpr int kZ64 = 4;         // z planes per FP64 stencil work item

// Solver scalars of one solve (device memory, written only by the thread 0
// of the last block of a kernel; read by every thread of the next kernels).
struct GState {
  double shift;      // mean of b (removed when remove_mean)
  double bb, rr, rsum;
  double rz, rz_ref, beta, alpha, gshift;
  double tol2, delta2;
  int iters, refinements, status, first, cur, refine, pending, breakdown, done, pad;
  unsigned counter;  // arrivals of the current kernel (atomicInc wraps to 0)
  unsigned pad2;
  long long kernels;  // kernels run by all graph solves of this workspace (never reset)
  DevSolveStats out;  // statistics of the last solve (copied to the caller's slot)
  // flexible CG with the learned preconditioner
  int plain;          // 1 once the solve runs as plain CG (network dropped)
  int since;          // iterations since the residual norm last halved
  int plain_iters;    // iterations run as plain CG
  int skip;           // the flexible direction was unusable: no update, refine
  double best;        // smallest r32.r32 seen (stagnation test)
  double rr32;        // r32.r32 of the current recurrence residual
  double zr;          // z~.r32 of the current direction
  double zmean;       // mean of the current z (removed from it)
  // learned initial guess
  double gmean, gscale, galpha, gzmean;
  // x32 update deferred by one iteration (plain inner loop of the graph
  // form): the update pass of every other iteration leaves x32 alone and
  // records alpha; the next one adds both terms.  Until then every reader of
  // x32 adds xalpha * p (p in buffer xbuf) itself.
  int xdef, xbuf;
  double xalpha;  // alpha of the deferred term
  double xcoef;   // xalpha / beta of the next direction (its p = r + beta p_deferred)
};

constexpr size_t kStateBytes = 512;
constexpr int kPartSlots = 6;  // values one last-block reduction may carry
static_assert(sizeof(GState) <= kStateBytes, "GState slot");

struct GArgs {
  int mx, my, mz;
  size_t n;
  double* x;
  double* b;
  double* r;
  float* r32;
  float* d32;
  float* p0;
  float* p1;
  float* q32;
  int zero_x0, remove_mean, gauge;
  double gauge_value;
  double rtol, delta;
  int max_iters, max_outer;
  GState* S;
  double* part;  // 3 * kGMax doubles
  cudaGraphConditionalHandle h_out, h_in;
  int kind;              // kOp* operator
  double c;              // nu dt / h^2 (velocity operators)
  float c32;
  int pitch;             // row pitch of the FP32 vectors (r32, d32, p0, p1) in cells: mx, or mx rounded up to
                         // a multiple of 4 for a velocity matrix (its padding cells hold 0)
  int lpr;               // float4 lanes: lanes per grid row (4, 8, 16 or 32); a warp covers 32 / lpr rows
  int w32x, w32y, w32z;  // FP32 work items: (float4 or scalar) columns / lpr (32), rows / (8 * 32 / lpr), planes / kZ32
  int w64x, w64y, w64z;  // FP64 work items: columns / 32, rows / 8, planes / kZ64
  // learned preconditioner (pressure matrix, float4 kernels)
  __nv_bfloat16* net_in;  // the network's input plane
  const float* net_out;   // the network's output
  const int* net_err;     // set by a timed-out tensor-core wait of the network
  int net_kernels;        // kernels of one network application
  int stagnation;         // flexible CG: iterations without halving |r| before plain CG
  int gwarm;              // learned guess corrects the starting x (source r = b' - A x) instead of replacing it
  cudaGraphConditionalHandle h_net;
  // batched launch (irb_kernel): the problem's synchronisation words (arrive
  // = reduction counter, pad[0] = reduction generation, error = a block gave
  // up waiting; zero before the launch), where its statistics go, and the
  // limit of one wait
  SolveCtrl* ctrl;
  DevSolveStats* stats;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ int ftid() { return threadIdx.y * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t vtid() { return size_t(blockIdx.x) * kGThreads + ftid(); }
__device__ __forceinline__ size_t vstride() { return size_t(gridDim.x) * kGThreads; }

// The blocks that work on one problem: this block's index among them and
// their count (the whole grid in the graph form; a range of it in the
// batched launch).
struct Blk {
  int bid, nb;
};
__device__ __forceinline__ Blk grid_blk() { return Blk{int(blockIdx.x), int(gridDim.x)}; }

__device__ __forceinline__ void count_kernel(GState* S) {
  if (blockIdx.x == 0 && ftid() == 0) S->kernels += 1;
}

// Block sums of v[] (one shuffle tree per warp, then the warps in order),
// stored in slot B.bid of part; arrival on *counter (atomicInc wraps it back
// to 0 with the last of the B.nb arrivals).  Returns true in every thread of
// the block that arrived last.
template <int K>
__device__ bool arrive_slots(const double (&v)[K], double* part, unsigned* counter, double (&sh)[K][kGThreads / 32],
                             Blk B) {
  __shared__ int s_last;
  const int t = ftid(), lane = t & 31, wid = t >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = v[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[k][wid] = s;
  }
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < kGThreads / 32; ++w) s += sh[k][w];
      part[k * kGMax + B.bid] = s;
    }
    __threadfence();
    s_last = atomicInc(counter, unsigned(B.nb) - 1) == unsigned(B.nb) - 1;
  }
  __syncthreads();
  return s_last != 0;
}

// In the block that arrived last: out[] = the sums over the B.nb slots in
// block order (the same bits for the same partials whatever the schedule),
// in every thread.
template <int K>
__device__ void sum_slots(const double* part, double (&sh)[K][kGThreads / 32], double (&out)[K], Blk B) {
  const int t = ftid(), lane = t & 31, wid = t >> 5;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    acc[k] = 0.0;
    for (unsigned bk = unsigned(t); bk < unsigned(B.nb); bk += kGThreads) acc[k] += __ldcg(part + k * kGMax + bk);
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  }
  __syncthreads();  // thread 0's reads of sh in arrive_slots are complete
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][wid] = acc[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int w = 0; w < kGThreads / 32; ++w) s += sh[k][w];
    out[k] = s;
  }
}

// Block sums of v[], stored in slot blockIdx.x; returns true in every thread
// of the block that arrived last, with out[] = the sums over all slots in
// block order.
template <int K>
__device__ bool reduce_last(const double (&v)[K], double* part, unsigned* counter, double (&out)[K]) {
  __shared__ double sh[K][kGThreads / 32];
  const Blk B = grid_blk();
  if (!arrive_slots<K>(v, part, counter, sh, B)) return false;
  sum_slots<K>(part, sh, out, B);
  return true;
}

// ---------------------------------------------------------------------------
// prologue: sum of b, then r = b' - A x0 with b' = b - mean (in place)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGThreads) g_pro_sum(const GArgs a) {
  count_kernel(a.S);
  double s = 0.0;
  if (a.remove_mean)
    for (size_t e = vtid(); e < a.n; e += vstride()) s += a.b[e];
  double v[1] = {s}, o[1];
  if (!reduce_last<1>(v, a.part, &a.S->counter, o) || ftid() != 0) return;
  GState* S = a.S;
  S->shift = a.remove_mean ? o[0] / double(a.n) : 0.0;
  S->iters = 0;
  S->refinements = 0;
  S->status = kErrNotConverged;
  S->first = 1;
  S->cur = 0;
  S->refine = 0;
  S->pending = 0;
  S->xdef = 0;
  S->breakdown = 0;
  S->done = 0;
  S->beta = 0.0;
  S->rz = 0.0;
  S->plain = 0;
  S->since = 0;
  S->plain_iters = 0;
  S->skip = 0;
  S->best = 0.0;
  S->rr32 = 0.0;
  S->zr = 0.0;
  S->zmean = 0.0;
}

// A deferred x32 term (GState::xdef): p is the deferred direction, nullptr
// when there is none.
struct XDef {
  const float* p = nullptr;
  float alpha = 0.f;
};

// x32 at FP32 cell e32 with a deferred term added, rounded as the update pass
// would have added it.
__device__ __forceinline__ float x32_at(const GArgs& a, const XDef& xd, size_t e32) {
  return xd.p ? fmaf(xd.alpha, xd.p[e32], a.d32[e32]) : a.d32[e32];
}

__device__ __forceinline__ XDef xdef_of(const GArgs& a, const GState* S) {
  XDef xd;
  if (S->xdef) {
    xd.p = S->xbuf ? a.p1 : a.p0;
    xd.alpha = float(S->xalpha);
  }
  return xd;
}

// FP64 residual r = b - A xv over the tiles (scalar lanes, z-marching).
// MODE 0 (prologue): b' = b - shift (stored when remove_mean), xv = x or 0
//   (zero_x0: x := 0); sums b'.b', r.r, sum(r); sets the initial state.
// MODE 1 (refinement, after the inner loop): only when S->refine; xv =
//   x + x32 on the fly (x itself unchanged); sums r.r, sum(r).
// MODE 2 (epilogue): only when b != 0 and the loop ended without
//   convergence; xv = x + x32 if x32 is pending; sums r.r.
// The pass of g_resid64 over the blocks B: r = b' - A xv, with b' = b -
// shift (MODE 0; stored when remove_mean) and xv = 0 (zero), x + x32 (add32)
// or x; s[0] += b'.b' (MODE 0), s[1] += r.r, s[2] += sum(r).
//
// A warp covers 64 consecutive x cells of one row (two per lane, 32 apart),
// z by marching kZ64 planes; the x neighbours come from the neighbouring
// lanes by shuffles (cell 31 / 32 of the row segment across the two halves,
// the segment's ends by loads), so each plane step issues two independent
// cells per lane.  Lanes past the row's end shadow its last cell and store
// nothing.  The operator kind is a template constant.
template <int MODE, int KIND>
__device__ __forceinline__ void resid64_rows(const GArgs& a, double shift, bool add32, bool zero, double (&s)[3],
                                             Blk B, XDef xd) {
  const int mx = a.mx, my = a.my, mz = a.mz;
  const size_t sy = size_t(mx), sz = size_t(mx) * my;
  const size_t py = size_t(a.pitch), pz = size_t(a.pitch) * my;  // the FP32 layout
  auto X = [&](size_t e, size_t e32) { return zero ? 0.0 : (add32 ? a.x[e] + double(x32_at(a, xd, e32)) : a.x[e]); };
  const int lane = threadIdx.x;
  double sb = 0.0, sr = 0.0, ss = 0.0;
  const int wxn = (mx + 63) / 64;
  const int items = wxn * a.w64y * a.w64z;
  for (int w = B.bid; w < items; w += B.nb) {
    const int wx = w % wxn, wy = (w / wxn) % a.w64y, wz = w / (wxn * a.w64y);
    const int j = wy * 8 + threadIdx.y, k0 = wz * kZ64;
    if (j >= my) continue;  // the whole warp (one row per warp)
    const int k1 = min(k0 + kZ64, mz);
    const int ia = wx * 64 + lane, ib = ia + 32;
    const bool va = ia < mx, vb = ib < mx;
    const int iac = va ? ia : mx - 1, ibc = vb ? ib : mx - 1;  // lanes past the row shadow its last cell
    size_t ca = (size_t(k0) * my + j) * mx + iac, cb = (size_t(k0) * my + j) * mx + ibc;
    size_t pa = (size_t(k0) * my + j) * py + iac, pb = (size_t(k0) * my + j) * py + ibc;
    double xca = X(ca, pa), xcb = X(cb, pb);
    double xma = k0 > 0 ? X(ca - sz, pa - pz) : xca, xmb = k0 > 0 ? X(cb - sz, pb - pz) : xcb;
    for (int k = k0; k < k1; ++k, ca += sz, cb += sz, pa += pz, pb += pz) {
      const bool up = k < mz - 1;
      const double xpa = up ? X(ca + sz, pa + pz) : xca, xpb = up ? X(cb + sz, pb + pz) : xcb;
      const double xsa = j > 0 ? X(ca - sy, pa - py) : xca, xsb = j > 0 ? X(cb - sy, pb - py) : xcb;
      const double xna = j < my - 1 ? X(ca + sy, pa + py) : xca, xnb = j < my - 1 ? X(cb + sy, pb + py) : xcb;
      double wa = __shfl_up_sync(0xffffffffu, xca, 1), ea = __shfl_down_sync(0xffffffffu, xca, 1);
      double wb = __shfl_up_sync(0xffffffffu, xcb, 1), eb = __shfl_down_sync(0xffffffffu, xcb, 1);
      const double a31 = __shfl_sync(0xffffffffu, xca, 31), b0 = __shfl_sync(0xffffffffu, xcb, 0);
      if (lane == 0) {
        wa = ia > 0 ? X(ca - 1, pa - 1) : xca;
        wb = a31;
      }
      if (lane == 31) {
        ea = b0;
        eb = ib + 1 < mx ? X(cb + 1, pb + 1) : xcb;
      }
      // a shadow lane holds the row's last cell, so a cell at the row's end
      // sees itself as its east neighbour, as the boundary rule wants
      if (va) {
        const double ax = stencil_row<double>(KIND, a.c, ia, j, k, mx, my, mz, xca, wa, ea, xsa, xna, xma, xpa);
        double bv = a.b[ca];
        if (MODE == 0) {
          bv -= shift;
          if (a.remove_mean) a.b[ca] = bv;
          if (zero) a.x[ca] = 0.0;
          sb = fma(bv, bv, sb);
        }
        const double rv = bv - ax;
        a.r[ca] = rv;
        sr = fma(rv, rv, sr);
        ss += rv;
      }
      if (vb) {
        const double ax = stencil_row<double>(KIND, a.c, ib, j, k, mx, my, mz, xcb, wb, eb, xsb, xnb, xmb, xpb);
        double bv = a.b[cb];
        if (MODE == 0) {
          bv -= shift;
          if (a.remove_mean) a.b[cb] = bv;
          if (zero) a.x[cb] = 0.0;
          sb = fma(bv, bv, sb);
        }
        const double rv = bv - ax;
        a.r[cb] = rv;
        sr = fma(rv, rv, sr);
        ss += rv;
      }
      xma = xca;
      xca = xpa;
      xmb = xcb;
      xcb = xpb;
    }
  }
  s[0] = sb;
  s[1] = sr;
  s[2] = ss;
}

template <int MODE>
__device__ __forceinline__ void resid64_pass(const GArgs& a, double shift, bool add32, bool zero, double (&s)[3],
                                             Blk B, XDef xd = XDef{}) {
  switch (a.kind) {
    case kOpVelU: resid64_rows<MODE, kOpVelU>(a, shift, add32, zero, s, B, xd); break;
    case kOpVelV: resid64_rows<MODE, kOpVelV>(a, shift, add32, zero, s, B, xd); break;
    case kOpVelW: resid64_rows<MODE, kOpVelW>(a, shift, add32, zero, s, B, xd); break;
    default: resid64_rows<MODE, kOpPressure>(a, shift, add32, zero, s, B, xd); break;
  }
}

template <int MODE>
__global__ void __launch_bounds__(kGThreads) g_resid64(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  if (MODE == 1 && !S->refine) {
    if (blockIdx.x == 0 && ftid() == 0) cudaGraphSetConditional(a.h_out, 0u);  // cap or breakdown: leave
    return;
  }
  if (MODE == 2 && (S->bb == 0.0 || S->status == kOk)) return;
  double v[3], o[3];
  resid64_pass<MODE>(a, MODE == 0 ? S->shift : 0.0, MODE == 1 || (MODE == 2 && S->pending), MODE == 0 && a.zero_x0, v,
                     grid_blk(), MODE == 0 ? XDef{} : xdef_of(a, S));
  if (!reduce_last<3>(v, a.part, &S->counter, o) || ftid() != 0) return;
  if (MODE == 0) {
    S->bb = o[0];
    S->rr = o[1];
    S->rsum = o[2];
    S->tol2 = a.rtol * a.rtol * o[0];
    S->delta2 = a.delta * a.delta;
    if (o[0] == 0.0) {
      S->status = kOk;
      S->done = 1;
      S->rr = 0.0;
    }
    cudaGraphSetConditional(a.h_out, o[0] == 0.0 ? 0u : 1u);
  } else if (MODE == 1) {
    S->rr = o[1];
    S->rsum = o[2];
    S->refinements += 1;
    S->refine = 0;
    cudaGraphSetConditional(a.h_out, 1u);
  } else {
    S->rr = o[1];
    if (S->status == kErrNotConverged && o[1] <= S->tol2) S->status = kOk;
  }
}

// Cell e of the FP64 layout in the FP32 layout (row pitch a.pitch; the
// grids hold fewer than 2^31 cells).
__device__ __forceinline__ size_t c32_of(const GArgs& a, size_t e) {
  if (a.pitch == a.mx) return e;
  const unsigned row = unsigned(e) / unsigned(a.mx);
  return e + size_t(row) * size_t(a.pitch - a.mx);
}

// g_prep's pass over the blocks B: fold a pending x32 into x, load r32 =
// r - rmean unless leaving, clear x32; the padding cells of the FP32 rows
// are set to 0.  Returns this thread's part of r32.r32 (FP32).
__device__ __forceinline__ float prep_pass(const GArgs& a, bool fold, bool leave, double rmean, Blk B,
                                           XDef xd = XDef{}) {
  const size_t t0 = size_t(B.bid) * kGThreads + ftid(), st = size_t(B.nb) * kGThreads;
  float f = 0.f;
  for (size_t e = t0; e < a.n; e += st) {
    const size_t e32 = c32_of(a, e);
    if (fold) a.x[e] += double(x32_at(a, xd, e32));
    if (!leave) {
      const float v = float(a.r[e] - rmean);
      a.r32[e32] = v;
      f = fmaf(v, v, f);
    }
    if (fold || !leave) a.d32[e32] = 0.f;
  }
  if (a.pitch != a.mx) {
    const unsigned pad = unsigned(a.pitch - a.mx), rows = unsigned(a.my) * unsigned(a.mz);
    for (size_t q = t0; q < size_t(rows) * pad; q += st) {
      const unsigned row = unsigned(q) / pad, i = unsigned(a.mx) + unsigned(q) - row * pad;
      const size_t e32 = size_t(row) * unsigned(a.pitch) + i;
      a.r32[e32] = 0.f;
      a.d32[e32] = 0.f;
    }
  }
  return f;
}

// g_finish's pass over the blocks B: x := 0 (zero) or x += x32 (fold);
// returns this thread's part of sum(x).
__device__ __forceinline__ double finish_pass(const GArgs& a, bool zero, bool fold, Blk B, XDef xd = XDef{}) {
  const size_t t0 = size_t(B.bid) * kGThreads + ftid(), st = size_t(B.nb) * kGThreads;
  double s = 0.0;
  for (size_t e = t0; e < a.n; e += st) {
    double xv = zero ? 0.0 : a.x[e];
    if (!zero && fold) xv += double(x32_at(a, xd, c32_of(a, e)));
    if (zero || fold) a.x[e] = xv;
    s += xv;
  }
  return s;
}

// ---------------------------------------------------------------------------
// outer body, first node: leave (converged / caps) or start a new FP32
// recurrence from the true residual.  Folds a pending x32 into x either way.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGThreads) g_prep(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  const bool ok = S->rr <= S->tol2;
  const bool leave = ok || S->refinements > a.max_outer || S->iters >= a.max_iters;
  const bool fold = S->pending != 0;
  // the singular pressure system works on zero-mean residuals
  const double rmean = a.kind == kOpPressure ? S->rsum / double(a.n) : 0.0;
  const float f = prep_pass(a, fold, leave, rmean, grid_blk(), xdef_of(a, S));
  double v[1] = {double(f)}, o[1];
  if (!reduce_last<1>(v, a.part, &S->counter, o) || ftid() != 0) return;
  S->pending = 0;
  S->xdef = 0;
  if (leave) {
    if (ok) S->status = kOk;
    S->done = 1;
    cudaGraphSetConditional(a.h_in, 0u);
    return;
  }
  if (!S->first) S->beta = o[0] / S->rz;  // keep the direction across the refinement
  S->rz = o[0];
  S->rz_ref = S->rr;
  cudaGraphSetConditional(a.h_in, 1u);
}

// ---------------------------------------------------------------------------
// The FP32 operator over the work items of this block: for every cell of the
// block's tiles, q = A v with v given by P4 (a float4 of four x-consecutive
// cells) and P1 (one cell); `emit(c4, v, q)` receives the centre values.
// One warp covers 128 x cells of one row; x neighbours by warp shuffles,
// y neighbours by loads, z by marching kZ32 planes in registers.
// ---------------------------------------------------------------------------
// Four x-consecutive rows (cells i0 .. i0 + 3 of row j, plane k) of the
// velocity matrix of component KIND - 1 (the rule of stencil_row, with the
// same operations in the same order): the row and plane conditions are
// decided once for the four cells, the x conditions only where i0 is at a
// wall.  Neighbours outside the array arrive as the cell's own value.
template <int KIND>
__device__ __forceinline__ float4 vel_rows4(float c, int i0, int j, int k, int mx, int my, int mz, const float4& pc,
                                            float west, float east, const float4& ps, const float4& pn,
                                            const float4& pm, const float4& pp) {
  constexpr int comp = KIND - 1;
  const bool jlo = j == 0, jhi = j == my - 1, klo = k == 0, khi = k == mz - 1;
  if ((comp == 1 && (jlo || jhi)) || (comp == 2 && (klo || khi))) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float xc[4] = {pc.x, pc.y, pc.z, pc.w};
  const float s_[4] = {ps.x, ps.y, ps.z, ps.w}, n_[4] = {pn.x, pn.y, pn.z, pn.w};
  const float m_[4] = {pm.x, pm.y, pm.z, pm.w}, p_[4] = {pp.x, pp.y, pp.z, pp.w};
  float q[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int i = i0 + t;
    const float g = -xc[t];
    float xm = t == 0 ? west : xc[t - 1];
    float xp = t == 3 ? east : xc[t + 1];
    if (comp != 0) {
      if (i == 0) xm = g;
      if (i == mx - 1) xp = g;
    }
    const float ym = comp != 1 && jlo ? g : s_[t];
    const float yp = comp != 1 && jhi ? g : n_[t];
    const float zm = comp != 2 && klo ? g : m_[t];
    const float zp = comp != 2 && khi ? g : p_[t];
    const float lap = fmaf(6.f, xc[t], -(((((xm + xp) + ym) + yp) + zm) + zp));
    // padding cells of the FP32 rows (i >= mx) stay 0
    q[t] = (comp == 0 && (i == 0 || i == mx - 1)) || i >= mx ? 0.f : fmaf(c, lap, xc[t]);
  }
  return make_float4(q[0], q[1], q[2], q[3]);
}

template <int KIND, typename F4, typename F1, typename E>
__device__ __forceinline__ void march_f32(const GArgs& a, F4 P4, F1 P1, E emit, Blk B = grid_blk()) {
  const int my = a.my, mz = a.mz, nx4 = a.pitch >> 2;
  const size_t sy4 = size_t(nx4), sz4 = size_t(nx4) * my;
  const int lane = threadIdx.x, L = a.lpr, sl = lane & (L - 1), seg = lane / L, rpw = 32 / L;
  const int items = a.w32x * a.w32y * a.w32z;
  for (int w = B.bid; w < items; w += B.nb) {
    const int wx = w % a.w32x, wy = (w / a.w32x) % a.w32y, wz = w / (a.w32x * a.w32y);
    const int i4 = wx * L + sl, j0 = (wy * 8 + threadIdx.y) * rpw, k0 = wz * kZ32;
    if (j0 >= my) continue;  // the whole warp
    const bool row = j0 + seg < my;
    const int j = row ? j0 + seg : my - 1;  // rows past the grid shadow the last row
    const bool on = row && i4 < nx4;
    const bool has_w = i4 > 0, has_e = i4 + 1 < nx4;
    size_t c4 = (size_t(k0) * my + j) * nx4 + (i4 < nx4 ? i4 : nx4 - 1);  // idle lanes shadow the last column
    float4 pc = P4(c4);
    float4 pm = k0 > 0 ? P4(c4 - sz4) : pc;
#pragma unroll
    for (int kk = 0; kk < kZ32; ++kk) {
      const int k = k0 + kk;
      if (k >= mz) break;
      const float4 pp = k < mz - 1 ? P4(c4 + sz4) : pc;
      const float4 ps = j > 0 ? P4(c4 - sy4) : pc;
      const float4 pn = j < my - 1 ? P4(c4 + sy4) : pc;
      float west = __shfl_up_sync(0xffffffffu, pc.w, 1, L);
      float east = __shfl_down_sync(0xffffffffu, pc.x, 1, L);
      if (sl == 0) west = has_w ? P1(4 * c4 - 1) : pc.x;
      else if (!has_w) west = pc.x;
      if (sl == L - 1) east = has_e ? P1(4 * c4 + 4) : pc.w;
      else if (!has_e) east = pc.w;
      float4 q;
      if (KIND == kOpPressure) {
        q.x = fmaf(6.f, pc.x, -(((((west + pc.y) + ps.x) + pn.x) + pm.x) + pp.x));
        q.y = fmaf(6.f, pc.y, -(((((pc.x + pc.z) + ps.y) + pn.y) + pm.y) + pp.y));
        q.z = fmaf(6.f, pc.z, -(((((pc.y + pc.w) + ps.z) + pn.z) + pm.z) + pp.z));
        q.w = fmaf(6.f, pc.w, -(((((pc.z + east) + ps.w) + pn.w) + pm.w) + pp.w));
      } else {  // velocity rows: wall and ghost rules by the cell's indices
        q = vel_rows4<KIND>(a.c32, 4 * i4, j, k, a.mx, my, mz, pc, west, east, ps, pn, pm, pp);
      }
      if (on) emit(c4, pc, q);
      pm = pc;
      pc = pp;
      c4 += sz4;
    }
  }
}

// The direction pass of the pressure matrix: p = P4(c4) (a float4 of four
// x-consecutive cells; P1 one cell) stored at p4; returns this thread's
// part of p.Ap as the sum over the grid's edges of (p_i - p_j)^2 (the
// Neumann matrix has n_c on the diagonal and -1 per in-box neighbour, so
// p.Ap = sum over neighbour pairs of the squared difference), which needs p
// only at the +x, +y and +z neighbours.  One warp covers 128 x cells of one
// row, +x by warp shuffles.
//
// For a velocity matrix H = I + c L (KIND = kOpVelU + comp) the same pass
// gives p.Hp = sum p_i^2 + c (sum over in-array edges (p_i - p_j)^2 + 2 sum
// over ghost faces p_i^2): a ghost neighbour -p_i adds 2 p_i^2, a wall row
// holds p = 0 (its residual is 0), so an edge to it adds p_i^2; the ghost
// faces are the array's boundary faces across the two tangential axes, and
// x edges to the padding of the FP32 rows are left out.
template <int KIND = kOpPressure, typename F4, typename F1>
__device__ __forceinline__ double edge_pass(const GArgs& a, F4 P4, F1 P1, float4* p4, Blk B = grid_blk()) {
  auto sq = [](float d) { return d * d; };
  const int my = a.my, mz = a.mz, nx4 = a.pitch >> 2;
  const size_t sy4 = size_t(nx4), sz4 = size_t(nx4) * my;
  const int lane = threadIdx.x, L = a.lpr, sl = lane & (L - 1), seg = lane / L, rpw = 32 / L;
  double acc = 0.0;
  const int items = a.w32x * a.w32y * a.w32z;
  for (int w = B.bid; w < items; w += B.nb) {
    const int wx = w % a.w32x, wy = (w / a.w32x) % a.w32y, wz = w / (a.w32x * a.w32y);
    const int i4 = wx * L + sl, j0 = (wy * 8 + threadIdx.y) * rpw, k0 = wz * kZ32;
    if (j0 >= my) continue;  // the whole warp
    const bool row = j0 + seg < my;
    const int j = row ? j0 + seg : my - 1;  // rows past the grid shadow the last row
    const bool on = row && i4 < nx4;
    const bool has_e = i4 + 1 < nx4;
    size_t c4 = (size_t(k0) * my + j) * nx4 + (i4 < nx4 ? i4 : nx4 - 1);  // idle lanes shadow the last column
    float4 pc = P4(c4);
#pragma unroll
    for (int kk = 0; kk < kZ32; ++kk) {
      const int k = k0 + kk;
      if (k >= mz) break;
      const float4 pp = k < mz - 1 ? P4(c4 + sz4) : pc;
      const float4 pn = j < my - 1 ? P4(c4 + sy4) : pc;
      float east = __shfl_down_sync(0xffffffffu, pc.x, 1, L);
      if (sl == L - 1) east = has_e ? P1(4 * c4 + 4) : pc.w;
      else if (!has_e) east = pc.w;
      if (on) {
        p4[c4] = pc;
        if (KIND == kOpPressure) {
          // x edges inside the float4 and to the east cell (0 at the wall),
          // y edges to the next row, z edges to the next plane (0 at walls)
          float e = sq(pc.x - pc.y) + sq(pc.y - pc.z) + sq(pc.z - pc.w) + sq(pc.w - east);
          e += (sq(pc.x - pn.x) + sq(pc.y - pn.y)) + (sq(pc.z - pn.z) + sq(pc.w - pn.w));
          e += (sq(pc.x - pp.x) + sq(pc.y - pp.y)) + (sq(pc.z - pp.z) + sq(pc.w - pp.w));
          acc += double(e);
        } else {
          constexpr int comp = KIND - 1;
          const int i0 = 4 * i4, mx = a.mx;
          const float pv[5] = {pc.x, pc.y, pc.z, pc.w, east};
          float e = 0.f;
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (i0 + t + 1 < mx) e += sq(pv[t] - pv[t + 1]);
          e += (sq(pc.x - pn.x) + sq(pc.y - pn.y)) + (sq(pc.z - pn.z) + sq(pc.w - pn.w));
          e += (sq(pc.x - pp.x) + sq(pc.y - pp.y)) + (sq(pc.z - pp.z) + sq(pc.w - pp.w));
          const float d2 = (pc.x * pc.x + pc.y * pc.y) + (pc.z * pc.z + pc.w * pc.w);
          float gh = 0.f;
          if (comp != 0) {
            if (i0 == 0) gh += pc.x * pc.x;
            const int tl = mx - 1 - i0;  // the cell at the +x face, if in this float4
            if (tl >= 0 && tl < 4) gh += pv[tl] * pv[tl];
          }
          if (comp != 1) gh += (j == 0 ? d2 : 0.f) + (j == my - 1 ? d2 : 0.f);
          if (comp != 2) gh += (k == 0 ? d2 : 0.f) + (k == mz - 1 ? d2 : 0.f);
          acc += double(fmaf(a.c32, fmaf(2.f, gh, e), d2));
        }
      }
      pc = pp;
      c4 += sz4;
    }
  }
  return acc;
}

// alpha = rz / p.Ap, or a breakdown (the last block's thread 0)
__device__ __forceinline__ void set_alpha(GState* S, double num, double pq) {
  if (!(pq > 0.0) || !isfinite(pq)) {
    S->breakdown = 1;
    S->status = kErrBreakdown;
    S->done = 1;
  } else {
    S->alpha = num / pq;
  }
}

// inner body: p = r32 + beta p_old, stored; p.Ap by edge_pass; alpha = rz / p.Ap
__global__ void __launch_bounds__(kGThreads, kIterBlocks) g_dir(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  if (S->refine | S->done | S->breakdown) return;  // the loop was left earlier in this pass of its body
  const bool first = S->first != 0;
  const float beta = float(S->beta);
  const int cur = S->cur;
  float* pnew = cur ? a.p1 : a.p0;
  const float* pold = cur ? a.p0 : a.p1;
  const float4* r4 = reinterpret_cast<const float4*>(a.r32);
  const float4* o4 = reinterpret_cast<const float4*>(pold);
  auto P4 = [&](size_t e) {
    const float4 rv = __ldg(r4 + e);
    if (first) return rv;
    const float4 ov = __ldg(o4 + e);
    return make_float4(fmaf(beta, ov.x, rv.x), fmaf(beta, ov.y, rv.y), fmaf(beta, ov.z, rv.z), fmaf(beta, ov.w, rv.w));
  };
  auto P1 = [&](size_t e) { return first ? __ldg(a.r32 + e) : fmaf(beta, __ldg(pold + e), __ldg(a.r32 + e)); };
  double v[1] = {edge_pass(a, P4, P1, reinterpret_cast<float4*>(pnew))}, o[1];
  if (!reduce_last<1>(v, a.part, &S->counter, o) || ftid() != 0) return;
  set_alpha(S, S->rz, o[0]);
}

// inner body for the velocity matrices on float4 lanes (the FP32 rows padded
// to a multiple of 4): p = r32 + beta p_old, stored; p.Hp by the edge form
// of edge_pass; alpha = rz / p.Hp
template <int KIND>
__global__ void __launch_bounds__(kGThreads, kIterBlocks) g_dir_v(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  if (S->refine | S->done | S->breakdown) return;  // the loop was left earlier in this pass of its body
  const bool first = S->first != 0;
  const float beta = float(S->beta);
  const int cur = S->cur;
  float* pnew = cur ? a.p1 : a.p0;
  const float* pold = cur ? a.p0 : a.p1;
  const float4* r4 = reinterpret_cast<const float4*>(a.r32);
  const float4* o4 = reinterpret_cast<const float4*>(pold);
  auto P4 = [&](size_t e) {
    const float4 rv = __ldg(r4 + e);
    if (first) return rv;
    const float4 ov = __ldg(o4 + e);
    return make_float4(fmaf(beta, ov.x, rv.x), fmaf(beta, ov.y, rv.y), fmaf(beta, ov.z, rv.z), fmaf(beta, ov.w, rv.w));
  };
  auto P1 = [&](size_t e) { return first ? __ldg(a.r32 + e) : fmaf(beta, __ldg(pold + e), __ldg(a.r32 + e)); };
  double v[1] = {edge_pass<KIND>(a, P4, P1, reinterpret_cast<float4*>(pnew))}, o[1];
  if (!reduce_last<1>(v, a.part, &S->counter, o) || ftid() != 0) return;
  set_alpha(S, S->rz, o[0]);
}

// The update pass over the float4 lanes: q = A p again from the stored p
// (pnew), x32 += alpha p, r32 -= alpha q; returns this thread's part of
// |r32|^2.
// NC: p may be read through the non-coherent path (it was written by an
// earlier kernel; false in the batched launch, where other blocks of the
// same launch wrote it).
// XM: 0 updates x32 here; 1 leaves x32 alone (the term alpha p is deferred
// to the next iteration); 2 adds this iteration's term and the deferred one,
// xc (p - r) with xc = alpha_deferred / beta: since p = r + beta p_deferred,
// p - r is beta p_deferred, so no earlier direction is read.  x32 is then
// read and written every other iteration only.
template <int KIND, bool NC = true, int XM = 0>
__device__ __forceinline__ double upd_pass(const GArgs& a, float alpha, const float* pnew, Blk B = grid_blk(),
                                           float xc = 0.f) {
  const float4* p4 = reinterpret_cast<const float4*>(pnew);
  float4* d4 = reinterpret_cast<float4*>(a.d32);
  float4* r4 = reinterpret_cast<float4*>(a.r32);
  auto P4 = [&](size_t e) { return NC ? __ldg(p4 + e) : p4[e]; };
  auto P1 = [&](size_t e) { return NC ? __ldg(pnew + e) : pnew[e]; };
  double acc = 0.0;
  march_f32<KIND>(a, P4, P1, [&](size_t c4, const float4& pv, const float4& qv) {
    float4 rv = r4[c4];
    if (XM != 1) {
      float4 dv = d4[c4];
      dv.x = fmaf(alpha, pv.x, dv.x);
      dv.y = fmaf(alpha, pv.y, dv.y);
      dv.z = fmaf(alpha, pv.z, dv.z);
      dv.w = fmaf(alpha, pv.w, dv.w);
      if (XM == 2) {
        dv.x = fmaf(xc, pv.x - rv.x, dv.x);
        dv.y = fmaf(xc, pv.y - rv.y, dv.y);
        dv.z = fmaf(xc, pv.z - rv.z, dv.z);
        dv.w = fmaf(xc, pv.w - rv.w, dv.w);
      }
      d4[c4] = dv;
    }
    rv.x = fmaf(-alpha, qv.x, rv.x);
    rv.y = fmaf(-alpha, qv.y, rv.y);
    rv.z = fmaf(-alpha, qv.z, rv.z);
    rv.w = fmaf(-alpha, qv.w, rv.w);
    r4[c4] = rv;
    acc += double(fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, rv.w * rv.w))));
  }, B);
  return acc;
}

// inner body: the update pass, then the loop control.  XM = 1 defers this
// iteration's x32 term, XM = 2 adds it and the deferred one (upd_pass); the
// body alternates them, starting with 1, so a pass of the body always begins
// with no deferred term (the outer body folds any into x before the next
// pass) and an XM = 2 kernel runs only right after an XM = 1 kernel of the
// same pass.
template <int KIND, int XM>
__global__ void __launch_bounds__(kGThreads, kIterBlocks) g_upd(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  if (S->breakdown | S->refine | S->done) {
    if (blockIdx.x == 0 && ftid() == 0) cudaGraphSetConditional(a.h_in, 0u);
    return;
  }
  const float* pnew = S->cur ? a.p1 : a.p0;
  static_assert(XM == 1 || XM == 2, "the graph's update kernels defer or apply");
  double v[1] = {upd_pass<KIND, true, XM>(a, float(S->alpha), pnew, grid_blk(), float(S->xcoef))}, o[1];
  if (!reduce_last<1>(v, a.part, &S->counter, o) || ftid() != 0) return;
  const double rz_new = o[0];
  if (XM == 2) {
    S->xdef = 0;
  } else {
    S->xdef = 1;
    S->xbuf = S->cur;
    S->xalpha = S->alpha;
  }
  S->first = 0;
  S->cur ^= 1;
  S->iters += 1;
  S->pending = 1;
  if (rz_new <= S->delta2 * S->rz_ref || rz_new <= S->tol2) {
    S->refine = 1;  // beta of the next direction comes from the replaced residual
    cudaGraphSetConditional(a.h_in, 0u);
    return;
  }
  S->beta = rz_new / S->rz;
  S->rz = rz_new;
  if (S->xdef) S->xcoef = S->xalpha / S->beta;
  if (S->iters >= a.max_iters) {
    S->done = 1;
    cudaGraphSetConditional(a.h_in, 0u);
  } else {
    cudaGraphSetConditional(a.h_in, 1u);
  }
}

// ---------------------------------------------------------------------------
// Scalar-lane march for any operator kind and any width (the batched
// launch's pressure matrices whose width is not a multiple of 4): one thread
// per x cell, x and y neighbours through L1, z by marching.  `emit(c, v, q)`
// returns the FP32 contribution of cell c to the pass's dot product; per
// work item the contributions are summed in FP32, then in FP64.
// ---------------------------------------------------------------------------
template <int KIND, typename F1, typename E>
__device__ __forceinline__ double march_s32(const GArgs& a, F1 P, E emit, Blk B = grid_blk()) {
  const int mx = a.mx, my = a.my, mz = a.mz;
  const size_t sy = size_t(mx), sz = size_t(mx) * my;
  double acc = 0.0;
  const int items = a.w32x * a.w32y * a.w32z;
  for (int w = B.bid; w < items; w += B.nb) {
    const int wx = w % a.w32x, wy = (w / a.w32x) % a.w32y, wz = w / (a.w32x * a.w32y);
    const int i = wx * 32 + threadIdx.x, j = wy * 8 + threadIdx.y, k0 = wz * kZ32;
    if (i >= mx || j >= my) continue;
    size_t c = (size_t(k0) * my + j) * mx + i;
    float xc = P(c);
    float xm = k0 > 0 ? P(c - sz) : xc;
    float part = 0.f;
#pragma unroll
    for (int kk = 0; kk < kZ32; ++kk) {
      const int k = k0 + kk;
      if (k >= mz) break;
      const float xp = k < mz - 1 ? P(c + sz) : xc;
      const float xw = i > 0 ? P(c - 1) : xc;
      const float xe = i < mx - 1 ? P(c + 1) : xc;
      const float xs = j > 0 ? P(c - sy) : xc;
      const float xn = j < my - 1 ? P(c + sy) : xc;
      const float q = stencil_row<float>(KIND, a.c32, i, j, k, mx, my, mz, xc, xw, xe, xs, xn, xm, xp);
      part += emit(c, xc, q);
      xm = xc;
      xc = xp;
      c += sz;
    }
    acc += double(part);
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Flexible CG with the learned preconditioner (pressure matrix, float4
// lanes).  See the file header for the recurrence.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// outer body, first node: as g_prep (leave, or load r32 = r - mean(r) from
// the FP64 true residual, folding a pending x32 into x); records r32.r32 and
// the residual of this refinement; the stagnation reference starts at the
// first pass.
__global__ void __launch_bounds__(kGThreads) f_prep(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  const bool ok = S->rr <= S->tol2;
  const bool leave = ok || S->refinements > a.max_outer || S->iters >= a.max_iters;
  const bool fold = S->pending != 0;
  const double rmean = S->rsum / double(a.n);
  float f = 0.f;
  for (size_t e = vtid(); e < a.n; e += vstride()) {
    if (fold) a.x[e] += double(a.d32[e]);
    if (!leave) {
      const float v = float(a.r[e] - rmean);
      a.r32[e] = v;
      f = fmaf(v, v, f);
    }
    if (fold || !leave) a.d32[e] = 0.f;
  }
  double v[1] = {double(f)}, o[1];
  if (!reduce_last<1>(v, a.part, &S->counter, o) || ftid() != 0) return;
  S->pending = 0;
  if (leave) {
    if (ok) S->status = kOk;
    S->done = 1;
    cudaGraphSetConditional(a.h_in, 0u);
    return;
  }
  S->rr32 = o[0];
  S->rz_ref = S->rr;
  if (S->iters == 0) S->best = o[0];
  cudaGraphSetConditional(a.h_in, 1u);
}

// inner body, first node: the network's input xin = BF16(s r32), s =
// sqrt(V / r32.r32) (unit RMS; the network is linear, so the scale of z
// does not matter to flexible CG), and the IF condition of the network
// node: off once the solve runs as plain CG.
__global__ void __launch_bounds__(kGThreads) f_norm(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  const bool net = S->plain == 0;
  if (blockIdx.x == 0 && ftid() == 0) {
    cudaGraphSetConditional(a.h_net, net ? 1u : 0u);
    if (net) S->kernels += a.net_kernels;
  }
  if (!net) return;
  const float sc = S->rr32 > 0.0 ? float(sqrt(double(a.n) / S->rr32)) : 0.f;
  const float4* r4 = reinterpret_cast<const float4*>(a.r32);
  uint2* x2 = reinterpret_cast<uint2*>(a.net_in);
  for (size_t e = vtid(); e < a.n / 4; e += vstride()) {
    const float4 rv = __ldg(r4 + e);
    x2[e] = make_uint2(bf16x2_bits(rv.x * sc, rv.y * sc), bf16x2_bits(rv.z * sc, rv.w * sc));
  }
}

// inner body, after the network: with z the network's output (r32 once the
// solve runs as plain CG) and q_old = A p_old formed again from the stored
// previous direction: z.r32, z.q_old, sum z, sum r32, sum q_old, r32.r32.
// The last block removes the mean of z and forms z~.r32 and the
// Polak-Ribiere beta = -alpha_old z~.q_old / (z~.r)_old; a breakdown of the
// network's step (z~.r32 = 0 or not finite) switches to plain CG along the
// residual.
__global__ void __launch_bounds__(kGThreads, 4) f_beta(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  const bool plain = S->plain != 0, first = S->first != 0;
  const float4* z4 = reinterpret_cast<const float4*>(plain ? a.r32 : a.net_out);
  const float4* r4 = reinterpret_cast<const float4*>(a.r32);
  const float* pold = S->cur ? a.p0 : a.p1;  // the direction of the last update
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  auto add = [&](const float4& zv, const float4& rv, const float4& qv) {
    acc[0] += double(fmaf(zv.x, rv.x, fmaf(zv.y, rv.y, fmaf(zv.z, rv.z, zv.w * rv.w))));
    acc[1] += double(fmaf(zv.x, qv.x, fmaf(zv.y, qv.y, fmaf(zv.z, qv.z, zv.w * qv.w))));
    acc[2] += double((zv.x + zv.y) + (zv.z + zv.w));
    acc[3] += double((rv.x + rv.y) + (rv.z + rv.w));
    acc[4] += double((qv.x + qv.y) + (qv.z + qv.w));
    acc[5] += double(fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, rv.w * rv.w))));
  };
  if (!first) {
    const float4* o4 = reinterpret_cast<const float4*>(pold);
    auto P4 = [&](size_t e) { return __ldg(o4 + e); };
    auto P1 = [&](size_t e) { return __ldg(pold + e); };
    march_f32<kOpPressure>(a, P4, P1, [&](size_t c4, const float4&, const float4& qv) { add(__ldg(z4 + c4), __ldg(r4 + c4), qv); });
  } else {
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (size_t e = vtid(); e < a.n / 4; e += vstride()) add(__ldg(z4 + e), __ldg(r4 + e), zero);
  }
  double o[6];
  if (!reduce_last<6>(acc, a.part, &S->counter, o) || ftid() != 0) return;
  double m = o[2] / double(a.n);
  double rz = o[0] - m * o[3];
  double zq = o[1] - m * o[4];
  if (!plain && !(rz != 0.0 && isfinite(rz) && isfinite(zq))) {
    S->plain = 1;  // the network's step is unusable: plain CG along r32
    S->first = 1;
    m = o[3] / double(a.n);
    rz = o[5] - m * o[3];
    zq = 0.0;
  }
  if (!(rz != 0.0) || !isfinite(rz)) {
    S->breakdown = 1;
    S->status = kErrBreakdown;
    S->done = 1;
    return;
  }
  S->zmean = m;
  S->beta = S->first ? 0.0 : -S->alpha * zq / S->zr;
  S->zr = rz;
}

// inner body: p = (z - mean z) + beta p_old, stored; p.Ap by edge_pass;
// alpha = z~.r / p.Ap
__global__ void __launch_bounds__(kGThreads, 4) f_dir(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  if (S->breakdown) return;
  const bool first = S->first != 0;
  const float beta = float(S->beta), m = float(S->zmean);
  const float* zsrc = S->plain ? a.r32 : a.net_out;
  const int cur = S->cur;
  float* pnew = cur ? a.p1 : a.p0;
  const float* pold = cur ? a.p0 : a.p1;
  const float4* z4 = reinterpret_cast<const float4*>(zsrc);
  const float4* o4 = reinterpret_cast<const float4*>(pold);
  auto P4 = [&](size_t e) {
    const float4 zv = __ldg(z4 + e);
    const float4 zc = make_float4(zv.x - m, zv.y - m, zv.z - m, zv.w - m);
    if (first) return zc;
    const float4 ov = __ldg(o4 + e);
    return make_float4(fmaf(beta, ov.x, zc.x), fmaf(beta, ov.y, zc.y), fmaf(beta, ov.z, zc.z), fmaf(beta, ov.w, zc.w));
  };
  auto P1 = [&](size_t e) {
    const float zc = __ldg(zsrc + e) - m;
    return first ? zc : fmaf(beta, __ldg(pold + e), zc);
  };
  double v[1] = {edge_pass(a, P4, P1, reinterpret_cast<float4*>(pnew))}, o[1];
  if (!reduce_last<1>(v, a.part, &S->counter, o) || ftid() != 0) return;
  const double pq = o[0];
  if (!S->plain && (!(pq > 0.0) || !isfinite(pq))) {
    S->plain = 1;  // no usable flexible direction: plain CG from the true residual
    S->first = 1;
    S->skip = 1;
    return;
  }
  set_alpha(S, S->zr, pq);
}

// inner body: the update pass, then the loop control of flexible CG:
// refine in FP64 when |r32|^2 fell by delta^2 (or below the tolerance),
// switch to plain CG (after a refinement to the true residual) once the
// residual norm has not halved for `stagnation` iterations, stop at the cap
__global__ void __launch_bounds__(kGThreads, 4) f_upd(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  if (S->breakdown || S->skip) {
    // every block reads the flags before the first block changes them: the
    // last block to pass clears skip (arrival order by the counter)
    __syncthreads();
    if (ftid() == 0) {
      const bool last = atomicInc(&S->counter, gridDim.x - 1) == gridDim.x - 1;
      if (last) {
        if (S->skip) {
          S->skip = 0;
          S->refine = 1;
        }
        cudaGraphSetConditional(a.h_in, 0u);
      }
    }
    return;
  }
  const float* pnew = S->cur ? a.p1 : a.p0;
  double v[1] = {upd_pass<kOpPressure>(a, float(S->alpha), pnew)}, o[1];
  if (!reduce_last<1>(v, a.part, &S->counter, o) || ftid() != 0) return;
  const double rr_new = o[0];
  S->first = 0;
  S->cur ^= 1;
  S->iters += 1;
  if (S->plain) S->plain_iters += 1;
  S->pending = 1;
  S->rr32 = rr_new;
  bool restart = false;
  if (rr_new < 0.25 * S->best) {
    S->best = rr_new;
    S->since = 0;
  } else if (!S->plain && ++S->since >= a.stagnation) {
    S->plain = 1;  // the network stopped helping: plain CG from the true residual
    S->first = 1;
    restart = true;
  }
  if (restart || rr_new <= S->delta2 * S->rz_ref || rr_new <= S->tol2) {
    S->refine = 1;
    cudaGraphSetConditional(a.h_in, 0u);
    return;
  }
  if (S->iters >= a.max_iters) {
    S->done = 1;
    cudaGraphSetConditional(a.h_in, 0u);
  } else {
    cudaGraphSetConditional(a.h_in, 1u);
  }
}

// ---------------------------------------------------------------------------
// Learned initial guess x0 = alpha (z - mean z), z = U(s (b - mean b))
// ---------------------------------------------------------------------------
// sum b, sum b^2 -> mean and the input scale s = sqrt(V / |b - mean|^2)
__global__ void __launch_bounds__(kGThreads) g_gsum(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  double sb = 0.0, sq = 0.0;
  for (size_t e = vtid(); e < a.n; e += vstride()) {
    const double bv = a.b[e];
    sb += bv;
    sq = fma(bv, bv, sq);
  }
  double v[2] = {sb, sq}, o[2];
  if (!reduce_last<2>(v, a.part, &S->counter, o) || ftid() != 0) return;
  const double V = double(a.n), mean = o[0] / V, var = o[1] - mean * o[0];
  S->gmean = mean;
  S->gscale = var > 0.0 && isfinite(var) ? sqrt(V / var) : 0.0;
  S->kernels += a.net_kernels;
}

// warm form: the source of the guess is the residual of the starting x,
// r = (b - mean b) - A x in FP64 (into a.r), and its scale s = sqrt(V / |r|^2)
__global__ void __launch_bounds__(kGThreads) g_gres(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  const Blk B = grid_blk();
  const int mx = a.mx, my = a.my, mz = a.mz;
  const size_t sy = size_t(mx), sz = size_t(mx) * my;
  const double mean = S->gmean;
  double sr = 0.0;
  const int items = a.w64x * a.w64y * a.w64z;
  for (int w = B.bid; w < items; w += B.nb) {
    const int wx = w % a.w64x, wy = (w / a.w64x) % a.w64y, wz = w / (a.w64x * a.w64y);
    const int i = wx * 32 + threadIdx.x, j = wy * 8 + threadIdx.y, k0 = wz * kZ64;
    if (i >= mx || j >= my) continue;
    const int k1 = min(k0 + kZ64, mz);
    size_t c = (size_t(k0) * my + j) * mx + i;
    double xc = a.x[c];
    double xm = k0 > 0 ? a.x[c - sz] : xc;
    for (int k = k0; k < k1; ++k, c += sz) {
      const double xp = k < mz - 1 ? a.x[c + sz] : xc;
      const double xw = i > 0 ? a.x[c - 1] : xc;
      const double xe = i < mx - 1 ? a.x[c + 1] : xc;
      const double xs = j > 0 ? a.x[c - sy] : xc;
      const double xn = j < my - 1 ? a.x[c + sy] : xc;
      const double ax = stencil_row<double>(kOpPressure, 0.0, i, j, k, mx, my, mz, xc, xw, xe, xs, xn, xm, xp);
      const double rv = (a.b[c] - mean) - ax;
      a.r[c] = rv;
      sr = fma(rv, rv, sr);
      xm = xc;
      xc = xp;
    }
  }
  double v[1] = {sr}, o[1];
  if (!reduce_last<1>(v, a.part, &S->counter, o) || ftid() != 0) return;
  S->gmean = 0.0;  // the residual has zero sum (b - mean b is zero-mean, A kills constants)
  S->gscale = o[0] > 0.0 && isfinite(o[0]) ? sqrt(double(a.n) / o[0]) : 0.0;
}

__global__ void __launch_bounds__(kGThreads) g_gnorm(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  const double mean = S->gmean, sc = S->gscale;
  const double* src = a.gwarm ? a.r : a.b;
  uint2* x2 = reinterpret_cast<uint2*>(a.net_in);
  for (size_t e = vtid(); e < a.n / 4; e += vstride()) {
    const size_t c = 4 * e;
    x2[e] = make_uint2(bf16x2_bits(float((src[c] - mean) * sc), float((src[c + 1] - mean) * sc)),
                       bf16x2_bits(float((src[c + 2] - mean) * sc), float((src[c + 3] - mean) * sc)));
  }
}

// sum z, z.(b - mean b), z.A z (FP64; as the sum of squared differences over
// the grid's edges) -> alpha = z~.b / z~.A z~ (0 when the network returns
// nothing usable, so that the solve starts from 0)
__global__ void __launch_bounds__(kGThreads) g_gdots(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  const int mx = a.mx, my = a.my, mz = a.mz;
  const size_t sy = size_t(mx), sz = size_t(mx) * my;
  const double mean = S->gmean;
  const double* src = a.gwarm ? a.r : a.b;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (size_t c = vtid(); c < a.n; c += vstride()) {
    const int i = int(c % sy), j = int((c / sy) % my), k = int(c / sz);
    const double zc = double(a.net_out[c]);
    s0 += zc;
    s1 = fma(zc, src[c] - mean, s1);
    if (i < mx - 1) { const double d = zc - double(a.net_out[c + 1]); s2 = fma(d, d, s2); }
    if (j < my - 1) { const double d = zc - double(a.net_out[c + sy]); s2 = fma(d, d, s2); }
    if (k < mz - 1) { const double d = zc - double(a.net_out[c + sz]); s2 = fma(d, d, s2); }
  }
  double v[3] = {s0, s1, s2}, o[3];
  if (!reduce_last<3>(v, a.part, &S->counter, o) || ftid() != 0) return;
  const double zm = o[0] / double(a.n);
  const double al = o[1] / o[2];  // sum (b - mean b) = 0, so z~.b = z.(b - mean b)
  const bool ok = o[2] > 0.0 && isfinite(al) && !(a.net_err && *a.net_err);
  S->gzmean = ok ? zm : 0.0;
  S->galpha = ok ? al : 0.0;
}

__global__ void __launch_bounds__(kGThreads) g_gset(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  const double al = S->galpha, zm = S->gzmean;
  if (a.gwarm)
    for (size_t e = vtid(); e < a.n; e += vstride()) a.x[e] += al * (double(a.net_out[e]) - zm);
  else
    for (size_t e = vtid(); e < a.n; e += vstride()) a.x[e] = al * (double(a.net_out[e]) - zm);
}

// ---------------------------------------------------------------------------
// epilogue: x = x + pending x32 (0 when b = 0), sum(x) for the gauge; then
// the gauge shift and the statistics
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGThreads) g_finish(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  const double s = finish_pass(a, S->bb == 0.0, S->pending != 0, grid_blk(), xdef_of(a, S));
  double v[1] = {s}, o[1];
  if (!reduce_last<1>(v, a.part, &S->counter, o) || ftid() != 0) return;
  S->pending = 0;
  S->gshift = a.gauge ? a.gauge_value - o[0] / double(a.n) : 0.0;
}

__global__ void __launch_bounds__(kGThreads) g_shift(const GArgs a) {
  GState* S = a.S;
  count_kernel(S);
  if (a.gauge) {
    const double sh = S->gshift;
    for (size_t e = vtid(); e < a.n; e += vstride()) a.x[e] += sh;
  }
  if (blockIdx.x == 0 && ftid() == 0) {
    DevSolveStats* st = &S->out;
    st->iters = S->iters;
    st->outer_iters = S->refinements;
    st->restarts = S->plain_iters;
    st->status = a.net_err && *a.net_err ? kErrTimeout : S->status;
    st->b_norm = sqrt(S->bb);
    st->rel_resid = S->bb > 0.0 ? sqrt(S->rr / S->bb) : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Batched form: many independent systems (the cavities of a batch, one
// operator kind per launch) in one persistent cooperative launch.  Problem
// k owns the blocks [starts[k], starts[k+1]) and runs the whole solve of
// the graph form on them: the same passes (float4 lanes where the grid's
// width is a multiple of 4, scalar lanes otherwise), the same FP32
// recurrence, refinement rule and gauge, with the loop control in registers
// (every block of a problem holds the same bits) and a problem-wide
// reduction (reduce_all) wherever the graph form ends a kernel.  Problems
// never wait on each other.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait (thread 0) until the problem's reduction generation reaches
// `target`.  Gives up, recording CFD_ERR_TIMEOUT in ctrl->error, once
// timeout_ns have passed (checked on the first unsatisfied poll and every 64
// polls after it, so a limit of 0 gives up at once), and also when another
// block of the problem has given up.
__device__ bool wait_gen(SolveCtrl* ctrl, unsigned target, unsigned long long timeout_ns) {
  const unsigned* gen = reinterpret_cast<const unsigned*>(&ctrl->pad[0]);
  const unsigned long long t0 = global_ns();
  unsigned polls = 0;
  while (int(ld_acquire_gpu(gen) - target) < 0) {
    if ((polls++ & 63u) == 0) {
      if (ld_volatile_s32(&ctrl->error) != 0) return false;
      if (global_ns() - t0 >= timeout_ns) {
        atomicCAS(&ctrl->error, 0, kErrTimeout);
        return false;
      }
    }
  }
  return true;
}

// Problem-wide form of reduce_last: the same slots and summation order, but
// every block of the problem obtains the totals.  The block that arrives
// last sums the slots, stores the totals beside them and raises the
// generation to `target` with a release; the others wait for it (acquire)
// and read the totals.  Because no block enters the next reduction before
// the generation is raised, the slots and totals are never overwritten
// while still being read, and every store a block made before arriving is
// visible to every block after the reduction.  Returns false (in every
// thread of the block) when the wait gave up.
template <int K>
__device__ bool reduce_all(const double (&v)[K], const GArgs& a, unsigned target, double (&out)[K], Blk B) {
  __shared__ double sh[K][kGThreads / 32];
  __shared__ int s_ok;
  double* tot = a.part + size_t(kPartSlots - 1) * kGMax;  // totals: the last slot row (K < kPartSlots)
  if (arrive_slots<K>(v, a.part, &a.ctrl->arrive, sh, B)) {
    sum_slots<K>(a.part, sh, out, B);
    if (ftid() == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) tot[k] = out[k];
      st_release_gpu(reinterpret_cast<unsigned*>(&a.ctrl->pad[0]), target);
    }
    __syncthreads();  // every thread has read sh before the next reduction writes it
    return true;
  }
  if (ftid() == 0) s_ok = wait_gen(a.ctrl, target, a.timeout_ns) ? 1 : 0;
  __syncthreads();
  if (!s_ok) return false;
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = __ldcg(tot + k);
  return true;
}

// resident blocks per SM of the batched kernel (3 measured slower: the
// streaming passes want the warps more than the registers)
constexpr int kBatchBlocks = 4;


template <int KIND>
__global__ void __launch_bounds__(kGThreads, kBatchBlocks) irb_kernel(const GArgs* __restrict__ tab,
                                                           const int* __restrict__ starts, int nprob) {
  int lo = 0, hi = nprob - 1;
  const int blk = int(blockIdx.x);
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const GArgs& a = tab[lo];
  const Blk B{blk - starts[lo], starts[lo + 1] - starts[lo]};
  const bool vec = a.pitch % 4 == 0;
  const double n = double(a.n);
  unsigned gen = 0;
  bool ok_sync = true;
  auto all = [&](auto& v, auto& o) {
    ok_sync = ok_sync && reduce_all(v, a, ++gen, o, B);
    return ok_sync;
  };

  // prologue: mean of b, then r = b' - A x0 (g_pro_sum, g_resid64<0>)
  double shift = 0.0;
  if (a.remove_mean) {
    double s1[1] = {0.0}, o1[1];
    for (size_t e = size_t(B.bid) * kGThreads + ftid(); e < a.n; e += size_t(B.nb) * kGThreads) s1[0] += a.b[e];
    if (!all(s1, o1)) goto out;
    shift = o1[0] / n;
  }
  {
    double v3[3], o3[3];
    resid64_pass<0>(a, shift, false, a.zero_x0 != 0, v3, B);
    if (!all(v3, o3)) goto out;
    const double bb = o3[0];
    double rr = o3[1], rsum = o3[2];
    const double tol2 = a.rtol * a.rtol * bb, delta2 = a.delta * a.delta;
    int status = kErrNotConverged, iters = 0, refinements = 0;
    bool pending = false, first = true;
    int cur = 0;
    double rz = 0.0, beta = 0.0;
    if (bb == 0.0) {
      status = kOk;
      rr = 0.0;
    } else {
      for (;;) {
        // outer pass (g_prep): fold x32, load r32 = r - mean(r) unless leaving
        const bool okr = rr <= tol2;
        const bool leave = okr || refinements > a.max_outer || iters >= a.max_iters;
        const bool fold = pending;
        const double rmean = a.kind == kOpPressure ? rsum / n : 0.0;
        double v1[1] = {double(prep_pass(a, fold, leave, rmean, B))}, o1[1];
        if (!all(v1, o1)) goto out;
        pending = false;
        if (leave) {
          if (okr) status = kOk;
          break;
        }
        if (!first) beta = o1[0] / rz;  // keep the direction across the refinement
        rz = o1[0];
        const double rz_ref = rr;
        // inner loop (g_dir / g_upd, or their velocity and scalar forms)
        bool refine = false, broke = false;
        for (;;) {
          float* pnew = cur ? a.p1 : a.p0;
          const float* pold = cur ? a.p0 : a.p1;
          const float b32 = float(beta);
          const bool fst = first;
          double vd[1], od[1];
          if (vec) {
            const float4* r4 = reinterpret_cast<const float4*>(a.r32);
            const float4* o4 = reinterpret_cast<const float4*>(pold);
            auto P4 = [&](size_t e) {
              const float4 rv = r4[e];
              if (fst) return rv;
              const float4 ov = o4[e];
              return make_float4(fmaf(b32, ov.x, rv.x), fmaf(b32, ov.y, rv.y), fmaf(b32, ov.z, rv.z),
                                 fmaf(b32, ov.w, rv.w));
            };
            auto P1 = [&](size_t e) { return fst ? a.r32[e] : fmaf(b32, pold[e], a.r32[e]); };
            vd[0] = edge_pass<KIND>(a, P4, P1, reinterpret_cast<float4*>(pnew), B);
          } else {
            auto P = [&](size_t e) { return fst ? a.r32[e] : fmaf(b32, pold[e], a.r32[e]); };
            vd[0] = march_s32<KIND>(a, P, [&](size_t c, float pc, float q) {
              pnew[c] = pc;
              return pc * q;
            }, B);
          }
          if (!all(vd, od)) goto out;
          if (!(od[0] > 0.0) || !isfinite(od[0])) {
            broke = true;
            break;
          }
          const double alpha = rz / od[0];
          double vu[1], ou[1];
          if (vec) {
            vu[0] = upd_pass<KIND, false>(a, float(alpha), pnew, B);
          } else {
            const float al = float(alpha);
            vu[0] = march_s32<KIND>(a, [&](size_t e) { return pnew[e]; }, [&](size_t c, float pc, float q) {
              a.d32[c] = fmaf(al, pc, a.d32[c]);
              const float rv = fmaf(-al, q, a.r32[c]);
              a.r32[c] = rv;
              return rv * rv;
            }, B);
          }
          if (!all(vu, ou)) goto out;
          const double rz_new = ou[0];
          first = false;
          cur ^= 1;
          iters += 1;
          pending = true;
          if (rz_new <= delta2 * rz_ref || rz_new <= tol2) {
            refine = true;  // beta of the next direction comes from the replaced residual
            break;
          }
          beta = rz_new / rz;
          rz = rz_new;
          if (iters >= a.max_iters) break;
        }
        if (broke) status = kErrBreakdown;
        if (!refine) break;
        // refinement (g_resid64<1>): r = b - A (x + x32)
        resid64_pass<1>(a, 0.0, true, false, v3, B);
        if (!all(v3, o3)) goto out;
        rr = o3[1];
        rsum = o3[2];
        refinements += 1;
      }
      // epilogue (g_resid64<2>)
      if (status != kOk) {
        resid64_pass<2>(a, 0.0, pending, false, v3, B);
        if (!all(v3, o3)) goto out;
        rr = o3[1];
        if (status == kErrNotConverged && rr <= tol2) status = kOk;
      }
    }
    // g_finish: fold x32 (x := 0 when b = 0), mean of x for the gauge
    {
      double s1[1] = {finish_pass(a, bb == 0.0, pending, B)}, o1[1];
      if (!all(s1, o1)) goto out;
      // g_shift
      if (a.gauge) {
        const double sh = a.gauge_value - o1[0] / n;
        for (size_t e = size_t(B.bid) * kGThreads + ftid(); e < a.n; e += size_t(B.nb) * kGThreads) a.x[e] += sh;
      }
      // every block has finished its part of the solve before the statistics
      // are written
      double z1[1] = {0.0}, zo[1];
      if (!all(z1, zo)) goto out;
    }
    if (B.bid == 0 && ftid() == 0) {
      DevSolveStats* st = a.stats;
      st->iters = iters;
      st->outer_iters = refinements;
      st->restarts = 0;
      st->status = status;
      st->b_norm = sqrt(bb);
      st->rel_resid = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    return;
  }
out:
  // a wait gave up (this or another block of the problem): the solve ends
  // with CFD_ERR_TIMEOUT, x holds what the passes left
  if (B.bid == 0 && ftid() == 0) a.stats->status = kErrTimeout;
}

// One resident wave of `kernel`, at most kGMax blocks and `work` items.
template <typename K>
int wave_blocks(K kernel, size_t work) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kGThreads, 0);
  size_t b = size_t(sms > 0 ? sms : 1) * size_t(per_sm > 0 ? per_sm : 1);
  if (b > size_t(kGMax)) b = kGMax;
  if (b > work) b = work;
  return int(b < 1 ? 1 : b);
}

bool same_args(const IrArgs& x, const IrArgs& y) {
  return x.g.mx == y.g.mx && x.g.my == y.g.my && x.g.mz == y.g.mz && x.x == y.x && x.b == y.b && x.r == y.r &&
         x.r32 == y.r32 && x.d32 == y.d32 && x.p0_32 == y.p0_32 && x.p1_32 == y.p1_32 && x.q32 == y.q32 &&
         x.zero_x0 == y.zero_x0 && x.remove_mean == y.remove_mean && x.gauge == y.gauge &&
         x.gauge_value == y.gauge_value && x.rtol == y.rtol && x.delta == y.delta && x.max_iters == y.max_iters &&
         x.max_outer == y.max_outer && x.kind == y.kind && x.c == y.c && x.net == y.net &&
         x.net_mode == y.net_mode && x.flexible == y.flexible && x.guess == y.guess && x.stagnation == y.stagnation &&
         x.guess_warm == y.guess_warm;
}

}  // namespace

struct IrGraph {
  cudaGraph_t graph = nullptr;
  cudaGraph_t net = nullptr;  // the captured network (child of the guess prefix)
  cudaGraphExec_t exec = nullptr;
  IrArgs key{};
  GState* state = nullptr;
};

size_t ir_graph_state_bytes() { return kStateBytes + size_t(kPartSlots) * kGMax * sizeof(double); }

bool ir_graph_eligible(const IrArgs& a) {
  if (a.net && (a.flexible || a.guess)) return a.kind == kOpPressure && a.g.mx % 4 == 0 && a.g.mx >= 4;
  return a.kind != kOpPressure || (a.g.mx % 4 == 0 && a.g.mx >= 4);
}

namespace {
// float4 lanes: the pressure matrix on rows of a multiple of 4 cells; the
// velocity matrices always (their FP32 rows are padded to a multiple of 4)
bool use_vec_kernels(const IrArgs& a) { return a.kind != kOpPressure || a.g.mx % 4 == 0; }

int fp32_pitch(const IrArgs& a) { return a.kind == kOpPressure || a.g.mx % 4 == 0 ? a.g.mx : (a.g.mx + 3) / 4 * 4; }
}  // namespace

size_t ir_fp32_vector_cells(int nx, int ny, int nz) {
  size_t best = size_t(nx) * ny * nz;
  for (int c = 0; c < 3; ++c) {
    IrArgs a{};
    a.kind = kOpVelU + c;
    a.g = GridDims{nx + (c == 0), ny + (c == 1), nz + (c == 2)};
    const size_t cells = size_t(fp32_pitch(a)) * a.g.my * a.g.mz;
    best = best > cells ? best : cells;
  }
  return best;
}


namespace {

cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* dep, void* fn, int blocks,
                       dim3 block, GArgs* args) {
  cudaKernelNodeParams kp{};
  kp.func = fn;
  kp.gridDim = dim3(unsigned(blocks));
  kp.blockDim = block;
  kp.sharedMemBytes = 0;
  void* params[1] = {args};
  kp.kernelParams = params;
  kp.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, dep, dep ? 1 : 0, &kp);
}

cudaError_t add_cond(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* dep, cudaGraphConditionalHandle h,
                     cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaError_t e = cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &np);
  if (e == cudaSuccess) *body = np.conditional.phGraph_out[0];
  return e;
}

cudaError_t add_while(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* dep,
                      cudaGraphConditionalHandle h, cudaGraph_t* body) {
  return add_cond(g, node, dep, h, cudaGraphCondTypeWhile, body);
}

// Capture the U-Net's forward pass (kernel launches only) into graph g.
cudaError_t capture_net(cfd_unet* net, cudaGraph_t g, int* kernels) {
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  int rc = CFD_OK;
  if (e == cudaSuccess) {
    rc = unet_forward_on(net, cs, kernels);
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &out);
    if (e2 != cudaSuccess) e = e2;
  }
  cudaStreamDestroy(cs);
  if (e == cudaSuccess && rc != CFD_OK) e = cudaErrorInvalidValue;
  return e;
}

GArgs make_args(const IrArgs& ia, void* state_buf);
cudaError_t build_graph(IrGraph* G, const IrArgs& ia, GArgs a, bool vec, size_t items32, size_t items64,
                        size_t vec_work, dim3 tile, dim3 flat, bool flexible, bool guess);

cudaError_t build(IrGraph* G, const IrArgs& ia, void* state_buf) {
  GArgs a = make_args(ia, state_buf);
  const bool vec = use_vec_kernels(ia);
  const size_t items32 = size_t(a.w32x) * a.w32y * a.w32z;
  const size_t items64 = size_t(a.w64x) * a.w64y * a.w64z;
  const size_t vec_work = (a.n / 4 + kGThreads - 1) / kGThreads;
  const dim3 tile(32, 8), flat(kGThreads);
  const bool flexible = ia.net && ia.flexible, guess = ia.net && ia.guess;
  if (flexible || guess) {
    UNetView nv{};
    if (!vec || a.kind != kOpPressure || !unet_view(ia.net, &nv) || nv.nx != a.mx || nv.ny != a.my || nv.nz != a.mz)
      return cudaErrorInvalidValue;
    a.net_in = nv.xin;
    a.net_out = nv.z;
    a.net_err = nv.err;
    a.stagnation = ia.stagnation > 0 ? ia.stagnation : 50;
    a.gwarm = guess && ia.guess_warm ? 1 : 0;
  }
  return build_graph(G, ia, a, vec, items32, items64, vec_work, tile, flat, flexible, guess);
}

GArgs make_args(const IrArgs& ia, void* state_buf) {
  GArgs a{};
  a.mx = ia.g.mx;
  a.my = ia.g.my;
  a.mz = ia.g.mz;
  a.n = size_t(a.mx) * a.my * a.mz;
  a.x = ia.x;
  a.b = ia.b;
  a.r = ia.r;
  a.r32 = ia.r32;
  a.d32 = ia.d32;
  a.p0 = ia.p0_32;
  a.p1 = ia.p1_32;
  a.q32 = ia.q32;
  a.zero_x0 = ia.zero_x0;
  a.remove_mean = ia.remove_mean;
  a.gauge = ia.gauge;
  a.gauge_value = ia.gauge_value;
  a.rtol = ia.rtol;
  a.delta = ia.delta;
  a.max_iters = ia.max_iters;
  a.max_outer = ia.max_outer;
  a.S = static_cast<GState*>(state_buf);
  a.part = reinterpret_cast<double*>(static_cast<char*>(state_buf) + kStateBytes);
  a.kind = ia.kind;
  a.c = ia.c;
  a.c32 = float(ia.c);
  const bool vec = use_vec_kernels(ia);
  a.pitch = fp32_pitch(ia);
  a.lpr = 32;
  a.w32x = vec ? (a.pitch / 4 + 31) / 32 : (a.mx + 31) / 32;
  a.w32y = (a.my + 7) / 8;
  a.w32z = (a.mz + kZ32 - 1) / kZ32;
  a.w64x = (a.mx + 31) / 32;
  a.w64y = a.w32y;
  a.w64z = (a.mz + kZ64 - 1) / kZ64;
  return a;
}

cudaError_t build_graph(IrGraph* G, const IrArgs& ia, GArgs a, bool vec, size_t items32, size_t items64,
                        size_t vec_work, dim3 tile, dim3 flat, bool flexible, bool guess) {
  cudaGraph_t top = nullptr;
  cudaError_t e = cudaGraphCreate(&top, 0);
  if (e != cudaSuccess) return e;
  G->graph = top;
  // the network's forward pass on its own (the kernel count goes into the
  // arguments of the nodes that account for it)
  cudaGraph_t netg = nullptr;
  if (flexible || guess) {
    if ((e = cudaGraphCreate(&netg, 0)) != cudaSuccess) return e;
    G->net = netg;
    if ((e = capture_net(ia.net, netg, &a.net_kernels)) != cudaSuccess) return e;
  }
  if ((e = cudaGraphConditionalHandleCreate(&a.h_out, top, 0u, cudaGraphCondAssignDefault)) != cudaSuccess) return e;

  cudaGraphNode_t n0, n1, n2, n3, n4, n5, n6;
  cudaMemsetParams mp{};
  mp.dst = &a.S->counter;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = 1;
  mp.height = 1;
  if ((e = cudaGraphAddMemsetNode(&n0, top, nullptr, 0, &mp)) != cudaSuccess) return e;
  cudaGraphNode_t pre = n0;
  if (guess) {  // x0 = alpha (z - mean z), z = U(s (b - mean b)); warm: x0 = x + alpha z~, z = U(s r)
    cudaGraphNode_t g1, g1r, g2, g3, g4, g5;
    if ((e = add_kernel(top, &g1, &pre, (void*)g_gsum, wave_blocks(g_gsum, vec_work), flat, &a)) != cudaSuccess)
      return e;
    if (a.gwarm) {
      if ((e = add_kernel(top, &g1r, &g1, (void*)g_gres, wave_blocks(g_gres, size_t(a.w64x) * a.w64y * a.w64z),
                          dim3(32, 8), &a)) != cudaSuccess)
        return e;
      g1 = g1r;
    }
    if ((e = add_kernel(top, &g2, &g1, (void*)g_gnorm, wave_blocks(g_gnorm, vec_work), flat, &a)) != cudaSuccess)
      return e;
    if ((e = cudaGraphAddChildGraphNode(&g3, top, &g2, 1, netg)) != cudaSuccess) return e;
    if ((e = add_kernel(top, &g4, &g3, (void*)g_gdots, wave_blocks(g_gdots, vec_work * 4), flat, &a)) != cudaSuccess)
      return e;
    if ((e = add_kernel(top, &g5, &g4, (void*)g_gset, wave_blocks(g_gset, vec_work * 4), flat, &a)) != cudaSuccess)
      return e;
    pre = g5;
  }
  if ((e = add_kernel(top, &n1, &pre, (void*)g_pro_sum, wave_blocks(g_pro_sum, vec_work), flat, &a)) != cudaSuccess)
    return e;
  if ((e = add_kernel(top, &n2, &n1, (void*)g_resid64<0>, wave_blocks(g_resid64<0>, items64), tile, &a)) !=
      cudaSuccess)
    return e;
  cudaGraph_t outer = nullptr, inner = nullptr;
  if ((e = add_while(top, &n3, &n2, a.h_out, &outer)) != cudaSuccess) return e;
  if ((e = cudaGraphConditionalHandleCreate(&a.h_in, outer, 0u, 0u)) != cudaSuccess) return e;
  cudaGraphNode_t b1, b2, b3, i1, i2;
  void* prep = flexible ? (void*)f_prep : (void*)g_prep;
  if ((e = add_kernel(outer, &b1, nullptr, prep, flexible ? wave_blocks(f_prep, vec_work) : wave_blocks(g_prep, vec_work),
                      flat, &a)) != cudaSuccess)
    return e;
  if ((e = add_while(outer, &b2, &b1, a.h_in, &inner)) != cudaSuccess) return e;
  if (flexible) {
    // f_norm -> IF(network) { U-Net } -> f_beta -> f_dir -> f_upd
    if ((e = cudaGraphConditionalHandleCreate(&a.h_net, inner, 0u, 0u)) != cudaSuccess) return e;
    cudaGraphNode_t f1, f2, f3, f4, f5;
    cudaGraph_t netbody = nullptr;
    if ((e = add_kernel(inner, &f1, nullptr, (void*)f_norm, wave_blocks(f_norm, vec_work), flat, &a)) != cudaSuccess)
      return e;
    if ((e = add_cond(inner, &f2, &f1, a.h_net, cudaGraphCondTypeIf, &netbody)) != cudaSuccess) return e;
    if ((e = capture_net(ia.net, netbody, nullptr)) != cudaSuccess) return e;
    if ((e = add_kernel(inner, &f3, &f2, (void*)f_beta, wave_blocks(f_beta, items32), tile, &a)) != cudaSuccess)
      return e;
    if ((e = add_kernel(inner, &f4, &f3, (void*)f_dir, wave_blocks(f_dir, items32), tile, &a)) != cudaSuccess)
      return e;
    if ((e = add_kernel(inner, &f5, &f4, (void*)f_upd, wave_blocks(f_upd, items32), tile, &a)) != cudaSuccess)
      return e;
  } else {
    // (dir -> upd) x kItersPerPass, the update kernels alternating between
    // deferring and applying the x32 term; the velocity matrices have one
    // instantiation per component
    static_assert(kItersPerPass % 2 == 0, "the update kernels of a pass come in defer / apply pairs");
    void* fd = nullptr;
    void* fu[2] = {nullptr, nullptr};
    int nd = 1, nu[2] = {1, 1};
    auto pick = [&](auto dir, auto upd_defer, auto upd_apply) {
      fd = (void*)dir;
      fu[0] = (void*)upd_defer;
      fu[1] = (void*)upd_apply;
      nd = wave_blocks(dir, items32);
      nu[0] = wave_blocks(upd_defer, items32);
      nu[1] = wave_blocks(upd_apply, items32);
    };
    if (vec && a.kind == kOpPressure) pick(g_dir, g_upd<kOpPressure, 1>, g_upd<kOpPressure, 2>);
    else if (a.kind == kOpVelU) pick(g_dir_v<kOpVelU>, g_upd<kOpVelU, 1>, g_upd<kOpVelU, 2>);
    else if (a.kind == kOpVelV) pick(g_dir_v<kOpVelV>, g_upd<kOpVelV, 1>, g_upd<kOpVelV, 2>);
    else pick(g_dir_v<kOpVelW>, g_upd<kOpVelW, 1>, g_upd<kOpVelW, 2>);
    cudaGraphNode_t prev = nullptr;
    for (int it = 0; it < kItersPerPass; ++it) {
      if ((e = add_kernel(inner, &i1, prev ? &prev : nullptr, fd, nd, tile, &a)) != cudaSuccess) return e;
      if ((e = add_kernel(inner, &i2, &i1, fu[it % 2], nu[it % 2], tile, &a)) != cudaSuccess) return e;
      prev = i2;
    }
  }
  if ((e = add_kernel(outer, &b3, &b2, (void*)g_resid64<1>, wave_blocks(g_resid64<1>, items64), tile, &a)) !=
      cudaSuccess)
    return e;
  if ((e = add_kernel(top, &n4, &n3, (void*)g_resid64<2>, wave_blocks(g_resid64<2>, items64), tile, &a)) !=
      cudaSuccess)
    return e;
  if ((e = add_kernel(top, &n5, &n4, (void*)g_finish, wave_blocks(g_finish, vec_work), flat, &a)) != cudaSuccess)
    return e;
  if ((e = add_kernel(top, &n6, &n5, (void*)g_shift, wave_blocks(g_shift, vec_work), flat, &a)) != cudaSuccess)
    return e;
  return cudaGraphInstantiate(&G->exec, top, 0);
}

void release(IrGraph* G) {
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->graph) cudaGraphDestroy(G->graph);
  if (G->net) cudaGraphDestroy(G->net);
  G->exec = nullptr;
  G->graph = nullptr;
  G->net = nullptr;
}

}  // namespace

void destroy_ir_graph(IrGraph* G) {
  if (!G) return;
  release(G);
  delete G;
}

cudaError_t launch_ir_graph(const IrArgs& a, void* state_buf, IrGraph** cache, cudaStream_t s) {
  IrGraph* G = *cache;
  if (!G) {
    G = new IrGraph();
    *cache = G;
  }
  if (!G->exec || !same_args(G->key, a) || G->state != state_buf) {
    release(G);
    const cudaError_t e = build(G, a, state_buf);
    if (e != cudaSuccess) {
      release(G);
      return e;
    }
    G->key = a;
    G->state = static_cast<GState*>(state_buf);
  }
  cudaError_t e = cudaGraphLaunch(G->exec, s);
  // the graph writes its statistics to a fixed slot, so that the caller's
  // per-step slot does not force a new graph
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(a.stats, &G->state->out, sizeof(DevSolveStats), cudaMemcpyDeviceToDevice, s);
  return e;
}

cudaError_t launch_learned_guess(const IrArgs& ia, void* state_buf, cudaStream_t s, int64_t* launches) {
  GArgs a = make_args(ia, state_buf);
  UNetView nv{};
  if (!ia.net || a.kind != kOpPressure || a.mx % 4 != 0 || !unet_view(ia.net, &nv) || nv.nx != a.mx ||
      nv.ny != a.my || nv.nz != a.mz)
    return cudaErrorInvalidValue;
  a.net_in = nv.xin;
  a.net_out = nv.z;
  a.net_err = nv.err;
  const size_t vec_work = (a.n / 4 + kGThreads - 1) / kGThreads;
  cudaError_t e = cudaMemsetAsync(&a.S->counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  g_gsum<<<wave_blocks(g_gsum, vec_work), kGThreads, 0, s>>>(a);
  g_gnorm<<<wave_blocks(g_gnorm, vec_work), kGThreads, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int nk = 0;
  if (unet_forward_on(ia.net, s, &nk) != CFD_OK) return cudaErrorLaunchFailure;
  g_gdots<<<wave_blocks(g_gdots, vec_work * 4), kGThreads, 0, s>>>(a);
  g_gset<<<wave_blocks(g_gset, vec_work * 4), kGThreads, 0, s>>>(a);
  if (launches) *launches += nk;  // the four guess kernels count themselves on the device
  return cudaGetLastError();
}

namespace {
// Batched launch, float4 lanes: as many lanes per row as the row needs
// (a power of two from 4 to 32), so that narrow grids keep every lane busy
// and the blocks of a problem march through fewer (row, plane) steps.
void set_batch_lanes(GArgs& g) {
  if (g.pitch % 4 != 0) return;  // scalar lanes
  const int nx4 = g.pitch / 4;
  int L = 4;
  while (L < nx4 && L < 32) L *= 2;
  g.lpr = L;
  g.w32x = (nx4 + L - 1) / L;
  const int rows = 8 * (32 / L);
  g.w32y = (g.my + rows - 1) / rows;
}
}  // namespace

void ir_batch_work(const IrArgs& ia, int* items, int* extent) {
  GArgs g{};
  g.mx = ia.g.mx;
  g.my = ia.g.my;
  g.mz = ia.g.mz;
  g.pitch = fp32_pitch(ia);
  g.w32x = (g.mx + 31) / 32;  // scalar lanes
  g.w32y = (g.my + 7) / 8;
  g.w32z = (g.mz + kZ32 - 1) / kZ32;
  set_batch_lanes(g);
  *items = g.w32x * g.w32y * g.w32z;
  *extent = ia.g.mx > ia.g.my ? (ia.g.mx > ia.g.mz ? ia.g.mx : ia.g.mz) : (ia.g.my > ia.g.mz ? ia.g.my : ia.g.mz);
}

size_t ir_batch_table_bytes(int nprob) { return sizeof(GArgs) * size_t(nprob > 0 ? nprob : 0); }

cudaError_t ir_batch_table(const IrArgs* args, void* const* states, int nprob, void* d_table, cudaStream_t s) {
  std::vector<GArgs> t(size_t(nprob > 0 ? nprob : 0));
  for (int k = 0; k < nprob; ++k) {
    GArgs g = make_args(args[k], states[k]);
    set_batch_lanes(g);
    g.ctrl = args[k].ctrl;
    g.stats = args[k].stats;
    g.timeout_ns = args[k].timeout_ns;
    t[size_t(k)] = g;
  }
  cudaError_t e = cudaMemcpyAsync(d_table, t.data(), ir_batch_table_bytes(nprob), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // t is released on return
  return e;
}

namespace {
using IrbKernel = void (*)(const GArgs*, const int*, int);
IrbKernel irb_for(int kind) {
  switch (kind) {
    case kOpVelU: return irb_kernel<kOpVelU>;
    case kOpVelV: return irb_kernel<kOpVelV>;
    case kOpVelW: return irb_kernel<kOpVelW>;
    default: return irb_kernel<kOpPressure>;
  }
}
}  // namespace

int ir_batch_blocks_per_sm(int kind) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, irb_for(kind), kGThreads, 0);
  return b;
}

cudaError_t launch_ir_batch(const void* d_table, const int* d_starts, int nprob, int total_blocks, int kind,
                            cudaStream_t s, int64_t* launches) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(total_blocks));
  cfg.blockDim = dim3(32, 8);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (launches) *launches += 1;
  const GArgs* t = static_cast<const GArgs*>(d_table);
  return cudaLaunchKernelEx(&cfg, irb_for(kind), t, d_starts, nprob);
}

cudaError_t ir_graph_kernel_count(const void* state_buf, cudaStream_t s, long long* out) {
  const GState* S = static_cast<const GState*>(state_buf);
  cudaError_t e = cudaMemcpyAsync(out, &S->kernels, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace cfd
