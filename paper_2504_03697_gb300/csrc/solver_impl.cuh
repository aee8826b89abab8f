// Device code of the matrix-free 7-point operators and the persistent
// conjugate-gradient solves of the cavity projection path (sm_103a): helpers
// and kernel templates, instantiated by solver_k_*.cu (one kernel family per
// translation unit, so that they compile in parallel) and launched by
// solver.cu.
//
// Sec. 3.1 of arXiv 2504.03697: the pressure Poisson system is solved by
// (preconditioned) conjugate gradients; Table 1 lists its pieces (spmv,
// precondition, dot, vector add / scale / multiply_add_inplace).  Here the
// operator is never assembled: each row is evaluated from the grid indices.
//
// Row evaluation.  Every operator of the step is "6 x_c minus the sum of six
// neighbour values", with out-of-box neighbours substituted so that the
// boundary rule comes out exactly:
//   * pressure (homogeneous Neumann walls): a missing neighbour takes x_c,
//     so the row is n_c x_c - sum(interior neighbours), n_c = 3..6;
//   * velocity diffusion, tangential axis: a missing neighbour takes -x_c,
//     the ghost 2W - x_c with the wall value W moved to the right-hand side;
//   * velocity diffusion, own axis: the wall faces are stored (always 0) and
//     their rows are fixed (output 0).
// Velocity rows return x_c + c (6 x_c - sum) (backward Euler, c = nu dt/h^2).
// This keeps the FP64 work at 5 adds + 1 FMA per row (velocity: + 1 FMA),
// which matters on GB300, whose FP64 pipe is far slower than its HBM.
//
// CG layout.  One persistent, cooperatively launched kernel runs the whole
// solve with two grid-wide all-reduces per iteration:
//   phase D (tiled stencil): p_new = z + beta p_old on a shared-memory tile
//     with halo (z = r, or r / diag for Jacobi), store p_new, q = A p_new,
//     partial p.q;
//   phase U:  x += alpha p_new, r -= alpha q, partial r.r (and r.z).
// Tiles are kTileX x kTileY x tz cells; tile t belongs to block t mod grid.
// When every block owns at most kRegCells / tz tiles ("register path", the
// small grids where the solve is latency-bound), the block keeps p_new and q
// of its own cells in registers from phase D to phase U: q is never stored
// and phase U touches only x and r.  Otherwise q goes through memory and
// phase U is a flat pass.  Reductions are deterministic (cfd_common.cuh), so
// a solve is bitwise reproducible run to run for a given launch shape.

#pragma once

#include <cudaTypedefs.h>

#include <cmath>

#include "cfd_internal.h"
#include "operator_rows.cuh"

namespace cfd {

namespace {

constexpr int kModeApply = 0;  // y = A x
constexpr int kModeResid = 1;  // r = (b - shift) - A x, partials b.b, r.r, r.z
constexpr int kModeDir = 2;    // p_new = z + beta p_old; q = A p_new; partial p.q

constexpr int kTileW = kTileX + 2;
constexpr int kTileH = kTileY + 2;
constexpr int kMaxTz = 8;     // deepest tile (cells per thread along z)
constexpr int kTileSlots = kTileW * kTileH * (kMaxTz + 2);
constexpr int kRegCells = 8;  // own cells per thread kept in registers (register path)

// Number of in-box neighbours of a pressure cell (the diagonal of A).
__device__ __forceinline__ int neighbour_count(int i, int j, int k, int mx, int my, int mz) {
  return (i > 0) + (i < mx - 1) + (j > 0) + (j < my - 1) + (k > 0) + (k < mz - 1);
}

// Value source of the tiled stencil: the vector the operator is applied to.
template <typename T, int MODE, int PRECOND>
struct Source {
  const T* in;      // x (apply / resid) or r (dir)
  const T* pold;    // dir only
  T beta;
  bool first;
  const T* invd;    // shared table 1/n, n = 0..6 (Jacobi)
  int mx, my, mz;

  __device__ __forceinline__ T operator()(size_t e, int i, int j, int k) const {
    if (MODE == kModeDir) {
      T z = in[e];
      if (PRECOND) z *= invd[neighbour_count(i, j, k, mx, my, mz)];
      return first ? z : fma(beta, pold[e], z);
    } else {
      return in[e];
    }
  }
};

struct TileShape {
  int mx, my, mz, tz;
  int ntx, nty, ntz;
  __host__ __device__ __forceinline__ int count() const { return ntx * nty * ntz; }
};

__host__ __device__ __forceinline__ TileShape make_tiles(int mx, int my, int mz, int tz) {
  TileShape t;
  t.mx = mx; t.my = my; t.mz = mz; t.tz = tz;
  t.ntx = (mx + kTileX - 1) / kTileX;
  t.nty = (my + kTileY - 1) / kTileY;
  t.ntz = (mz + tz - 1) / tz;
  return t;
}

// Outputs / accumulators of one stencil pass.
template <typename T>
struct Sink {
  T* y;          // apply: y; resid: r; dir: q (nullptr on the register path)
  T* pnew;       // dir
  T* b;          // resid: right-hand side (read, optionally rewritten)
  T bshift;      // resid: subtracted from b
  bool write_b;  // resid
  int kind;
  T c;
};

// Evaluate tile t and its one-cell halo (edges and corners excluded: the
// 7-point stencil never reads them) into shared memory, all loads in flight
// at once.  Ends with a block barrier.
template <typename T, int MODE, int PRECOND>
__device__ __forceinline__ void load_tile(const TileShape& ts, int t, const Source<T, MODE, PRECOND>& src, T* s,
                                          int& x0, int& y0, int& z0) {
  const int bx = t % ts.ntx;
  const int rest = t / ts.ntx;
  const int by = rest % ts.nty;
  const int bz = rest / ts.nty;
  x0 = bx * kTileX;
  y0 = by * kTileY;
  z0 = bz * ts.tz;
  const int D = ts.tz + 2;
  const int slots = kTileW * kTileH * D;
  for (int l = threadIdx.x; l < slots; l += kSolveThreads) {
    const int lx = l % kTileW;
    const int r2 = l / kTileW;
    const int ly = r2 % kTileH;
    const int lz = r2 / kTileH;
    const int gi = x0 + lx - 1, gj = y0 + ly - 1, gk = z0 + lz - 1;
    const int halo = (lx == 0 || lx == kTileW - 1) + (ly == 0 || ly == kTileH - 1) + (lz == 0 || lz == D - 1);
    T v = T(0);
    if (halo <= 1 && gi >= 0 && gi < ts.mx && gj >= 0 && gj < ts.my && gk >= 0 && gk < ts.mz)
      v = src(idx3(gi, gj, gk, ts.mx, ts.my), gi, gj, gk);
    s[l] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ int tile_cell(int kz, int tx, int ty) {
  return ((kz + 1) * kTileH + (ty + 1)) * kTileW + (tx + 1);
}

template <typename T>
__device__ __forceinline__ T row_from_smem(const Sink<T>& out, const T* s, int c, int i, int j, int k, int mx, int my,
                                           int mz) {
  return stencil_row<T>(out.kind, out.c, i, j, k, mx, my, mz, s[c], s[c - 1], s[c + 1], s[c - kTileW], s[c + kTileW],
                        s[c - kTileW * kTileH], s[c + kTileW * kTileH]);
}

// Memory-path stencil pass over all tiles of this block.  Partial sums
// accumulate per thread in T (FP64 solves: double; the FP32 inner solve:
// float, a handful of terms per thread) and are reduced across threads and
// blocks in FP64 by the caller.  Resid mode: acc = {b.b, r.r, r.z (Jacobi)
// or sum(r) (no preconditioner)}.
template <typename T, int MODE, int PRECOND>
__device__ void stencil_tiles(const TileShape& ts, const Source<T, MODE, PRECOND>& src, const Sink<T>& out,
                              T (&acc)[3], T* s, VBlock vb) {
  const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
  const int mx = ts.mx, my = ts.my, mz = ts.mz;
  const int ntiles = ts.count();
  for (int t = vb.bid; t < ntiles; t += vb.nb) {
    int x0, y0, z0;
    load_tile<T, MODE, PRECOND>(ts, t, src, s, x0, y0, z0);
    const int i = x0 + tx, j = y0 + ty;
    if (i < mx && j < my) {
      const int z1 = min(z0 + ts.tz, mz);
      for (int k = z0; k < z1; ++k) {
        const int c = tile_cell(k - z0, tx, ty);
        const T pc = s[c];
        const T y = row_from_smem<T>(out, s, c, i, j, k, mx, my, mz);
        const size_t e = idx3(i, j, k, mx, my);
        if (MODE == kModeApply) {
          out.y[e] = y;
        } else if (MODE == kModeDir) {
          out.pnew[e] = pc;
          out.y[e] = y;
          acc[0] = fma(pc, y, acc[0]);
        } else {  // resid
          T bv = out.b[e] - out.bshift;
          if (out.write_b) out.b[e] = bv;
          const T r = bv - y;
          out.y[e] = r;
          acc[0] = fma(bv, bv, acc[0]);
          acc[1] = fma(r, r, acc[1]);
          if (PRECOND) acc[2] = fma(r * r, src.invd[neighbour_count(i, j, k, mx, my, mz)], acc[2]);
          else acc[2] += r;
        }
      }
    }
    __syncthreads();
  }
}

// Register-path phase D: tiles of compile-time depth RTZ, at most
// kRegCells / RTZ per block; p_new is stored (neighbours need it next
// iteration), p_new and q of own cells stay in preg / qreg.
template <int RTZ, int PRECOND>
__device__ void dir_tiles_reg(const TileShape& ts, const Source<double, kModeDir, PRECOND>& src, double* pnew,
                              const Sink<double>& out, double (&acc)[3], double* s, double (&preg)[kRegCells],
                              double (&qreg)[kRegCells], VBlock vb) {
  const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
  const int mx = ts.mx, my = ts.my, mz = ts.mz;
  const int ntiles = ts.count();
#pragma unroll
  for (int kt = 0; kt < kRegCells / RTZ; ++kt) {
    const int t = vb.bid + kt * vb.nb;
    if (t >= ntiles) break;
    int x0, y0, z0;
    load_tile<double, kModeDir, PRECOND>(ts, t, src, s, x0, y0, z0);
    const int i = x0 + tx, j = y0 + ty;
#pragma unroll
    for (int kz = 0; kz < RTZ; ++kz) {
      const int k = z0 + kz;
      double pc = 0.0, y = 0.0;
      if (i < mx && j < my && k < mz) {
        const int c = tile_cell(kz, tx, ty);
        pc = s[c];
        y = row_from_smem<double>(out, s, c, i, j, k, mx, my, mz);
        pnew[idx3(i, j, k, mx, my)] = pc;
        acc[0] = fma(pc, y, acc[0]);
      }
      preg[kt * RTZ + kz] = pc;
      qreg[kt * RTZ + kz] = y;
    }
    __syncthreads();
  }
}

// Register-path phase U over the same own cells.
template <int RTZ, int PRECOND>
__device__ void update_reg(const TileShape& ts, double alpha, double* x, double* r, const double* invd,
                           double (&acc)[3], const double (&preg)[kRegCells], const double (&qreg)[kRegCells],
                           VBlock vb) {
  const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
  const int mx = ts.mx, my = ts.my, mz = ts.mz;
  const int ntiles = ts.count();
#pragma unroll
  for (int kt = 0; kt < kRegCells / RTZ; ++kt) {
    const int t = vb.bid + kt * vb.nb;
    if (t >= ntiles) break;
    const int bx = t % ts.ntx;
    const int rest = t / ts.ntx;
    const int by = rest % ts.nty;
    const int bz = rest / ts.nty;
    const int i = bx * kTileX + tx, j = by * kTileY + ty, z0 = bz * RTZ;
    if (i >= mx || j >= my) continue;
#pragma unroll
    for (int kz = 0; kz < RTZ; ++kz) {
      const int k = z0 + kz;
      if (k >= mz) break;
      const size_t e = idx3(i, j, k, mx, my);
      x[e] = fma(alpha, preg[kt * RTZ + kz], x[e]);
      const double re = fma(-alpha, qreg[kt * RTZ + kz], r[e]);
      r[e] = re;
      acc[0] = fma(re, re, acc[0]);
      if (PRECOND) acc[1] = fma(re * re, invd[neighbour_count(i, j, k, mx, my, mz)], acc[1]);
    }
  }
}

// Multi-problem launches: starts[p] .. starts[p+1] are problem p's blocks.
// Returns this block's problem (0 for a single-problem launch, -1 for a
// block past the last problem) and narrows vb to that problem's blocks.
__device__ __forceinline__ int find_problem(const int* starts, int nprob, VBlock& vb) {
  if (nprob <= 0) return 0;
  const int b = int(blockIdx.x);
  if (b >= starts[nprob]) return -1;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (starts[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  vb.bid = b - starts[lo];
  vb.nb = starts[lo + 1] - starts[lo];
  return lo;
}

__device__ __forceinline__ size_t gtid(VBlock vb) { return size_t(vb.bid) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride(VBlock vb) { return size_t(vb.nb) * blockDim.x; }

// num / den formed once per block by thread 0 and broadcast through *slot:
// the same value every thread would form from the same (block-uniform)
// operands, without each of them issuing an FP64 division, which on GB300's
// FP64 pipe is a long instruction chain.  The caller must pass through a
// block barrier (an all-reduce) before the same slot is used again.
__device__ __forceinline__ double block_div(double num, double den, double* slot) {
  if (threadIdx.x == 0) *slot = num / den;
  __syncthreads();
  return *slot;
}

// ---------------------------------------------------------------------------
// Persistent FP64 (P)CG.  PRECOND: 0 none, 1 Jacobi.  RTZ: 0 memory path
// (runtime tile depth a.tz), else register path with tile depth RTZ.
// ---------------------------------------------------------------------------
template <int PRECOND, int RTZ, bool MULTI>
__global__ void __launch_bounds__(kSolveThreads) cg_fp64_kernel(const __grid_constant__ CgArgs a0, const CgArgs* table,
                                                                const int* starts, int nprob) {
  VBlock vb{int(blockIdx.x), int(gridDim.x)};
  const int prob = MULTI ? find_problem(starts, nprob, vb) : 0;
  if (prob < 0) return;
  const CgArgs& a = MULTI ? table[prob] : a0;
  __shared__ double s_tile[kTileSlots];
  __shared__ double s_red[32 * 3];
  __shared__ double s_div[2];
  __shared__ double s_invd[8];
  if (threadIdx.x < 8) s_invd[threadIdx.x] = threadIdx.x == 0 ? 0.0 : 1.0 / double(threadIdx.x);
  __syncthreads();

  const int mx = a.g.mx, my = a.g.my, mz = a.g.mz;
  const size_t n = size_t(mx) * my * mz;
  const TileShape ts = make_tiles(mx, my, mz, RTZ > 0 ? RTZ : a.tz);
  const double c = a.c;
  DevSolveStats* st = a.stats;
  unsigned int round = 0;

  auto fail = [&]() {
    if (threadIdx.x == 0) {
      int e = ld_volatile_s32(&a.ctrl->error);
      st->status = e != 0 ? e : kErrTimeout;
    }
  };
  auto allreduce = [&](double (&v)[3], double (&o)[3]) {
    return grid_allreduce<3>(v, o, a.ctrl, a.partials, s_red, a.timeout_ns, round, vb);
  };

  double acc[3], tot[3];
  double preg[kRegCells], qreg[kRegCells];

  // ---- mean of b (pressure systems are only solvable for zero-mean b) ----
  double shift = 0.0;
  if (a.remove_mean) {
    acc[0] = acc[1] = acc[2] = 0.0;
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) acc[0] += a.b[e];
    if (!allreduce(acc, tot)) return fail();
    shift = tot[0] / double(n);
  }

  // ---- initial residual r = b - A x0 ----
  acc[0] = acc[1] = acc[2] = 0.0;
  if (a.zero_x0) {
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) {
      const double bv = a.b[e] - shift;
      if (a.remove_mean) a.b[e] = bv;
      a.x[e] = 0.0;
      a.r[e] = bv;
      acc[0] = fma(bv, bv, acc[0]);
      if (PRECOND) {
        const int i = int(e % mx), j = int((e / mx) % my), k = int(e / (size_t(mx) * my));
        acc[2] = fma(bv * bv, s_invd[neighbour_count(i, j, k, mx, my, mz)], acc[2]);
      }
    }
    acc[1] = acc[0];
  } else {
    Source<double, kModeResid, PRECOND> src{a.x, nullptr, 0.0, false, s_invd, mx, my, mz};
    Sink<double> out{a.r, nullptr, a.b, shift, a.remove_mean != 0, a.kind, c};
    stencil_tiles<double, kModeResid, PRECOND>(ts, src, out, acc, s_tile, vb);
  }
  if (!allreduce(acc, tot)) return fail();
  const double bb = tot[0];
  double rr = tot[1];
  double rz = PRECOND ? tot[2] : tot[1];

  int status = kErrNotConverged, iters = 0, restarts = 0;
  double rr_true = -1.0;
  if (bb == 0.0) {
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) a.x[e] = 0.0;
    status = kOk;
    rr_true = 0.0;
  } else {
    const double tol2 = a.rtol * a.rtol * bb;
    bool first = true;
    double beta = 0.0;
    int cur = 0;
    while (true) {
      if (rr <= tol2) {
        // the recurrence says converged: confirm with the true residual
        acc[0] = acc[1] = acc[2] = 0.0;
        Source<double, kModeResid, PRECOND> src{a.x, nullptr, 0.0, false, s_invd, mx, my, mz};
        Sink<double> out{a.r, nullptr, a.b, 0.0, false, a.kind, c};
        stencil_tiles<double, kModeResid, PRECOND>(ts, src, out, acc, s_tile, vb);
        if (!allreduce(acc, tot)) return fail();
        rr_true = tot[1];
        if (rr_true <= tol2) {
          status = kOk;
          break;
        }
        if (++restarts > a.max_restarts) break;
        rr = rr_true;
        rz = PRECOND ? tot[2] : tot[1];
        rr_true = -1.0;
        first = true;
      }
      if (iters >= a.max_iters) break;
      // phase D: p_new = z + beta p_old fused into q = A p_new, partial p.q
      double* pnew = cur ? a.d1 : a.d0;
      const double* pold = cur ? a.d0 : a.d1;
      acc[0] = acc[1] = acc[2] = 0.0;
      {
        Source<double, kModeDir, PRECOND> src{a.r, pold, beta, first, s_invd, mx, my, mz};
        if (RTZ > 0) {
          Sink<double> out{nullptr, pnew, nullptr, 0.0, false, a.kind, c};
          dir_tiles_reg<(RTZ > 0 ? RTZ : 1), PRECOND>(ts, src, pnew, out, acc, s_tile, preg, qreg, vb);
        } else {
          Sink<double> out{a.q, pnew, nullptr, 0.0, false, a.kind, c};
          stencil_tiles<double, kModeDir, PRECOND>(ts, src, out, acc, s_tile, vb);
        }
      }
      if (!allreduce(acc, tot)) return fail();
      const double pq = tot[0];
      if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz)) {
        status = kErrBreakdown;
        break;
      }
      const double alpha = block_div(rz, pq, &s_div[0]);
      // phase U: x += alpha p, r -= alpha q, partial r.r (and r.z)
      acc[0] = acc[1] = acc[2] = 0.0;
      if (RTZ > 0) {
        update_reg<(RTZ > 0 ? RTZ : 1), PRECOND>(ts, alpha, a.x, a.r, s_invd, acc, preg, qreg, vb);
      } else {
        for (size_t e = gtid(vb); e < n; e += gstride(vb)) {
          const double pe = pnew[e];
          const double qe = a.q[e];
          a.x[e] = fma(alpha, pe, a.x[e]);
          const double re = fma(-alpha, qe, a.r[e]);
          a.r[e] = re;
          acc[0] = fma(re, re, acc[0]);
          if (PRECOND) {
            const int i = int(e % mx), j = int((e / mx) % my), k = int(e / (size_t(mx) * my));
            acc[1] = fma(re * re, s_invd[neighbour_count(i, j, k, mx, my, mz)], acc[1]);
          }
        }
      }
      if (!allreduce(acc, tot)) return fail();
      rr = tot[0];
      const double rz_new = PRECOND ? tot[1] : tot[0];
      beta = block_div(rz_new, rz, &s_div[1]);
      rz = rz_new;
      first = false;
      cur ^= 1;
      ++iters;
    }
    if (rr_true < 0.0) {
      // left without a true-residual check (cap, breakdown, restarts): measure it
      acc[0] = acc[1] = acc[2] = 0.0;
      Source<double, kModeResid, PRECOND> src{a.x, nullptr, 0.0, false, s_invd, mx, my, mz};
      Sink<double> out{a.r, nullptr, a.b, 0.0, false, a.kind, c};
      stencil_tiles<double, kModeResid, PRECOND>(ts, src, out, acc, s_tile, vb);
      if (!allreduce(acc, tot)) return fail();
      rr_true = tot[1];
    }
  }

  // ---- gauge: shift x to the requested mean ----
  if (a.gauge) {
    acc[0] = acc[1] = acc[2] = 0.0;
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) acc[0] += a.x[e];
    if (!allreduce(acc, tot)) return fail();
    const double sh = a.gauge_value - tot[0] / double(n);
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) a.x[e] += sh;
  }

  if (vb.bid == 0 && threadIdx.x == 0) {
    st->iters = iters;
    st->outer_iters = 0;
    st->restarts = restarts;
    st->status = status;
    st->b_norm = sqrt(bb);
    st->rel_resid = bb > 0.0 ? sqrt(rr_true / bb) : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Single-reduction FP64 CG (Chronopoulos-Gear form): one grid all-reduce per
// iteration instead of two.  With w = A r and s = A p carried by recurrence,
//   beta_k = g_k / g_{k-1},  alpha_k = g_k / (d_k - beta_k g_k / alpha_{k-1})
//   p_k = r_k + beta_k p_{k-1},  s_k = w_k + beta_k s_{k-1}
//   x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k s_k
//   w_{k+1} = A r_{k+1},  g_{k+1} = r_{k+1}.r_{k+1},  d_{k+1} = w_{k+1}.r_{k+1}
// (g_0 = r_0.r_0, d_0 = w_0.r_0, beta_0 = 0, alpha_0 = g_0 / d_0): the same
// iterates as the two-reduction form in exact arithmetic.  One tiled pass
// per iteration: each block evaluates r_{k+1} on its tile AND its halo from
// r_k, w_k, s_{k-1} (all written before the previous all-reduce), so the
// stencil w_{k+1} = A r_{k+1} needs no barrier of its own.  r, w and s are
// double-buffered (neighbours read iteration k's values while this block
// writes k+1's); p and x belong to one block only and stay in registers on
// the register path (RTZ > 0) or in memory otherwise.  Unpreconditioned
// only; the convergence test, true-residual restarts, gauge and statistics
// follow the two-reduction kernel.
// ---------------------------------------------------------------------------

// r_{k+1} = r_k - alpha (w_k + beta s_{k-1}) at any cell (tile or halo)
struct NextResidual {
  const double* r;
  const double* w;
  const double* s;
  double alpha, beta;
  bool first;
  __device__ __forceinline__ double operator()(size_t e, int, int, int) const {
    const double se = first ? w[e] : fma(beta, s[e], w[e]);
    return fma(-alpha, se, r[e]);
  }
};

struct PlainValue {
  const double* in;
  __device__ __forceinline__ double operator()(size_t e, int, int, int) const { return in[e]; }
};

// load_tile for any value functor (see load_tile)
template <typename F>
__device__ __forceinline__ void load_tile_fn(const TileShape& ts, int t, const F& src, double* s, int& x0, int& y0,
                                             int& z0) {
  const int bx = t % ts.ntx;
  const int rest = t / ts.ntx;
  const int by = rest % ts.nty;
  const int bz = rest / ts.nty;
  x0 = bx * kTileX;
  y0 = by * kTileY;
  z0 = bz * ts.tz;
  const int D = ts.tz + 2;
  const int slots = kTileW * kTileH * D;
  for (int l = threadIdx.x; l < slots; l += kSolveThreads) {
    const int lx = l % kTileW;
    const int r2 = l / kTileW;
    const int ly = r2 % kTileH;
    const int lz = r2 / kTileH;
    const int gi = x0 + lx - 1, gj = y0 + ly - 1, gk = z0 + lz - 1;
    const int halo = (lx == 0 || lx == kTileW - 1) + (ly == 0 || ly == kTileH - 1) + (lz == 0 || lz == D - 1);
    double v = 0.0;
    if (halo <= 1 && gi >= 0 && gi < ts.mx && gj >= 0 && gj < ts.my && gk >= 0 && gk < ts.mz)
      v = src(idx3(gi, gj, gk, ts.mx, ts.my), gi, gj, gk);
    s[l] = v;
  }
  __syncthreads();
}

// w = A r on this block's tiles; acc += {r.r, w.r}
__device__ void apply_dot_tiles(const TileShape& ts, const double* r, double* w, int kind, double c, double (&acc)[3],
                                double* s, VBlock vb) {
  const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
  const int ntiles = ts.count();
  Sink<double> out{nullptr, nullptr, nullptr, 0.0, false, kind, c};
  for (int t = vb.bid; t < ntiles; t += vb.nb) {
    int x0, y0, z0;
    load_tile_fn(ts, t, PlainValue{r}, s, x0, y0, z0);
    const int i = x0 + tx, j = y0 + ty;
    if (i < ts.mx && j < ts.my) {
      const int z1 = min(z0 + ts.tz, ts.mz);
      for (int k = z0; k < z1; ++k) {
        const int cl = tile_cell(k - z0, tx, ty);
        const double rv = s[cl];
        const double wv = row_from_smem<double>(out, s, cl, i, j, k, ts.mx, ts.my, ts.mz);
        w[idx3(i, j, k, ts.mx, ts.my)] = wv;
        acc[0] = fma(rv, rv, acc[0]);
        acc[1] = fma(wv, rv, acc[1]);
      }
    }
    __syncthreads();
  }
}

template <int RTZ>
__global__ void __launch_bounds__(kSolveThreads, RTZ > 0 ? 2 : 3) cg1_fp64_kernel(const __grid_constant__ CgArgs a) {
  VBlock vb{int(blockIdx.x), int(gridDim.x)};
  __shared__ double s_tile[kTileSlots];
  __shared__ double s_red[32 * 3];
  __shared__ double s_invd[8];
  __shared__ double s_sc[2];  // alpha, beta of the iteration (formed by thread 0)
  if (threadIdx.x < 8) s_invd[threadIdx.x] = threadIdx.x == 0 ? 0.0 : 1.0 / double(threadIdx.x);
  __syncthreads();

  const int mx = a.g.mx, my = a.g.my, mz = a.g.mz;
  const size_t n = size_t(mx) * my * mz;
  const TileShape ts = make_tiles(mx, my, mz, RTZ > 0 ? RTZ : a.tz);
  const int ntiles = ts.count();
  const double c = a.c;
  DevSolveStats* st = a.stats;
  unsigned int round = 0;
  const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
  // double-buffered r, w, s; p in memory on the memory path
  auto rb = [&](int i) { return i ? a.e0 : a.r; };
  auto wb = [&](int i) { return i ? a.d1 : a.d0; };
  auto sb = [&](int i) { return i ? a.e1 : a.q; };
  double* pm = a.e2;

  auto fail = [&]() {
    if (threadIdx.x == 0) {
      int e = ld_volatile_s32(&a.ctrl->error);
      st->status = e != 0 ? e : kErrTimeout;
    }
  };
  auto allreduce = [&](double (&v)[3], double (&o)[3]) {
    return grid_allreduce<3>(v, o, a.ctrl, a.partials, s_red, a.timeout_ns, round, vb);
  };

  double acc[3], tot[3];
  double xreg[kRegCells], preg[kRegCells];
#pragma unroll
  for (int q = 0; q < kRegCells; ++q) xreg[q] = preg[q] = 0.0;

  // own cells of the register path: tile t = bid + kt nb, depth RTZ
  auto own_cell = [&](int kt, int kz, size_t& e) -> bool {
    const int t = vb.bid + kt * vb.nb;
    if (t >= ntiles) return false;
    const int bx = t % ts.ntx, rest = t / ts.ntx, by = rest % ts.nty, bz = rest / ts.nty;
    const int i = bx * kTileX + tx, j = by * kTileY + ty, k = bz * ts.tz + kz;
    if (i >= mx || j >= my || k >= mz) return false;
    e = idx3(i, j, k, mx, my);
    return true;
  };
  // register path: x of own cells to / from memory
  auto store_x = [&]() {
    if (RTZ > 0) {
#pragma unroll
      for (int kt = 0; kt < kRegCells / (RTZ > 0 ? RTZ : 1); ++kt)
#pragma unroll
        for (int kz = 0; kz < (RTZ > 0 ? RTZ : 1); ++kz) {
          size_t e;
          if (own_cell(kt, kz, e)) a.x[e] = xreg[kt * RTZ + kz];
        }
    }
  };

  // ---- mean of b ----
  double shift = 0.0;
  if (a.remove_mean) {
    acc[0] = acc[1] = acc[2] = 0.0;
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) acc[0] += a.b[e];
    if (!allreduce(acc, tot)) return fail();
    shift = tot[0] / double(n);
  }

  // ---- r_0 = b - A x_0 into rb(0); b.b ----
  acc[0] = acc[1] = acc[2] = 0.0;
  if (a.zero_x0) {
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) {
      const double bv = a.b[e] - shift;
      if (a.remove_mean) a.b[e] = bv;
      a.x[e] = 0.0;
      rb(0)[e] = bv;
      acc[0] = fma(bv, bv, acc[0]);
    }
  } else {
    Source<double, kModeResid, 0> src{a.x, nullptr, 0.0, false, s_invd, mx, my, mz};
    Sink<double> out{rb(0), nullptr, a.b, shift, a.remove_mean != 0, a.kind, c};
    stencil_tiles<double, kModeResid, 0>(ts, src, out, acc, s_tile, vb);
  }
  if (!allreduce(acc, tot)) return fail();
  const double bb = tot[0];
  if (RTZ > 0) {
#pragma unroll
    for (int kt = 0; kt < kRegCells / (RTZ > 0 ? RTZ : 1); ++kt)
#pragma unroll
      for (int kz = 0; kz < (RTZ > 0 ? RTZ : 1); ++kz) {
        size_t e;
        if (own_cell(kt, kz, e)) xreg[kt * RTZ + kz] = a.x[e];
      }
  }

  int status = kErrNotConverged, iters = 0, restarts = 0;
  double rr_true = -1.0;
  int cur = 0;
  if (bb == 0.0) {
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) a.x[e] = 0.0;
#pragma unroll
    for (int q = 0; q < kRegCells; ++q) xreg[q] = 0.0;
    status = kOk;
    rr_true = 0.0;
  } else {
    const double tol2 = a.rtol * a.rtol * bb;
    // w_0 = A r_0; g = r.r, d = w.r
    acc[0] = acc[1] = acc[2] = 0.0;
    apply_dot_tiles(ts, rb(0), wb(0), a.kind, c, acc, s_tile, vb);
    if (!allreduce(acc, tot)) return fail();
    double g = tot[0], d = tot[1];
    double g_prev = 0.0, alpha_prev = 0.0;
    bool first = true;
    while (true) {
      if (g <= tol2) {
        // the recurrence says converged: confirm with the true residual
        store_x();
        acc[0] = acc[1] = acc[2] = 0.0;
        if (!allreduce(acc, tot)) return fail();  // x of every block stored
        Source<double, kModeResid, 0> src{a.x, nullptr, 0.0, false, s_invd, mx, my, mz};
        Sink<double> out{rb(cur), nullptr, a.b, 0.0, false, a.kind, c};
        stencil_tiles<double, kModeResid, 0>(ts, src, out, acc, s_tile, vb);
        if (!allreduce(acc, tot)) return fail();
        rr_true = tot[1];
        if (rr_true <= tol2) {
          status = kOk;
          break;
        }
        if (++restarts > a.max_restarts) break;
        rr_true = -1.0;
        acc[0] = acc[1] = acc[2] = 0.0;
        apply_dot_tiles(ts, rb(cur), wb(cur), a.kind, c, acc, s_tile, vb);
        if (!allreduce(acc, tot)) return fail();
        g = tot[0];
        d = tot[1];
        first = true;
      }
      if (iters >= a.max_iters) break;
      // the scalars once per block (see block_div); the slots are next
      // written after this iteration's all-reduce
      if (threadIdx.x == 0) {
        if (first) {
          s_sc[1] = 0.0;
          s_sc[0] = g / d;
        } else {
          const double b = g / g_prev;
          s_sc[1] = b;
          s_sc[0] = g / (d - b * g / alpha_prev);
        }
      }
      __syncthreads();
      const double alpha = s_sc[0], beta = s_sc[1];
      if (!(alpha > 0.0) || !isfinite(alpha) || !isfinite(beta)) {
        status = kErrBreakdown;
        break;
      }
      const double* r0 = rb(cur);
      const double* w0 = wb(cur);
      const double* s0 = sb(cur);
      double* r1 = rb(cur ^ 1);
      double* w1 = wb(cur ^ 1);
      double* s1 = sb(cur ^ 1);
      const NextResidual src{r0, w0, s0, alpha, beta, first};
      Sink<double> out{nullptr, nullptr, nullptr, 0.0, false, a.kind, c};
      acc[0] = acc[1] = acc[2] = 0.0;
      if (RTZ > 0) {
#pragma unroll
        for (int kt = 0; kt < kRegCells / (RTZ > 0 ? RTZ : 1); ++kt) {
          const int t = vb.bid + kt * vb.nb;
          if (t >= ntiles) break;
          int x0, y0, z0;
          load_tile_fn(ts, t, src, s_tile, x0, y0, z0);
          const int i = x0 + tx, j = y0 + ty;
#pragma unroll
          for (int kz = 0; kz < (RTZ > 0 ? RTZ : 1); ++kz) {
            const int k = z0 + kz;
            if (i < mx && j < my && k < mz) {
              const size_t e = idx3(i, j, k, mx, my);
              const int cl = tile_cell(kz, tx, ty);
              const double rk = r0[e];
              const double sk = first ? w0[e] : fma(beta, s0[e], w0[e]);
              const double pk = first ? rk : fma(beta, preg[kt * RTZ + kz], rk);
              preg[kt * RTZ + kz] = pk;
              xreg[kt * RTZ + kz] = fma(alpha, pk, xreg[kt * RTZ + kz]);
              const double rn = s_tile[cl];
              const double wn = row_from_smem<double>(out, s_tile, cl, i, j, k, mx, my, mz);
              r1[e] = rn;
              w1[e] = wn;
              s1[e] = sk;
              acc[0] = fma(rn, rn, acc[0]);
              acc[1] = fma(wn, rn, acc[1]);
            }
          }
          __syncthreads();
        }
      } else {
        for (int t = vb.bid; t < ntiles; t += vb.nb) {
          int x0, y0, z0;
          load_tile_fn(ts, t, src, s_tile, x0, y0, z0);
          const int i = x0 + tx, j = y0 + ty;
          if (i < mx && j < my) {
            const int z1 = min(z0 + ts.tz, mz);
            for (int k = z0; k < z1; ++k) {
              const size_t e = idx3(i, j, k, mx, my);
              const int cl = tile_cell(k - z0, tx, ty);
              const double rk = r0[e];
              const double sk = first ? w0[e] : fma(beta, s0[e], w0[e]);
              const double pk = first ? rk : fma(beta, pm[e], rk);
              pm[e] = pk;
              a.x[e] = fma(alpha, pk, a.x[e]);
              const double rn = s_tile[cl];
              const double wn = row_from_smem<double>(out, s_tile, cl, i, j, k, mx, my, mz);
              r1[e] = rn;
              w1[e] = wn;
              s1[e] = sk;
              acc[0] = fma(rn, rn, acc[0]);
              acc[1] = fma(wn, rn, acc[1]);
            }
          }
          __syncthreads();
        }
      }
      if (!allreduce(acc, tot)) return fail();
      g_prev = g;
      alpha_prev = alpha;
      g = tot[0];
      d = tot[1];
      first = false;
      cur ^= 1;
      ++iters;
    }
    if (rr_true < 0.0) {
      // left without a true-residual check (cap, breakdown, restarts): measure it
      store_x();
      acc[0] = acc[1] = acc[2] = 0.0;
      if (!allreduce(acc, tot)) return fail();
      Source<double, kModeResid, 0> src{a.x, nullptr, 0.0, false, s_invd, mx, my, mz};
      Sink<double> out{rb(cur), nullptr, a.b, 0.0, false, a.kind, c};
      stencil_tiles<double, kModeResid, 0>(ts, src, out, acc, s_tile, vb);
      if (!allreduce(acc, tot)) return fail();
      rr_true = tot[1];
    }
  }
  store_x();

  // ---- gauge: shift x to the requested mean ----
  if (a.gauge) {
    acc[0] = acc[1] = acc[2] = 0.0;
    if (!allreduce(acc, tot)) return fail();  // every block's x stored
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) acc[0] += a.x[e];
    if (!allreduce(acc, tot)) return fail();
    const double sh = a.gauge_value - tot[0] / double(n);
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) a.x[e] += sh;
  }

  if (vb.bid == 0 && threadIdx.x == 0) {
    st->iters = iters;
    st->outer_iters = 0;
    st->restarts = restarts;
    st->status = status;
    st->b_norm = sqrt(bb);
    st->rel_resid = bb > 0.0 ? sqrt(rr_true / bb) : 0.0;
  }
}

// One-shot y = A x (non-persistent; one block per tile).
__global__ void __launch_bounds__(kSolveThreads) apply_poisson_kernel(GridDims g, const double* x, double* y, int tz) {
  __shared__ double s_tile[kTileSlots];
  const TileShape ts = make_tiles(g.mx, g.my, g.mz, tz);
  double acc[3] = {0.0, 0.0, 0.0};
  Source<double, kModeApply, 0> src{x, nullptr, 0.0, false, nullptr, g.mx, g.my, g.mz};
  Sink<double> out{y, nullptr, nullptr, 0.0, false, kOpPressure, 0.0};
  stencil_tiles<double, kModeApply, 0>(ts, src, out, acc, s_tile, VBlock{int(blockIdx.x), int(gridDim.x)});
}

// ---------------------------------------------------------------------------
// TMA z-marching stencil for the FP32 direction phase.
//
// Work item = a kTileX x kTileY column of the grid over tma_zl planes.  One
// thread streams plane slabs of r32 and p_old (box kTmaBoxW x kTmaBoxH, x
// from x0 - 4 so that every copy starts on a 16-byte boundary; out-of-box
// elements are filled with zeros by the copy engine) into a ring of
// kTmaStages shared-memory stages with cp.async.bulk.tensor, each stage
// completing on its own mbarrier.  All threads compute plane k from the
// slabs of planes k-1, k, k+1 while planes k+2.. are in flight; the stage of
// plane k-1 is refilled once every thread is past the block barrier.  Every
// mbarrier wait is bounded (kTmaWaitNs); a give-up records
// CFD_ERR_TIMEOUT.  Each call issues and consumes the same planes, so no
// copy is in flight when it returns.
// ---------------------------------------------------------------------------
constexpr int kTmaStages = 4;
constexpr int kTmaSlabP = 416;  // floats per stage slab: 40 x 10 padded to 128-byte multiples
constexpr unsigned long long kTmaWaitNs = 1000000000ull;
static_assert(2 * kTmaStages * kTmaSlabP * 4 <= kTileSlots * 8, "TMA ring must fit in the tile buffer");

struct TmaRing {
  float* sr;        // kTmaStages slabs of r32
  float* sp;        // kTmaStages slabs of p_old
  uint64_t* full;   // one mbarrier per stage
  unsigned int gp;  // planes issued so far (ring position)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
  const unsigned long long t0 = global_ns();
  for (unsigned i = 0;; ++i) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 255u) == 255u && global_ns() - t0 > kTmaWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(float* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_issue_plane(const IrArgs& a, const CUtensorMap* mp, TmaRing& ring, unsigned g,
                                                int x0, int y0, int z) {
  const int s = int(g % kTmaStages);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(&ring.full[s], 2 * kTmaBoxW * kTmaBoxH * 4);
  tma_load_3d(ring.sr + s * kTmaSlabP, &a.map_r32, x0 - 4, y0 - 1, z, &ring.full[s]);
  tma_load_3d(ring.sp + s * kTmaSlabP, mp, x0 - 4, y0 - 1, z, &ring.full[s]);
}

// p_new = r32 + beta p_old (r32 alone on the first iteration), q = A p_new
// (Neumann pressure operator), partial p.q; returns false on a wait timeout.
__device__ bool dir_tma_f32(const IrArgs& a, const CUtensorMap* mp, float beta, bool first, float* pnew, float* q,
                            float& acc, TmaRing& ring, VBlock vb) {
  const int mx = a.g.mx, my = a.g.my, mz = a.g.mz;
  const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
  const int zl = a.tma_zl;
  const int ntx = (mx + kTileX - 1) / kTileX, nty = (my + kTileY - 1) / kTileY, nzc = (mz + zl - 1) / zl;
  const int items = ntx * nty * nzc;
  if (threadIdx.x == 0) asm volatile("fence.proxy.async.global;" ::: "memory");  // generic writes -> TMA reads
  for (int it = vb.bid; it < items; it += vb.nb) {
    const int bx = it % ntx, rest = it / ntx, by = rest % nty, bz = rest / nty;
    const int x0 = bx * kTileX, y0 = by * kTileY, z0 = bz * zl;
    const int z1 = min(z0 + zl, mz);
    const int np = (z1 - z0) + 2;  // planes z0-1 .. z1
    const unsigned base = ring.gp;
    if (threadIdx.x == 0)
      for (int lp = 0; lp < kTmaStages && lp < np; ++lp) tma_issue_plane(a, mp, ring, base + lp, x0, y0, z0 - 1 + lp);
    ring.gp += np;
    for (int lp = 0; lp < 2; ++lp) {
      const unsigned g = base + lp;
      if (!mbar_wait(&ring.full[g % kTmaStages], (g / kTmaStages) & 1u)) {
        atomicCAS(&a.ctrl->error, 0, kErrTimeout);
        return false;
      }
    }
    const int i = x0 + tx, j = y0 + ty;
    for (int kz = 0; kz < z1 - z0; ++kz) {
      const int lp = kz + 1;
      {
        const unsigned g = base + lp + 1;
        if (!mbar_wait(&ring.full[g % kTmaStages], (g / kTmaStages) & 1u)) {
          atomicCAS(&a.ctrl->error, 0, kErrTimeout);
          return false;
        }
      }
      if (i < mx && j < my) {
        const int k = z0 + kz;
        const float* rm = ring.sr + ((base + lp - 1) % kTmaStages) * kTmaSlabP;
        const float* rc = ring.sr + ((base + lp) % kTmaStages) * kTmaSlabP;
        const float* rq = ring.sr + ((base + lp + 1) % kTmaStages) * kTmaSlabP;
        const float* pm = ring.sp + ((base + lp - 1) % kTmaStages) * kTmaSlabP;
        const float* pc_ = ring.sp + ((base + lp) % kTmaStages) * kTmaSlabP;
        const float* pq = ring.sp + ((base + lp + 1) % kTmaStages) * kTmaSlabP;
        const int c = (ty + 1) * kTmaBoxW + (tx + 4);
        auto V = [&](const float* rs, const float* ps, int o) { return first ? rs[o] : fmaf(beta, ps[o], rs[o]); };
        const float pc = V(rc, pc_, c);
        float xm = V(rc, pc_, c - 1), xp = V(rc, pc_, c + 1);
        float ym = V(rc, pc_, c - kTmaBoxW), yp = V(rc, pc_, c + kTmaBoxW);
        float zm = V(rm, pm, c), zp = V(rq, pq, c);
        if (i == 0) xm = pc;
        if (i == mx - 1) xp = pc;
        if (j == 0) ym = pc;
        if (j == my - 1) yp = pc;
        if (k == 0) zm = pc;
        if (k == mz - 1) zp = pc;
        const float y = fmaf(6.f, pc, -(((((xm + xp) + ym) + yp) + zm) + zp));
        const size_t e = idx3(i, j, k, mx, my);
        pnew[e] = pc;
        q[e] = y;
        acc = fmaf(pc, y, acc);
      }
      __syncthreads();  // every thread is past plane lp-1's stage
      const int nxt = lp - 1 + kTmaStages;
      if (threadIdx.x == 0 && nxt < np) tma_issue_plane(a, mp, ring, base + nxt, x0, y0, z0 - 1 + nxt);
    }
  }
  __syncthreads();  // the ring aliases the tile buffer used by later phases
  return true;
}

// ---------------------------------------------------------------------------
// Mixed-precision CG with FP64 refinement (persistent; the pressure matrix,
// or a velocity matrix of the diffusion substep: a.kind, a.c).
//
// One conjugate-gradient recurrence runs in FP32: the search direction p,
// the operator output q, the recurrence residual r32 and the correction x32
// are FP32 vectors and the stencil runs in FP32; per-thread partial sums are
// FP32, their cross-thread / cross-block reductions and the CG scalars
// (alpha, beta) are FP64.  Refinement happens in FP64 whenever the FP32
// residual has fallen by the factor delta since the last refinement (or
// claims convergence): x += x32 in FP64, x32 = 0, the true residual
// r = b - A x is recomputed with the FP64 stencil, and r32 = r (mean
// removed for the singular pressure matrix) replaces the recurrence residual; the search direction is kept,
// so the refinement does not restart the Krylov process (the "reliable
// update" form of iterative refinement).  Convergence is only ever declared
// on the FP64 true residual: ||b - A x|| <= rtol ||b||.
// ---------------------------------------------------------------------------
template <bool MULTI>
__global__ void __launch_bounds__(kSolveThreads, 4) ir_kernel(const __grid_constant__ IrArgs a0, const IrArgs* table,
                                                             const int* starts, int nprob) {
  VBlock vb{int(blockIdx.x), int(gridDim.x)};
  const int prob = MULTI ? find_problem(starts, nprob, vb) : 0;
  if (prob < 0) return;
  const IrArgs& a = MULTI ? table[prob] : a0;
  __shared__ __align__(128) double s_raw[kTileSlots];
  __shared__ double s_red[32 * 3];
  __shared__ __align__(8) uint64_t s_full[kTmaStages];
  double* s64 = s_raw;
  float* s32 = reinterpret_cast<float*>(s_raw);
  // the TMA ring aliases the tile buffer: the two are never live at once
  TmaRing ring{s32, s32 + kTmaStages * kTmaSlabP, s_full, 0u};
  if (a.use_tma) {
    if (threadIdx.x == 0) {
      for (int s = 0; s < kTmaStages; ++s) mbar_init(&s_full[s], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }

  const int mx = a.g.mx, my = a.g.my, mz = a.g.mz;
  const size_t n = size_t(mx) * my * mz;
  const TileShape ts = make_tiles(mx, my, mz, a.tz);
  DevSolveStats* st = a.stats;
  unsigned int round = 0;

  auto fail = [&]() {
    if (threadIdx.x == 0) {
      int e = ld_volatile_s32(&a.ctrl->error);
      st->status = e != 0 ? e : kErrTimeout;
    }
  };
  auto allreduce = [&](double (&v)[3], double (&o)[3]) {
    return grid_allreduce<3>(v, o, a.ctrl, a.partials, s_red, a.timeout_ns, round, vb);
  };

  double acc[3], tot[3];

  double shift = 0.0;
  if (a.remove_mean) {
    acc[0] = acc[1] = acc[2] = 0.0;
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) acc[0] += a.b[e];
    if (!allreduce(acc, tot)) return fail();
    shift = tot[0] / double(n);
  }

  // r = b - A x0 (FP64), partials b.b, r.r, sum(r)
  acc[0] = acc[1] = acc[2] = 0.0;
  if (a.zero_x0) {
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) {
      const double bv = a.b[e] - shift;
      if (a.remove_mean) a.b[e] = bv;
      a.x[e] = 0.0;
      a.r[e] = bv;
      acc[0] = fma(bv, bv, acc[0]);
      acc[2] += bv;
    }
    acc[1] = acc[0];
  } else {
    Source<double, kModeResid, 0> src{a.x, nullptr, 0.0, false, nullptr, mx, my, mz};
    Sink<double> out{a.r, nullptr, a.b, shift, a.remove_mean != 0, a.kind, a.c};
    stencil_tiles<double, kModeResid, 0>(ts, src, out, acc, s64, vb);
  }
  if (!allreduce(acc, tot)) return fail();
  const double bb = tot[0];
  double rr = tot[1];  // FP64 true residual norm^2 at the last refinement
  double rsum = tot[2];

  int status = kErrNotConverged, refinements = 0, iters = 0;
  if (bb == 0.0) {
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) a.x[e] = 0.0;
    status = kOk;
    rr = 0.0;
  } else {
    const double tol2 = a.rtol * a.rtol * bb;
    const double delta2 = a.delta * a.delta;
    double rz = 0.0;     // FP32 recurrence residual norm^2 (FP64-reduced)
    double beta = 0.0;
    bool first = true;
    bool refine = true;  // load r32 from the FP64 residual
    int cur = 0;
    while (true) {
      if (refine) {
        if (rr <= tol2) {
          status = kOk;
          break;
        }
        if (refinements > a.max_outer) break;
        // r32 = r - mean(r); x32 = 0; rz = |r32|^2
        const double rmean = a.kind == kOpPressure ? rsum / double(n) : 0.0;  // singular system only
        float f = 0.f;
        for (size_t e = gtid(vb); e < n; e += gstride(vb)) {
          const float v = float(a.r[e] - rmean);
          a.r32[e] = v;
          a.d32[e] = 0.f;
          f = fmaf(v, v, f);
        }
        acc[0] = f;
        acc[1] = acc[2] = 0.0;
        if (!allreduce(acc, tot)) return fail();
        const double rz_new = tot[0];
        if (!first) beta = rz_new / rz;  // keep the direction: beta from the replaced residual
        rz = rz_new;
        refine = false;
      }
      if (iters >= a.max_iters) break;
      const double rz_ref = rr;  // residual level of the last refinement
      // phase D (FP32): p = r32 + beta p, q = A p, partial p.q
      float* pnew = cur ? a.p1_32 : a.p0_32;
      const float* pold = cur ? a.p0_32 : a.p1_32;
      float fa[3] = {0.f, 0.f, 0.f};
      if (a.use_tma) {
        if (!dir_tma_f32(a, cur ? &a.map_p0 : &a.map_p1, float(beta), first, pnew, a.q32, fa[0], ring, vb)) return fail();
      } else {
        Source<float, kModeDir, 0> src{a.r32, pold, float(beta), first, nullptr, mx, my, mz};
        Sink<float> out{a.q32, pnew, nullptr, 0.f, false, a.kind, float(a.c)};
        stencil_tiles<float, kModeDir, 0>(ts, src, out, fa, s32, vb);
      }
      acc[0] = fa[0];
      acc[1] = acc[2] = 0.0;
      if (!allreduce(acc, tot)) return fail();
      const double pq = tot[0];
      if (!(pq > 0.0) || !isfinite(pq)) {
        status = kErrBreakdown;
        break;
      }
      const float alpha = float(rz / pq);
      // phase U (FP32): x32 += alpha p, r32 -= alpha q, partial |r32|^2;
      // 16-byte vector accesses (the FP32 vectors are 256-byte aligned)
      float racc = 0.f;
      {
        const size_t n4 = n / 4;
        const float4* p4 = reinterpret_cast<const float4*>(pnew);
        const float4* q4 = reinterpret_cast<const float4*>(a.q32);
        float4* d4 = reinterpret_cast<float4*>(a.d32);
        float4* r4 = reinterpret_cast<float4*>(a.r32);
        for (size_t e = gtid(vb); e < n4; e += gstride(vb)) {
          const float4 pv = p4[e], qv = q4[e];
          float4 dv = d4[e], rv = r4[e];
          dv.x = fmaf(alpha, pv.x, dv.x);
          dv.y = fmaf(alpha, pv.y, dv.y);
          dv.z = fmaf(alpha, pv.z, dv.z);
          dv.w = fmaf(alpha, pv.w, dv.w);
          rv.x = fmaf(-alpha, qv.x, rv.x);
          rv.y = fmaf(-alpha, qv.y, rv.y);
          rv.z = fmaf(-alpha, qv.z, rv.z);
          rv.w = fmaf(-alpha, qv.w, rv.w);
          d4[e] = dv;
          r4[e] = rv;
          racc = fmaf(rv.x, rv.x, racc);
          racc = fmaf(rv.y, rv.y, racc);
          racc = fmaf(rv.z, rv.z, racc);
          racc = fmaf(rv.w, rv.w, racc);
        }
        for (size_t e = 4 * n4 + gtid(vb); e < n; e += gstride(vb)) {
          a.d32[e] = fmaf(alpha, pnew[e], a.d32[e]);
          const float re = fmaf(-alpha, a.q32[e], a.r32[e]);
          a.r32[e] = re;
          racc = fmaf(re, re, racc);
        }
      }
      acc[0] = racc;
      acc[1] = acc[2] = 0.0;
      if (!allreduce(acc, tot)) return fail();
      const double rz_new = tot[0];
      first = false;
      cur ^= 1;
      ++iters;
      if (rz_new <= delta2 * rz_ref || rz_new <= tol2) {
        // refinement in FP64: x += x32 (x32 cleared: an exit before the next
        // preparation must not add it again), r = b - A x (true residual)
        for (size_t e = gtid(vb); e < n; e += gstride(vb)) {
          a.x[e] += double(a.d32[e]);
          a.d32[e] = 0.f;
        }
        acc[0] = acc[1] = acc[2] = 0.0;
        if (!allreduce(acc, tot)) return fail();  // x complete before the stencil reads it
        {
          Source<double, kModeResid, 0> src{a.x, nullptr, 0.0, false, nullptr, mx, my, mz};
          Sink<double> out{a.r, nullptr, a.b, 0.0, false, a.kind, a.c};
          stencil_tiles<double, kModeResid, 0>(ts, src, out, acc, s64, vb);
        }
        if (!allreduce(acc, tot)) return fail();
        rr = tot[1];
        rsum = tot[2];
        ++refinements;
        refine = true;
        rz = rz;  // beta for the next direction uses the replaced residual
      } else {
        beta = rz_new / rz;
        rz = rz_new;
      }
    }
    if (status != kOk) {
      // leaving early: fold the pending FP32 correction into x and measure
      for (size_t e = gtid(vb); e < n; e += gstride(vb)) a.x[e] += double(a.d32[e]);
      acc[0] = acc[1] = acc[2] = 0.0;
      if (!allreduce(acc, tot)) return fail();
      {
        Source<double, kModeResid, 0> src{a.x, nullptr, 0.0, false, nullptr, mx, my, mz};
        Sink<double> out{a.r, nullptr, a.b, 0.0, false, a.kind, a.c};
        stencil_tiles<double, kModeResid, 0>(ts, src, out, acc, s64, vb);
      }
      if (!allreduce(acc, tot)) return fail();
      rr = tot[1];
      if (rr <= tol2 && status == kErrNotConverged) status = kOk;
    }
  }

  if (a.gauge) {
    acc[0] = acc[1] = acc[2] = 0.0;
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) acc[0] += a.x[e];
    if (!allreduce(acc, tot)) return fail();
    const double sh = a.gauge_value - tot[0] / double(n);
    for (size_t e = gtid(vb); e < n; e += gstride(vb)) a.x[e] += sh;
  }

  if (vb.bid == 0 && threadIdx.x == 0) {
    st->iters = iters;
    st->outer_iters = refinements;
    st->restarts = 0;
    st->status = status;
    st->b_norm = sqrt(bb);
    st->rel_resid = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

}  // namespace

}  // namespace cfd
