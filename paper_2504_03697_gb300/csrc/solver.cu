// Matrix-free 7-point operators and the persistent conjugate-gradient solves
// of the cavity projection path (sm_103a).
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
// This keeps the FP64 work at 5 adds + 1-2 FMAs per row, which matters on
// GB300, whose FP64 pipe is far slower than its HBM.
//
// CG layout.  One persistent, cooperatively launched kernel runs the whole
// solve with two grid-wide reductions per iteration:
//   phase D (tiled stencil): p_new = z + beta p_old on a shared-memory tile
//     with halo (z = r, or r / diag for Jacobi), write p_new, q = A p_new,
//     partial p.q;
//   phase U (flat):  x += alpha p_new, r -= alpha q, partial r.r (and r.z).
// The x/y halo lives in shared memory; each thread marches along z keeping
// the z-1 / z / z+1 values in registers.  Reductions are deterministic (see
// cfd_common.cuh), so a solve is bitwise reproducible run to run.

#include <cmath>

#include "cfd_internal.h"

namespace cfd {

namespace {

constexpr int kModeApply = 0;  // y = A x
constexpr int kModeResid = 1;  // r = (b - shift) - A x, partials b.b, r.r, r.z
constexpr int kModeDir = 2;    // p_new = z + beta p_old; q = A p_new; partial p.q

constexpr int kTileW = kTileX + 2;
constexpr int kTileH = kTileY + 2;

template <typename T>
__device__ __forceinline__ T stencil_row(int kind, T c, int i, int j, int k, int mx, int my, int mz, T xc,
                                         T xm, T xp, T ym, T yp, T zm, T zp) {
  if (kind == kOpPressure) {
    if (i == 0) xm = xc;
    if (i == mx - 1) xp = xc;
    if (j == 0) ym = xc;
    if (j == my - 1) yp = xc;
    if (k == 0) zm = xc;
    if (k == mz - 1) zp = xc;
    return T(6) * xc - (((((xm + xp) + ym) + yp) + zm) + zp);
  }
  const int comp = kind - 1;
  const bool wall_row = (comp == 0) ? (i == 0 || i == mx - 1)
                                    : (comp == 1) ? (j == 0 || j == my - 1) : (k == 0 || k == mz - 1);
  if (wall_row) return T(0);
  const T g = -xc;
  if (comp != 0) {
    if (i == 0) xm = g;
    if (i == mx - 1) xp = g;
  }
  if (comp != 1) {
    if (j == 0) ym = g;
    if (j == my - 1) yp = g;
  }
  if (comp != 2) {
    if (k == 0) zm = g;
    if (k == mz - 1) zp = g;
  }
  const T lap = T(6) * xc - (((((xm + xp) + ym) + yp) + zm) + zp);
  return xc + c * lap;
}

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
  __device__ __forceinline__ int count() const { return ntx * nty * ntz; }
};

__device__ __forceinline__ TileShape make_tiles(int mx, int my, int mz, int tz) {
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
  T* y;          // apply: y; resid: r; dir: q
  T* pnew;       // dir
  T* b;          // resid: right-hand side (read, optionally rewritten)
  T bshift;      // resid: subtracted from b
  bool write_b;  // resid
  int kind;
  T c;
};

// Tiled 7-point pass over all tiles owned by this block (tile t -> block
// t mod gridDim.x).  acc[0..2] receive the partial sums of the mode.
template <typename T, int MODE, int PRECOND>
__device__ void stencil_tiles(const TileShape& ts, const Source<T, MODE, PRECOND>& src, const Sink<T>& out,
                              double (&acc)[3], T* s) {
  const int tx = threadIdx.x % kTileX, ty = threadIdx.x / kTileX;
  const int mx = ts.mx, my = ts.my, mz = ts.mz;
  const int ntiles = ts.count();
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int bx = t % ts.ntx;
    const int rest = t / ts.ntx;
    const int by = rest % ts.nty;
    const int bz = rest / ts.nty;
    const int i = bx * kTileX + tx, j = by * kTileY + ty;
    const int z0 = bz * ts.tz, z1 = min(z0 + ts.tz, mz);
    const bool inx = i < mx, iny = j < my, own = inx && iny;
    T pm = T(0), pc = T(0), pn = T(0);
    if (own) {
      pc = src(idx3(i, j, z0, mx, my), i, j, z0);
      if (z0 > 0) pm = src(idx3(i, j, z0 - 1, mx, my), i, j, z0 - 1);
    }
    for (int k = z0; k < z1; ++k) {
      pn = (own && k + 1 < mz) ? src(idx3(i, j, k + 1, mx, my), i, j, k + 1) : T(0);
      if (ty == 0) s[tx + 1] = (inx && j > 0) ? src(idx3(i, j - 1, k, mx, my), i, j - 1, k) : T(0);
      if (ty == kTileY - 1)
        s[(kTileY + 1) * kTileW + tx + 1] = (inx && j + 1 < my) ? src(idx3(i, j + 1, k, mx, my), i, j + 1, k) : T(0);
      if (tx == 0) s[(ty + 1) * kTileW] = (iny && i > 0) ? src(idx3(i - 1, j, k, mx, my), i - 1, j, k) : T(0);
      if (tx == kTileX - 1)
        s[(ty + 1) * kTileW + kTileX + 1] = (iny && i + 1 < mx) ? src(idx3(i + 1, j, k, mx, my), i + 1, j, k) : T(0);
      s[(ty + 1) * kTileW + tx + 1] = pc;
      __syncthreads();
      if (own) {
        const T xm = s[(ty + 1) * kTileW + tx];
        const T xp = s[(ty + 1) * kTileW + tx + 2];
        const T ym = s[ty * kTileW + tx + 1];
        const T yp = s[(ty + 2) * kTileW + tx + 1];
        const T y = stencil_row<T>(out.kind, out.c, i, j, k, mx, my, mz, pc, xm, xp, ym, yp, pm, pn);
        const size_t e = idx3(i, j, k, mx, my);
        if (MODE == kModeApply) {
          out.y[e] = y;
        } else if (MODE == kModeDir) {
          out.pnew[e] = pc;
          out.y[e] = y;
          acc[0] = fma(double(pc), double(y), acc[0]);
        } else {  // resid
          T bv = out.b[e] - out.bshift;
          if (out.write_b) out.b[e] = bv;
          const T r = bv - y;
          out.y[e] = r;
          acc[0] = fma(double(bv), double(bv), acc[0]);
          acc[1] = fma(double(r), double(r), acc[1]);
          if (PRECOND) acc[2] = fma(double(r) * double(r), double(src.invd[neighbour_count(i, j, k, mx, my, mz)]), acc[2]);
        }
      }
      __syncthreads();
      pm = pc;
      pc = pn;
    }
  }
}

__device__ __forceinline__ size_t gtid() { return size_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride() { return size_t(gridDim.x) * blockDim.x; }

// ---------------------------------------------------------------------------
// Persistent FP64 (P)CG.  PRECOND: 0 none, 1 Jacobi.
// ---------------------------------------------------------------------------
template <int PRECOND>
__global__ void __launch_bounds__(kSolveThreads) cg_fp64_kernel(CgArgs a) {
  __shared__ double s_tile[kTileH * kTileW];
  __shared__ double s_red[32 * 3];
  __shared__ double s_invd[8];
  if (threadIdx.x < 8) s_invd[threadIdx.x] = threadIdx.x == 0 ? 0.0 : 1.0 / double(threadIdx.x);
  __syncthreads();

  const int mx = a.g.mx, my = a.g.my, mz = a.g.mz;
  const size_t n = size_t(mx) * my * mz;
  const TileShape ts = make_tiles(mx, my, mz, a.tz);
  const double c = a.c;
  DevSolveStats* st = a.stats;

  auto fail = [&]() {
    if (threadIdx.x == 0) {
      int e = ld_volatile_s32(&a.ctrl->error);
      st->status = e != 0 ? e : kErrTimeout;
    }
  };

  double acc[3], tot[3];

  // ---- mean of b (pressure systems are only solvable for zero-mean b) ----
  double shift = 0.0;
  if (a.remove_mean) {
    acc[0] = acc[1] = acc[2] = 0.0;
    for (size_t e = gtid(); e < n; e += gstride()) acc[0] += a.b[e];
    if (!grid_allreduce<3>(acc, tot, a.ctrl, a.partials, s_red, a.timeout_ns)) return fail();
    shift = tot[0] / double(n);
  }

  // ---- initial residual r = b - A x0 ----
  acc[0] = acc[1] = acc[2] = 0.0;
  if (a.zero_x0) {
    for (size_t e = gtid(); e < n; e += gstride()) {
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
    stencil_tiles<double, kModeResid, PRECOND>(ts, src, out, acc, s_tile);
  }
  if (!grid_allreduce<3>(acc, tot, a.ctrl, a.partials, s_red, a.timeout_ns)) return fail();
  const double bb = tot[0];
  double rr = tot[1];
  double rz = PRECOND ? tot[2] : tot[1];

  int status = kErrNotConverged, iters = 0, restarts = 0;
  double rr_true = -1.0;
  if (bb == 0.0) {
    for (size_t e = gtid(); e < n; e += gstride()) a.x[e] = 0.0;
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
        stencil_tiles<double, kModeResid, PRECOND>(ts, src, out, acc, s_tile);
        if (!grid_allreduce<3>(acc, tot, a.ctrl, a.partials, s_red, a.timeout_ns)) return fail();
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
        Sink<double> out{a.q, pnew, nullptr, 0.0, false, a.kind, c};
        stencil_tiles<double, kModeDir, PRECOND>(ts, src, out, acc, s_tile);
      }
      if (!grid_allreduce<3>(acc, tot, a.ctrl, a.partials, s_red, a.timeout_ns)) return fail();
      const double pq = tot[0];
      if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rz)) {
        status = kErrBreakdown;
        break;
      }
      const double alpha = rz / pq;
      // phase U: x += alpha p, r -= alpha q, partial r.r (and r.z)
      acc[0] = acc[1] = acc[2] = 0.0;
      for (size_t e = gtid(); e < n; e += gstride()) {
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
      if (!grid_allreduce<3>(acc, tot, a.ctrl, a.partials, s_red, a.timeout_ns)) return fail();
      rr = tot[0];
      const double rz_new = PRECOND ? tot[1] : tot[0];
      beta = rz_new / rz;
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
      stencil_tiles<double, kModeResid, PRECOND>(ts, src, out, acc, s_tile);
      if (!grid_allreduce<3>(acc, tot, a.ctrl, a.partials, s_red, a.timeout_ns)) return fail();
      rr_true = tot[1];
    }
  }

  // ---- gauge: shift x to the requested mean ----
  if (a.gauge) {
    acc[0] = acc[1] = acc[2] = 0.0;
    for (size_t e = gtid(); e < n; e += gstride()) acc[0] += a.x[e];
    if (!grid_allreduce<3>(acc, tot, a.ctrl, a.partials, s_red, a.timeout_ns)) return fail();
    const double sh = a.gauge_value - tot[0] / double(n);
    for (size_t e = gtid(); e < n; e += gstride()) a.x[e] += sh;
  }

  if (blockIdx.x == 0 && threadIdx.x == 0) {
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
  __shared__ double s_tile[kTileH * kTileW];
  const TileShape ts = make_tiles(g.mx, g.my, g.mz, tz);
  double acc[3] = {0.0, 0.0, 0.0};
  Source<double, kModeApply, 0> src{x, nullptr, 0.0, false, nullptr, g.mx, g.my, g.mz};
  Sink<double> out{y, nullptr, nullptr, 0.0, false, kOpPressure, 0.0};
  stencil_tiles<double, kModeApply, 0>(ts, src, out, acc, s_tile);
}

int tiles_of(GridDims g, int tz) {
  return ((g.mx + kTileX - 1) / kTileX) * ((g.my + kTileY - 1) / kTileY) * ((g.mz + tz - 1) / tz);
}

}  // namespace

int cg_max_coresident_blocks(int kind_is_ir) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  (void)kind_is_ir;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_fp64_kernel<0>, kSolveThreads, 0);
  int p1 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, cg_fp64_kernel<1>, kSolveThreads, 0);
  per_sm = per_sm < p1 ? per_sm : p1;
  if (per_sm > 4) per_sm = 4;
  return per_sm * sms;
}

cudaError_t launch_cg(const CgArgs& a, const LaunchGeom& lg, cudaStream_t s, int64_t* launches) {
  const size_t n = a.g.count();
  int blocks = lg.blocks;
  const int tiles = tiles_of(a.g, a.tz);
  const int flat = int((n + kSolveThreads - 1) / kSolveThreads);
  const int want = tiles > flat ? tiles : flat;
  if (blocks > want) blocks = want;
  if (blocks < 1) blocks = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t err;
  if (a.precond) err = cudaLaunchKernelEx(&cfg, cg_fp64_kernel<1>, a);
  else err = cudaLaunchKernelEx(&cfg, cg_fp64_kernel<0>, a);
  if (launches) *launches += 1;
  return err;
}

cudaError_t launch_apply_poisson(GridDims g, const double* x, double* y, int tz, cudaStream_t s,
                                 int64_t* launches) {
  const int tiles = tiles_of(g, tz);
  apply_poisson_kernel<<<tiles, kSolveThreads, 0, s>>>(g, x, y, tz);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_ir(const IrArgs&, const LaunchGeom&, cudaStream_t, int64_t*) {
  return cudaErrorNotSupported;
}

}  // namespace cfd
