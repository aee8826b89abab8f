// Tile-resident single-reduction FP64 CG (sm_103a).
//
// The method of cg1_fp64_kernel (Sec. 3.1 of arXiv 2504.03697: CG on the
// matrix-free pressure or velocity operator, FP64 throughout, in the
// single-reduction form of Chronopoulos and Gear), laid out for the grids
// whose kTileX x kTileY x kCgtDepth tiles number at most one per SM.  Every
// block owns one tile for the whole solve and keeps all five CG vectors of
// its cells (x, p, r, w = A r, s = A p) in registers; 256 threads with
// eight cells each along z, or 512 with four.  Only the tile boundary goes through memory: every
// iteration a block publishes r, w and s of its cells, and evaluates the
// next residual on its halo from the values that its neighbours published in
// the previous iteration (the recurrence gives the neighbours' values
// bitwise, so no second grid barrier is needed).  At these sizes the FP64
// pipe bounds the solve on GB300, not memory: what is left per iteration is
// 12 FP64 operations per cell, 2 per halo cell and one grid all-reduce of
// two sums, with the halo loads in flight while the own cells update and the
// x update inside the all-reduce's wait; the scalars of the recurrence are
// formed by one thread per block, since every FP64 operation that all
// threads repeat costs as much as a cell's stencil.

#include "solver_impl.cuh"
#include "solver_kernels.h"

namespace cfd {

namespace {

constexpr int kCgtDepth = kCgtTileDepth;
constexpr int kCgtW = kTileX + 2;
constexpr int kCgtH = kTileY + 2;
constexpr int kCgtD = kCgtDepth + 2;
constexpr int kCgtPlane = kCgtW * kCgtH;
constexpr int kCgtSlots = kCgtPlane * kCgtD;
// halo faces of a tile (edges and corners excluded: the 7-point stencil
// never reads them)
constexpr int kCgtHaloX = 2 * kTileY * kCgtDepth;
constexpr int kCgtHaloY = 2 * kTileX * kCgtDepth;
constexpr int kCgtHaloZ = 2 * kTileX * kTileY;
constexpr int kCgtHalo = kCgtHaloX + kCgtHaloY + kCgtHaloZ;
static_assert(kCgtSlots + 1 < (1 << 12), "halo slot must fit the 12-bit field");

__device__ __forceinline__ int cgt_slot(int lx, int ly, int lz) { return (lz * kCgtH + ly) * kCgtW + lx; }

// Halo slot l of a tile -> tile-local coordinates (0 and W-1 etc. are the
// faces; consecutive l run along x on the y and z faces, so loads coalesce).
__device__ __forceinline__ void cgt_halo_coords(int l, int& lx, int& ly, int& lz) {
  if (l < kCgtHaloX) {
    const int f = l / (kTileY * kCgtDepth), m = l % (kTileY * kCgtDepth);
    lx = f ? kCgtW - 1 : 0;
    ly = 1 + m % kTileY;
    lz = 1 + m / kTileY;
  } else if (l < kCgtHaloX + kCgtHaloY) {
    l -= kCgtHaloX;
    const int f = l / (kTileX * kCgtDepth), m = l % (kTileX * kCgtDepth);
    ly = f ? kCgtH - 1 : 0;
    lx = 1 + m % kTileX;
    lz = 1 + m / kTileX;
  } else {
    l -= kCgtHaloX + kCgtHaloY;
    const int f = l / (kTileX * kTileY), m = l % (kTileX * kTileY);
    lz = f ? kCgtD - 1 : 0;
    lx = 1 + m % kTileX;
    ly = 1 + m / kTileX;
  }
}

// The grid must hold exactly one block per tile (make_tiles(..., kCgtDepth))
// and be co-resident (cooperative launch).  LAYERS thread layers along z:
// kTileX * kTileY * LAYERS threads, kCgtDepth / LAYERS cells each.
template <int LAYERS>
__global__ void __launch_bounds__(kTileX * kTileY * LAYERS, 1) cgt_fp64_kernel(const __grid_constant__ CgArgs a) {
  constexpr int kCgtCells = kCgtDepth / LAYERS;
  constexpr int kCgtThreads = kTileX * kTileY * LAYERS;
  constexpr int kCgtHaloPer = (kCgtHalo + kCgtThreads - 1) / kCgtThreads;
  const VBlock vb{int(blockIdx.x), int(gridDim.x)};
  __shared__ double s_tile[kCgtSlots];
  __shared__ double s_red[32 * 3];
  __shared__ double s_sc[3];  // alpha, beta, 1 if they are usable
  __shared__ double s_tot[2];
  __shared__ int s_ok;

  const int mx = a.g.mx, my = a.g.my, mz = a.g.mz;
  const size_t n = size_t(mx) * my * mz;
  const TileShape ts = make_tiles(mx, my, mz, kCgtDepth);
  const int t = vb.bid;
  const int bx = t % ts.ntx, by = (t / ts.ntx) % ts.nty, bz = t / (ts.ntx * ts.nty);
  const int x0 = bx * kTileX, y0 = by * kTileY, z0 = bz * kCgtDepth;
  const int tx = threadIdx.x % kTileX, ty = (threadIdx.x / kTileX) % kTileY;
  const int zl = threadIdx.x / (kTileX * kTileY);
  const int i = x0 + tx, j = y0 + ty, kb = z0 + zl * kCgtCells;
  int nown = 0;  // own cells (i, j, kb + q), q < nown
  if (i < mx && j < my && kb < mz) nown = min(kCgtCells, mz - kb);
  // a grid of at most one tile per SM holds far fewer than 2^31 cells
  const int plane = mx * my;
  const int e0 = nown > 0 ? int(idx3(i, j, kb, mx, my)) : 0;
  const int c0 = cgt_slot(tx + 1, ty + 1, zl * kCgtCells + 1);

  // this thread's halo slots, packed unsigned: bits 20..31 the shared-memory
  // slot + 1 (0: no slot; slots < kCgtSlots < 4095), bits 0..19 the global
  // index + 1 (0: outside the box, where the row rule substitutes the value;
  // the launcher admits grids of fewer than 2^20 - 1 cells)
  unsigned int hp[kCgtHaloPer];
#pragma unroll
  for (int h = 0; h < kCgtHaloPer; ++h) {
    const int l = int(threadIdx.x) + h * kCgtThreads;
    hp[h] = 0u;
    if (l < kCgtHalo) {
      int lx, ly, lz;
      cgt_halo_coords(l, lx, ly, lz);
      hp[h] = unsigned(cgt_slot(lx, ly, lz) + 1) << 20;
      const int gi = x0 + lx - 1, gj = y0 + ly - 1, gk = z0 + lz - 1;
      if (gi >= 0 && gi < mx && gj >= 0 && gj < my && gk >= 0 && gk < mz)
        hp[h] |= unsigned(idx3(gi, gj, gk, mx, my)) + 1u;
    }
  }
  auto h_slot = [&](int h) { return int(hp[h] >> 20) - 1; };
  auto h_glob = [&](int h) { return int(hp[h] & 0xfffffu) - 1; };

  DevSolveStats* st = a.stats;
  unsigned int round = 0;
  // double-buffered published vectors (selected, not indexed: no local memory)
  auto Rb = [&](int b) { return b ? a.e0 : a.r; };
  auto Wb = [&](int b) { return b ? a.d1 : a.d0; };
  auto Sb = [&](int b) { return b ? a.e1 : a.q; };

  auto fail = [&]() {
    if (threadIdx.x == 0) {
      const int e = ld_volatile_s32(&a.ctrl->error);
      st->status = e != 0 ? e : kErrTimeout;
    }
  };
  // Every call ends with block barriers, which also order this block's
  // shared-memory reads of the tile before the next fill.
  auto allreduce = [&](double (&v)[3], double (&o)[3]) {
    return grid_allreduce<3>(v, o, a.ctrl, a.partials, s_red, a.timeout_ns, round, vb);
  };
  // The iteration's all-reduce of (r.r, w.r): the flat form of
  // grid_allreduce (same partial buffers, counter and summation order, so
  // the two interleave), split at the arrival so that work needing no total
  // overlaps the grid-wide wait.  The completing thread also forms the next
  // alpha and beta (the non-restart form) into s_sc.
  const unsigned int G = unsigned(vb.nb);
  auto arrive2 = [&](double (&v)[2]) -> unsigned int {
    block_reduce<2>(v, s_red);  // ends with a block barrier: this block's stores precede the release
    const unsigned int rd = round++;
    if (threadIdx.x == 0) {
      double* buf = a.partials + size_t(rd & 1u) * G * kMaxPartials;
      buf[size_t(vb.bid) * kMaxPartials + 0] = v[0];
      buf[size_t(vb.bid) * kMaxPartials + 1] = v[1];
      red_add_release_gpu(&a.ctrl->arrive, 1u);
    }
    return rd;
  };
  auto complete2 = [&](unsigned int rd, double g_old, double alpha_old, double (&o)[2]) -> bool {
    if (threadIdx.x == 0) s_ok = wait_counter(a.ctrl, &a.ctrl->arrive, (rd + 1u) * G, a.timeout_ns) ? 1 : 0;
    __syncthreads();
    if (!s_ok) return false;
    if (threadIdx.x < 32) {
      const double* buf = a.partials + size_t(rd & 1u) * G * kMaxPartials;
      double t0 = 0.0, t1 = 0.0;
      for (unsigned int b = threadIdx.x; b < G; b += 32) {
        t0 += __ldcg(&buf[size_t(b) * kMaxPartials + 0]);
        t1 += __ldcg(&buf[size_t(b) * kMaxPartials + 1]);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        t0 += __shfl_down_sync(0xffffffffu, t0, off);
        t1 += __shfl_down_sync(0xffffffffu, t1, off);
      }
      if (threadIdx.x == 0) {
        s_tot[0] = t0;
        s_tot[1] = t1;
        const double be = t0 / g_old;
        const double al = t0 / (t1 - be * t0 / alpha_old);
        s_sc[0] = al;
        s_sc[1] = be;
        s_sc[2] = (al > 0.0) && isfinite(al) && isfinite(be) ? 1.0 : 0.0;
      }
    }
    __syncthreads();
    o[0] = s_tot[0];
    o[1] = s_tot[1];
    return true;
  };
  auto row = [&](int q) -> double {
    const int c = c0 + q * kCgtPlane;
    return stencil_row<double>(a.kind, a.c, i, j, kb + q, mx, my, mz, s_tile[c], s_tile[c - 1], s_tile[c + 1],
                               s_tile[c - kCgtW], s_tile[c + kCgtW], s_tile[c - kCgtPlane], s_tile[c + kCgtPlane]);
  };
  // tile <- own values v, halo read from src (published before the last
  // grid barrier); ends with a block barrier
  auto fill = [&](const double (&v)[kCgtCells], const double* src) {
    double hv[kCgtHaloPer];
#pragma unroll
    for (int h = 0; h < kCgtHaloPer; ++h) hv[h] = h_glob(h) >= 0 ? __ldcg(src + h_glob(h)) : 0.0;
#pragma unroll
    for (int q = 0; q < kCgtCells; ++q)
      if (q < nown) s_tile[c0 + q * kCgtPlane] = v[q];
#pragma unroll
    for (int h = 0; h < kCgtHaloPer; ++h)
      if (h_slot(h) >= 0) s_tile[h_slot(h)] = hv[h];
    __syncthreads();
  };

  double x[kCgtCells], p[kCgtCells], r[kCgtCells], w[kCgtCells], s[kCgtCells];
#pragma unroll
  for (int q = 0; q < kCgtCells; ++q) x[q] = p[q] = r[q] = w[q] = s[q] = 0.0;
  double acc[3], tot[3];

  // ---- mean of b ----
  double shift = 0.0;
  if (a.remove_mean) {
    acc[0] = acc[1] = acc[2] = 0.0;
#pragma unroll
    for (int q = 0; q < kCgtCells; ++q)
      if (q < nown) acc[0] += a.b[e0 + q * plane];
    if (!allreduce(acc, tot)) return fail();
    shift = tot[0] / double(n);
  }

  // ---- r_0 = (b - shift) - A x_0, published in Rb(0); b.b ----
  acc[0] = acc[1] = acc[2] = 0.0;
  if (!a.zero_x0) {
#pragma unroll
    for (int q = 0; q < kCgtCells; ++q)
      if (q < nown) x[q] = a.x[e0 + q * plane];
    fill(x, a.x);
  }
#pragma unroll
  for (int q = 0; q < kCgtCells; ++q) {
    if (q < nown) {
      const int e = e0 + q * plane;
      const double bv = a.b[e] - shift;
      if (a.remove_mean) a.b[e] = bv;
      r[q] = a.zero_x0 ? bv : bv - row(q);
      Rb(0)[e] = r[q];
      acc[0] = fma(bv, bv, acc[0]);
    }
  }
  if (!allreduce(acc, tot)) return fail();
  const double bb = tot[0];

  // true residual b - A x of the x in registers, into w (free until the
  // next apply_dots) and Rb(buf); rr in out; false on a failed all-reduce
  auto true_residual = [&](int buf, double& out) -> bool {
#pragma unroll
    for (int q = 0; q < kCgtCells; ++q)
      if (q < nown) a.x[e0 + q * plane] = x[q];
    acc[0] = acc[1] = acc[2] = 0.0;
    if (!allreduce(acc, tot)) return false;  // every block's x stored
    fill(x, a.x);
#pragma unroll
    for (int q = 0; q < kCgtCells; ++q) {
      w[q] = 0.0;
      if (q < nown) {
        const int e = e0 + q * plane;
        w[q] = a.b[e] - row(q);
        Rb(buf)[e] = w[q];
        acc[0] = fma(w[q], w[q], acc[0]);
      }
    }
    if (!allreduce(acc, tot)) return false;
    out = tot[0];
    return true;
  };
  // w = A r from the r in registers (halo from Rb(buf)), published in
  // Wb(buf); g = r.r, d = w.r
  auto apply_dots = [&](int buf, double& g, double& d) -> bool {
    fill(r, Rb(buf));
    acc[0] = acc[1] = acc[2] = 0.0;
#pragma unroll
    for (int q = 0; q < kCgtCells; ++q) {
      if (q < nown) {
        w[q] = row(q);
        Wb(buf)[e0 + q * plane] = w[q];
        acc[0] = fma(r[q], r[q], acc[0]);
        acc[1] = fma(w[q], r[q], acc[1]);
      }
    }
    if (!allreduce(acc, tot)) return false;
    g = tot[0];
    d = tot[1];
    return true;
  };

  int status = kErrNotConverged, iters = 0, restarts = 0;
  double rr_true = -1.0;
  int cur = 0;
  if (bb == 0.0) {
#pragma unroll
    for (int q = 0; q < kCgtCells; ++q) x[q] = 0.0;
    status = kOk;
    rr_true = 0.0;
  } else {
    const double tol2 = a.rtol * a.rtol * bb;
    double g, d;
    if (!apply_dots(0, g, d)) return fail();
    bool first = true;
    while (true) {
      if (g <= tol2) {
        // the recurrence says converged: confirm with the true residual
        if (!true_residual(cur, rr_true)) return fail();
        if (rr_true <= tol2) {
          status = kOk;
          break;
        }
        if (++restarts > a.max_restarts) break;
        rr_true = -1.0;
#pragma unroll
        for (int q = 0; q < kCgtCells; ++q) r[q] = w[q];
        if (!apply_dots(cur, g, d)) return fail();
        first = true;
      }
      if (iters >= a.max_iters) break;
      // alpha and beta: formed once per block (FP64 divisions are long
      // chains on a slow pipe) by the thread that completed the last
      // all-reduce, or here on the first iteration of a (re)start
      if (first) {
        if (threadIdx.x == 0) {
          const double al = g / d;
          s_sc[0] = al;
          s_sc[1] = 0.0;
          s_sc[2] = (al > 0.0) && isfinite(al) ? 1.0 : 0.0;
        }
        __syncthreads();
      }
      const double alpha = s_sc[0], beta = s_sc[1];
      if (s_sc[2] == 0.0) {
        status = kErrBreakdown;
        break;
      }
      const int nxt = cur ^ 1;
      // halo: the neighbours' next residual, s = w + beta s, r - alpha s,
      // from what they published (loads in flight during the own update)
      double hr[kCgtHaloPer], hw[kCgtHaloPer], hsv[kCgtHaloPer];
#pragma unroll
      for (int h = 0; h < kCgtHaloPer; ++h) {
        hr[h] = hw[h] = hsv[h] = 0.0;
        if (h_glob(h) >= 0) {
          hr[h] = __ldcg(Rb(cur) + h_glob(h));
          hw[h] = __ldcg(Wb(cur) + h_glob(h));
          if (!first) hsv[h] = __ldcg(Sb(cur) + h_glob(h));
        }
      }
#pragma unroll
      for (int q = 0; q < kCgtCells; ++q) {
        if (q < nown) {
          const int e = e0 + q * plane;
          s[q] = first ? w[q] : fma(beta, s[q], w[q]);
          p[q] = first ? r[q] : fma(beta, p[q], r[q]);
          r[q] = fma(-alpha, s[q], r[q]);
          s_tile[c0 + q * kCgtPlane] = r[q];
          Rb(nxt)[e] = r[q];
          Sb(nxt)[e] = s[q];
        }
      }
#pragma unroll
      for (int h = 0; h < kCgtHaloPer; ++h) {
        if (h_slot(h) >= 0) {
          const double se = first ? hw[h] : fma(beta, hsv[h], hw[h]);
          s_tile[h_slot(h)] = fma(-alpha, se, hr[h]);
        }
      }
      __syncthreads();
      double acc2[2] = {0.0, 0.0}, tot2[2];
#pragma unroll
      for (int q = 0; q < kCgtCells; ++q) {
        if (q < nown) {
          w[q] = row(q);
          Wb(nxt)[e0 + q * plane] = w[q];
          acc2[0] = fma(r[q], r[q], acc2[0]);
          acc2[1] = fma(w[q], r[q], acc2[1]);
        }
      }
      const unsigned int rd = arrive2(acc2);
      // x += alpha p while the grid gathers
#pragma unroll
      for (int q = 0; q < kCgtCells; ++q)
        if (q < nown) x[q] = fma(alpha, p[q], x[q]);
      if (!complete2(rd, g, alpha, tot2)) return fail();
      g = tot2[0];
      d = tot2[1];
      first = false;
      cur = nxt;
      ++iters;
    }
    if (rr_true < 0.0) {
      // left without a true-residual check (cap, breakdown, restarts)
      if (!true_residual(cur, rr_true)) return fail();
    }
  }
#pragma unroll
  for (int q = 0; q < kCgtCells; ++q)
    if (q < nown) a.x[e0 + q * plane] = x[q];

  // ---- gauge: shift x to the requested mean ----
  if (a.gauge) {
    acc[0] = acc[1] = acc[2] = 0.0;
#pragma unroll
    for (int q = 0; q < kCgtCells; ++q)
      if (q < nown) acc[0] += x[q];
    if (!allreduce(acc, tot)) return fail();
    const double sh = a.gauge_value - tot[0] / double(n);
#pragma unroll
    for (int q = 0; q < kCgtCells; ++q)
      if (q < nown) a.x[e0 + q * plane] = x[q] + sh;
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

}  // namespace

// One thread layer (256 threads, 8 cells each): at 64^3 the pressure solve
// takes 4.40 ms against 4.95 ms with two layers (512 threads, 4 cells each),
// whose per-thread reduction and scalar work is twice as much per cell.
constexpr int kCgtLayers = 1;
Cg1Kernel cgt_kernel() { return cgt_fp64_kernel<kCgtLayers>; }
int cgt_threads() { return kTileX * kTileY * kCgtLayers; }
int cgt_tiles(GridDims g) { return make_tiles(g.mx, g.my, g.mz, kCgtDepth).count(); }

}  // namespace cfd
