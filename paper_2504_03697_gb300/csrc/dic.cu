// DIC-preconditioned CG for the pressure system (Sec. 3.1: PCG with the
// "simplified diagonal-based incomplete Cholesky" preconditioner, the
// paper's default).
//
// DIC of the Neumann matrix A (n_c on the diagonal, -1 per in-box
// neighbour), lexicographic order (x fastest):
//   d_c = n_c - sum over the lower neighbours n (x-1, y-1, z-1) of 1 / d_n,
//   M = (D + L) D^-1 (D + L^T),
// and z = M^-1 r by two triangular sweeps,
//   forward  t_c = (r_c + sum_lower t_n) / d_c,
//   backward z_c = (d_c t_c + sum_upper z_n) / d_c = t_c + (sum_upper z_n) / d_c.
// The set-up stores the reciprocal pivots 1 / d_c (the pivots themselves
// come out bit for bit as with d stored: each d_c uses 1 / d_n of its lower
// neighbours either way), so a sweep costs one FP64 multiply or FMA per cell
// instead of a division, which on GB300's FP64 pipe is a long instruction
// chain and made the single-CTA sweeps divide-bound.
// Cell c depends only on cells of the previous hyperplane i + j + k = const,
// so each sweep runs hyperplane by hyperplane (3N - 2 of them): the same
// values as the sequential recurrence.  The dependence chain is inherently
// sequential, so the sweeps run in one CTA (1024 threads, a block barrier per
// hyperplane) -- the cost that makes DIC slow on a GPU.
//
// The CG loop is host-driven (the preconditioner is a separate launch):
// vector kernels with fixed-order block partials, scalars formed on the
// device, one host read of the residual norm per iteration.

#include <cmath>
#include <cstring>
#include <vector>

#include "cfd_internal.h"
#include "dic.h"

namespace cfd {
namespace {

constexpr int kDicThreads = 1024;
constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 152 * 4;

__device__ __forceinline__ size_t gtid() { return size_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride() { return size_t(gridDim.x) * blockDim.x; }

// Cells of hyperplane L: (i, j, k) with i = L - j - k; thread loop over
// the (j, k) pairs whose i falls inside the grid.
template <typename F>
__device__ __forceinline__ void for_hyperplane(GridDims g, int L, F&& f) {
  const int kmin = max(0, L - (g.mx - 1) - (g.my - 1)), kmax = min(g.mz - 1, L);
  const int nk = kmax - kmin + 1;
  if (nk <= 0) return;
  const int pairs = nk * g.my;
  for (int q = threadIdx.x; q < pairs; q += blockDim.x) {
    const int k = kmin + q / g.my, j = q % g.my;
    const int i = L - j - k;
    if (i >= 0 && i < g.mx) f(i, j, k);
  }
}

// inv_d <- 1 / d (the reciprocal DIC pivots)
__global__ void __launch_bounds__(kDicThreads) dic_setup_kernel(GridDims g, double* inv_d) {
  const int levels = g.mx + g.my + g.mz - 2;
  const size_t sx = 1, sy = size_t(g.mx), sz = size_t(g.mx) * g.my;
  for (int L = 0; L < levels; ++L) {
    for_hyperplane(g, L, [&](int i, int j, int k) {
      const size_t c = (size_t(k) * g.my + j) * g.mx + i;
      const double n = double((i > 0) + (i < g.mx - 1) + (j > 0) + (j < g.my - 1) + (k > 0) + (k < g.mz - 1));
      // lower neighbours in increasing index order (z, then y, then x)
      double s = 0.0;
      if (k > 0) s += inv_d[c - sz];
      if (j > 0) s += inv_d[c - sy];
      if (i > 0) s += inv_d[c - sx];
      inv_d[c] = 1.0 / (n - s);
    });
    __syncthreads();
  }
}

// z = M^-1 r (t: forward-sweep scratch; inv_d: the reciprocal pivots)
__global__ void __launch_bounds__(kDicThreads) dic_apply_kernel(GridDims g, const double* inv_d, const double* r,
                                                                double* t, double* z) {
  const int levels = g.mx + g.my + g.mz - 2;
  const size_t sy = size_t(g.mx), sz = size_t(g.mx) * g.my;
  for (int L = 0; L < levels; ++L) {
    for_hyperplane(g, L, [&](int i, int j, int k) {
      const size_t c = (size_t(k) * g.my + j) * g.mx + i;
      double s = r[c];
      if (k > 0) s += t[c - sz];
      if (j > 0) s += t[c - sy];
      if (i > 0) s += t[c - 1];
      t[c] = s * inv_d[c];
    });
    __syncthreads();
  }
  for (int L = levels - 1; L >= 0; --L) {
    for_hyperplane(g, L, [&](int i, int j, int k) {
      const size_t c = (size_t(k) * g.my + j) * g.mx + i;
      double s = 0.0;
      if (i < g.mx - 1) s += z[c + 1];
      if (j < g.my - 1) s += z[c + sy];
      if (k < g.mz - 1) s += z[c + sz];
      z[c] = fma(s, inv_d[c], t[c]);
    });
    __syncthreads();
  }
}

// ---- vector kernels ----------------------------------------------------------

struct Scalars {
  double rz, alpha, beta, rr, pq, bb, mean;
  int flag;  // 1: p.q <= 0 or non-finite; 2: z.r <= 0 or non-finite
  int pad;
};

// partials[block] = sum a.b (sum of a when b is null), partials[nb + block] = sum a.c (c non-null)
__global__ void __launch_bounds__(kVecThreads) dot_kernel(const double* a, const double* b, const double* c, size_t n,
                                                          double* partials) {
  __shared__ double sh[2][kVecThreads / 32];
  double s0 = 0.0, s1 = 0.0;
  for (size_t e = gtid(); e < n; e += gstride()) {
    s0 = fma(a[e], b ? b[e] : 1.0, s0);
    if (c) s1 = fma(a[e], c[e], s1);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = s0;
    sh[1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) {
      t0 += sh[0][w];
      t1 += sh[1][w];
    }
    partials[blockIdx.x] = t0;
    partials[gridDim.x + blockIdx.x] = t1;
  }
}

__device__ double block_sum(const double* partials, int nb) {
  __shared__ double sh[kVecThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += kVecThreads) s += partials[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kVecThreads / 2; o > 0; o >>= 1) {
    if (int(threadIdx.x) < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

enum ScalarOp : int { kMean = 0, kBB = 1, kRZ = 2, kAlpha = 3, kRR = 4, kBeta = 5 };

__global__ void __launch_bounds__(kVecThreads) scalar_kernel(int op, const double* partials, int nb, size_t n,
                                                             Scalars* sc) {
  const double s0 = block_sum(partials, nb);
  if (threadIdx.x != 0) return;
  switch (op) {
    case kMean: sc->mean = s0 / double(n); break;
    case kBB: sc->bb = s0; sc->rr = s0; break;
    case kRZ:
      sc->rz = s0;
      if (!(s0 > 0.0) || !isfinite(s0)) sc->flag = 2;
      break;
    case kAlpha:
      sc->pq = s0;
      if (!(s0 > 0.0) || !isfinite(s0)) {
        sc->flag = 1;
        sc->alpha = 0.0;
      } else {
        sc->alpha = sc->rz / s0;
      }
      break;
    case kRR: sc->rr = s0; break;
    case kBeta:
      // Fletcher-Reeves with a fixed SPD preconditioner: beta = rz_new / rz
      if (!(s0 > 0.0) || !isfinite(s0)) {
        sc->flag = 2;
        sc->beta = 0.0;
      } else {
        sc->beta = s0 / sc->rz;
        sc->rz = s0;
      }
      break;
  }
}

__global__ void sub_mean_kernel(double* b, size_t n, const Scalars* sc) {
  const double m = sc->mean;
  for (size_t e = gtid(); e < n; e += gstride()) b[e] -= m;
}

__global__ void copy_kernel(const double* a, double* b, size_t n) {
  for (size_t e = gtid(); e < n; e += gstride()) b[e] = a[e];
}

__global__ void zero_kernel(double* a, size_t n) {
  for (size_t e = gtid(); e < n; e += gstride()) a[e] = 0.0;
}

// r = b - t
__global__ void residual_kernel(const double* b, const double* t, size_t n, double* r) {
  for (size_t e = gtid(); e < n; e += gstride()) r[e] = b[e] - t[e];
}

// x += alpha p; r -= alpha q; partials of r.r
__global__ void __launch_bounds__(kVecThreads) update_kernel(double* x, double* r, const double* p, const double* q,
                                                             size_t n, const Scalars* sc, double* partials) {
  __shared__ double sh[kVecThreads / 32];
  const double al = sc->alpha;
  double s = 0.0;
  for (size_t e = gtid(); e < n; e += gstride()) {
    x[e] = fma(al, p[e], x[e]);
    const double re = fma(-al, q[e], r[e]);
    r[e] = re;
    s = fma(re, re, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) t += sh[w];
    partials[blockIdx.x] = t;
  }
}

// p = z + beta p (p = z on a restart)
__global__ void direction_kernel(const double* z, double* p, size_t n, const Scalars* sc, int restart) {
  const double be = restart ? 0.0 : sc->beta;
  for (size_t e = gtid(); e < n; e += gstride()) p[e] = restart ? z[e] : fma(be, p[e], z[e]);
}

// x += shift (gauge)
__global__ void shift_kernel(double* x, size_t n, const Scalars* sc, double target) {
  const double sh = target - sc->mean;
  for (size_t e = gtid(); e < n; e += gstride()) x[e] += sh;
}

int grid_for(size_t n) {
  size_t b = (n + kVecThreads - 1) / kVecThreads;
  if (b > size_t(kVecBlocks)) b = kVecBlocks;
  return int(b < 1 ? 1 : b);
}

}  // namespace

size_t dic_scratch_bytes() { return size_t(2 * kVecBlocks) * 8 + 256; }

cudaError_t launch_dic_setup(GridDims g, double* inv_d, cudaStream_t s, int64_t* launches) {
  dic_setup_kernel<<<1, kDicThreads, 0, s>>>(g, inv_d);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_dic_apply(GridDims g, const double* inv_d, const double* r, double* t, double* z, cudaStream_t s,
                             int64_t* launches) {
  dic_apply_kernel<<<1, kDicThreads, 0, s>>>(g, inv_d, r, t, z);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

// x += target - mean(x) (scratch as for run_dic_pcg)
cudaError_t launch_gauge(GridDims g, double* x, double target, double* scratch, cudaStream_t s, int64_t* launches) {
  const size_t n = g.count();
  Scalars* sc = reinterpret_cast<Scalars*>(scratch + 2 * kVecBlocks);
  dot_kernel<<<kVecBlocks, kVecThreads, 0, s>>>(x, nullptr, nullptr, n, scratch);
  scalar_kernel<<<1, kVecThreads, 0, s>>>(kMean, scratch, kVecBlocks, n, sc);
  shift_kernel<<<grid_for(n), kVecThreads, 0, s>>>(x, n, sc, target);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

// Host-driven DIC-PCG; see dic.h.
cudaError_t run_dic_pcg(const DicArgs& a, cudaStream_t s, int64_t* launches, DicResult* res) {
  const GridDims g = a.g;
  const size_t n = g.count();
  double* parts = a.scratch;
  Scalars* sc = reinterpret_cast<Scalars*>(a.scratch + 2 * kVecBlocks);
  const int nb = kVecBlocks;
  cudaError_t err = cudaSuccess;
  auto ok = [&](cudaError_t e) {
    if (err == cudaSuccess && e != cudaSuccess) err = e;
    return err == cudaSuccess;
  };
  auto launched = [&]() {
    if (launches) *launches += 1;
    return ok(cudaGetLastError());
  };
  Scalars h{};
  auto read = [&]() {
    ok(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
    return ok(cudaStreamSynchronize(s));
  };
  auto dot = [&](const double* x, const double* y, const double* z) {
    dot_kernel<<<nb, kVecThreads, 0, s>>>(x, y, z, n, parts);
    return launched();
  };
  auto scalar = [&](int op) {
    scalar_kernel<<<1, kVecThreads, 0, s>>>(op, parts, nb, n, sc);
    return launched();
  };
  auto apply_a = [&](const double* x, double* y) { return ok(launch_apply_poisson(g, x, y, 0, s, launches)); };
  auto precond = [&]() { return ok(launch_dic_apply(g, a.d, a.r, a.t, a.z, s, launches)); };
  // z = M^-1 r; rz; p = z
  auto restart_dir = [&]() {
    precond();
    dot(a.z, a.r, nullptr);
    scalar(kRZ);
    direction_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.z, a.p, n, sc, 1);
    return launched();
  };

  res->iters = 0;
  res->restarts = 0;
  res->status = kErrNotConverged;
  res->rel_resid = 0.0;
  res->b_norm = 0.0;
  ok(cudaMemsetAsync(sc, 0, sizeof(Scalars), s));
  if (a.setup) ok(launch_dic_setup(g, a.d, s, launches));
  if (a.remove_mean) {
    dot(a.b, nullptr, nullptr);
    scalar(kMean);
    sub_mean_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.b, n, sc);
    launched();
  }
  dot(a.b, a.b, nullptr);
  scalar(kBB);
  if (!read()) return err;
  const double bb = h.bb;
  res->b_norm = std::sqrt(bb);
  if (bb == 0.0) {
    zero_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.x, n);
    launched();
    res->status = kOk;
    return err;
  }
  const double tol2 = a.rtol * a.rtol * bb;
  // r = b - A x0
  if (a.zero_x0) {
    zero_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.x, n);
    launched();
    copy_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.b, a.r, n);
    launched();
  } else {
    apply_a(a.x, a.q);
    residual_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.b, a.q, n, a.r);
    launched();
  }
  dot(a.r, a.r, nullptr);
  scalar(kRR);
  restart_dir();
  int status = kErrNotConverged;
  double rr_true = -1.0;
  while (err == cudaSuccess) {
    if (!read()) break;
    if (h.flag) {
      status = kErrBreakdown;
      break;
    }
    if (h.rr <= tol2) {
      // confirm with the true residual
      apply_a(a.x, a.q);
      residual_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.b, a.q, n, a.r);
      launched();
      dot(a.r, a.r, nullptr);
      scalar(kRR);
      if (!read()) break;
      rr_true = h.rr;
      if (rr_true <= tol2) {
        status = kOk;
        break;
      }
      if (++res->restarts > a.max_restarts) break;
      rr_true = -1.0;
      restart_dir();
      continue;
    }
    if (res->iters >= a.max_iters) break;
    apply_a(a.p, a.q);
    dot(a.p, a.q, nullptr);
    scalar(kAlpha);
    update_kernel<<<nb, kVecThreads, 0, s>>>(a.x, a.r, a.p, a.q, n, sc, parts);
    launched();
    scalar(kRR);
    precond();
    dot(a.z, a.r, nullptr);
    scalar(kBeta);
    direction_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.z, a.p, n, sc, 0);
    launched();
    ++res->iters;
  }
  if (err != cudaSuccess) return err;
  if (rr_true < 0.0) {
    apply_a(a.x, a.q);
    residual_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.b, a.q, n, a.r);
    launched();
    dot(a.r, a.r, nullptr);
    scalar(kRR);
    if (!read()) return err;
    rr_true = h.rr;
  }
  if (a.gauge) {
    dot(a.x, nullptr, nullptr);
    scalar(kMean);
    shift_kernel<<<grid_for(n), kVecThreads, 0, s>>>(a.x, n, sc, a.gauge_value);
    launched();
  }
  res->status = status;
  res->rel_resid = std::sqrt(rr_true / bb);
  return err;
}

}  // namespace cfd
