// Stand-alone building blocks of the Krylov iterations (Sec. 3.1, Table 1:
// spmv, dot, vector add / scale), callable one by one so that each can be
// measured against the HBM roofline on its own.  The persistent solvers fuse
// the same arithmetic into their phases; these are separate, streaming
// kernels:
//   * the matrix-free pressure operator in FP32 (the inner operator of the
//     mixed-precision solve), z-marching: each thread walks a column of
//     cells along z keeping the z-1, z, z+1 values in registers; when
//     nx % 4 == 0 it works on float4 with x neighbours exchanged by warp
//     shuffles, else on scalars with x/y neighbours through the L1 cache;
//   * the fused CG update x += alpha p, r -= alpha q returning r.r, in FP64
//     and in FP32 (16-byte vector accesses); the dot product is summed in FP64
//     by warp shuffles, then over the blocks in block order by the block that
//     finishes last, so the result does not depend on scheduling.

#include <cstdint>

#include "../../include/cfd.h"
#include "cfd_internal.h"

namespace cfd {
namespace {

constexpr int kBx = 32, kBy = 8, kZChunk = 32;
constexpr int kVecThreads = 256;

// y = A x (Neumann 7-point, A = n_c on the diagonal, -1 per in-box neighbour)
__global__ void __launch_bounds__(kBx * kBy) apply_f32_kernel(int nx, int ny, int nz, const float* __restrict__ x,
                                                              float* __restrict__ y) {
  const int i = blockIdx.x * kBx + threadIdx.x;
  const int j = blockIdx.y * kBy + threadIdx.y;
  const int k0 = blockIdx.z * kZChunk;
  if (i >= nx || j >= ny || k0 >= nz) return;
  const int k1 = min(k0 + kZChunk, nz);
  const size_t sy = size_t(nx), sz = size_t(nx) * ny;
  size_t c = (size_t(k0) * ny + j) * nx + i;
  float xc = __ldg(x + c);
  float xm = k0 > 0 ? __ldg(x + c - sz) : xc;
#pragma unroll 4
  for (int k = k0; k < k1; ++k, c += sz) {
    const float xp = k < nz - 1 ? __ldg(x + c + sz) : xc;
    const float xw = i > 0 ? __ldg(x + c - 1) : xc;
    const float xe = i < nx - 1 ? __ldg(x + c + 1) : xc;
    const float xs = j > 0 ? __ldg(x + c - sy) : xc;
    const float xn = j < ny - 1 ? __ldg(x + c + sy) : xc;
    y[c] = fmaf(6.f, xc, -(((((xw + xe) + xs) + xn) + xm) + xp));
    xm = xc;
    xc = xp;
  }
}

// Block sum of s, written to partials[blockIdx.x]; the block that finishes
// last (counted on *done) adds the partials in block order, in FP64, writes
// the total to *out and sets *done back to zero.  No block waits for another.
// The same operator on 16-byte vectors (nx % 4 == 0): one warp covers 128
// consecutive x cells of one row as 32 float4; a lane's west and east
// neighbours come from the lanes beside it by shuffles, the warp's two edge
// values by scalar loads.  Three vector loads per four cells instead of
// twenty scalar ones.  Each thread marches ZC planes along z.
template <int ZC>
__global__ void __launch_bounds__(kBx * kBy) apply_f32_vec_kernel(int nx, int ny, int nz, const float* __restrict__ x,
                                                                  float* __restrict__ y) {
  const int nx4 = nx >> 2;
  const int i4 = blockIdx.x * kBx + threadIdx.x;
  const int j = blockIdx.y * kBy + threadIdx.y;
  const int k0 = blockIdx.z * ZC;
  if (j >= ny || k0 >= nz) return;  // uniform over the warp (one row per warp)
  const bool on = i4 < nx4;
  const int lane = threadIdx.x;
  const int k1 = min(k0 + ZC, nz);
  const size_t sy = size_t(nx), sz = size_t(nx) * ny;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  float4* y4 = reinterpret_cast<float4*>(y);
  const size_t sy4 = sy >> 2, sz4 = sz >> 2;
  size_t c4 = (size_t(k0) * ny + j) * nx4 + (on ? i4 : nx4 - 1);  // idle lanes shadow the last column
  const bool has_w = i4 > 0, has_e = i4 + 1 < nx4;
  float4 xc = __ldg(x4 + c4);
  float4 xm = k0 > 0 ? __ldg(x4 + c4 - sz4) : xc;
#pragma unroll
  for (int kk = 0; kk < ZC; ++kk) {
    const int k = k0 + kk;
    if (k >= k1) break;
    const float4 xp = k < nz - 1 ? __ldg(x4 + c4 + sz4) : xc;
    const float4 xs = j > 0 ? __ldg(x4 + c4 - sy4) : xc;
    const float4 xn = j < ny - 1 ? __ldg(x4 + c4 + sy4) : xc;
    float west = __shfl_up_sync(0xffffffffu, xc.w, 1);
    float east = __shfl_down_sync(0xffffffffu, xc.x, 1);
    if (lane == 0) west = has_w ? __ldg(x + 4 * c4 - 1) : xc.x;
    else if (!has_w) west = xc.x;
    if (lane == kBx - 1) east = has_e ? __ldg(x + 4 * c4 + 4) : xc.w;
    else if (!has_e) east = xc.w;
    float4 out;
    out.x = fmaf(6.f, xc.x, -(((((west + xc.y) + xs.x) + xn.x) + xm.x) + xp.x));
    out.y = fmaf(6.f, xc.y, -(((((xc.x + xc.z) + xs.y) + xn.y) + xm.y) + xp.y));
    out.z = fmaf(6.f, xc.z, -(((((xc.y + xc.w) + xs.z) + xn.z) + xm.z) + xp.z));
    out.w = fmaf(6.f, xc.w, -(((((xc.z + east) + xs.w) + xn.w) + xm.w) + xp.w));
    if (on) y4[c4] = out;
    xm = xc;
    xc = xp;
    c4 += sz4;
  }
}

__device__ __forceinline__ void block_reduce_last(double s, double* partials, unsigned* done, double* out) {
  __shared__ double sh[kVecThreads / 32];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) t += sh[w];
    partials[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  const volatile double* vp = partials;
  double t = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) t += vp[b];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) {
    *out = t;
    *done = 0u;
  }
}

__global__ void __launch_bounds__(kVecThreads) update_f64_kernel(size_t n, double alpha, const double* __restrict__ p,
                                                                 const double* __restrict__ q, double* __restrict__ x,
                                                                 double* __restrict__ r, double* partials, unsigned* done, double* rr) {
  double s = 0.0;
  const size_t n2 = n / 2;
  const double2* p2 = reinterpret_cast<const double2*>(p);
  const double2* q2 = reinterpret_cast<const double2*>(q);
  double2* x2 = reinterpret_cast<double2*>(x);
  double2* r2 = reinterpret_cast<double2*>(r);
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n2; e += size_t(gridDim.x) * blockDim.x) {
    const double2 pv = p2[e], qv = q2[e];
    double2 xv = x2[e], rv = r2[e];
    xv.x = fma(alpha, pv.x, xv.x);
    xv.y = fma(alpha, pv.y, xv.y);
    rv.x = fma(-alpha, qv.x, rv.x);
    rv.y = fma(-alpha, qv.y, rv.y);
    x2[e] = xv;
    r2[e] = rv;
    s = fma(rv.x, rv.x, s);
    s = fma(rv.y, rv.y, s);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) {
    const size_t e = n - 1;
    x[e] = fma(alpha, p[e], x[e]);
    r[e] = fma(-alpha, q[e], r[e]);
    s = fma(r[e], r[e], s);
  }
  block_reduce_last(s, partials, done, rr);
}

__global__ void __launch_bounds__(kVecThreads) update_f32_kernel(size_t n, float alpha, const float* __restrict__ p,
                                                                 const float* __restrict__ q, float* __restrict__ x,
                                                                 float* __restrict__ r, double* partials, unsigned* done, double* rr) {
  double s = 0.0;
  const size_t n4 = n / 4;
  const float4* p4 = reinterpret_cast<const float4*>(p);
  const float4* q4 = reinterpret_cast<const float4*>(q);
  float4* x4 = reinterpret_cast<float4*>(x);
  float4* r4 = reinterpret_cast<float4*>(r);
  for (size_t e = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n4; e += size_t(gridDim.x) * blockDim.x) {
    const float4 pv = p4[e], qv = q4[e];
    float4 xv = x4[e], rv = r4[e];
    xv.x = fmaf(alpha, pv.x, xv.x);
    xv.y = fmaf(alpha, pv.y, xv.y);
    xv.z = fmaf(alpha, pv.z, xv.z);
    xv.w = fmaf(alpha, pv.w, xv.w);
    rv.x = fmaf(-alpha, qv.x, rv.x);
    rv.y = fmaf(-alpha, qv.y, rv.y);
    rv.z = fmaf(-alpha, qv.z, rv.z);
    rv.w = fmaf(-alpha, qv.w, rv.w);
    x4[e] = xv;
    r4[e] = rv;
    // four-term partial in FP32 (a handful of terms), accumulated in FP64
    s += double(fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, rv.w * rv.w))));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (size_t e = 4 * n4; e < n; ++e) {
      x[e] = fmaf(alpha, p[e], x[e]);
      r[e] = fmaf(-alpha, q[e], r[e]);
      s += double(r[e]) * double(r[e]);
    }
  }
  block_reduce_last(s, partials, done, rr);
}

// FP64 FMA throughput probe (the peak the FP64 kernels are reported
// against): every thread runs 8 independent chains x <- x a + b of `iters`
// DFMAs each, so that the FP64 pipe, not the FMA latency, bounds the rate;
// each thread stores its sum so that no chain can be dropped.
__global__ void __launch_bounds__(kVecThreads) fp64_fma_probe_kernel(int iters, double a, double b, double* out) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1e-3 * double(threadIdx.x) + double(k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum += x[k];
  out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = sum;
}

constexpr int kMaxBlocks = 2048;  // partial sums held by the scratch

// One resident wave of the update kernels (grid-stride loops), capped by the
// elements: each thread starts with at least four.
template <typename K>
int vec_blocks(size_t n, K kernel) {
  static int wave[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (wave[dev] == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kVecThreads, 0);
    const int w = sms * per_sm;
    wave[dev] = w < 1 ? 1 : (w > kMaxBlocks ? kMaxBlocks : w);
  }
  const size_t b = (n / 4 + kVecThreads - 1) / kVecThreads;
  return int(b > size_t(wave[dev]) ? size_t(wave[dev]) : (b < 1 ? 1 : b));
}

// scratch: kMaxBlocks FP64 partials, then the completion counter
constexpr size_t kScratchBytes = size_t(kMaxBlocks) * sizeof(double) + 16;

unsigned* done_counter(void* scratch) {
  return reinterpret_cast<unsigned*>(static_cast<char*>(scratch) + size_t(kMaxBlocks) * sizeof(double));
}

bool misaligned(const void* a, const void* b, const void* c, const void* d) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c) |
           reinterpret_cast<uintptr_t>(d)) &
          15) != 0;
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" {

int cfd_apply_poisson_f32(int32_t nx, int32_t ny, int32_t nz, const float* x_dev, float* y_dev, cfd_stream_t stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !x_dev || !y_dev)
    return cfd_internal_error(CFD_ERR_INVALID_ARG, "apply_poisson_f32: empty grid or NULL pointer");
  if (ny > 65535 * kBy || nz > 65535 * 2)
    return cfd_internal_error(CFD_ERR_INVALID_ARG, "apply_poisson_f32: grid too large");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (nx % 4 == 0 && !misaligned(x_dev, y_dev, x_dev, y_dev)) {
    // four planes per thread, two where that leaves fewer than two waves of
    // 8 resident blocks on each of 152 SMs (measured best at 64^3..320^3)
    const int nx4 = nx / 4;
    const unsigned gx = unsigned((nx4 + kBx - 1) / kBx), gy = unsigned((ny + kBy - 1) / kBy);
    const unsigned g4 = unsigned((nz + 3) / 4);
    if (size_t(gx) * gy * g4 >= 2 * 152 * 8)
      apply_f32_vec_kernel<4><<<dim3(gx, gy, g4), dim3(kBx, kBy), 0, s>>>(nx, ny, nz, x_dev, y_dev);
    else
      apply_f32_vec_kernel<2><<<dim3(gx, gy, unsigned((nz + 1) / 2)), dim3(kBx, kBy), 0, s>>>(nx, ny, nz, x_dev, y_dev);
  } else {
    const dim3 grid((nx + kBx - 1) / kBx, (ny + kBy - 1) / kBy, (nz + kZChunk - 1) / kZChunk);
    apply_f32_kernel<<<grid, dim3(kBx, kBy), 0, s>>>(nx, ny, nz, x_dev, y_dev);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CFD_OK : cfd_internal_error(CFD_ERR_CUDA, "apply_poisson_f32: %s", cudaGetErrorString(e));
}

size_t cfd_cg_update_scratch_bytes(void) { return kScratchBytes; }

int cfd_probe_fp64_fma(int blocks, int iters, double* out_dev, cfd_stream_t stream) {
  if (blocks < 1 || iters < 1 || !out_dev || (reinterpret_cast<uintptr_t>(out_dev) & 7))
    return cfd_internal_error(CFD_ERR_INVALID_ARG, "probe_fp64_fma: blocks, iters >= 1 and an aligned output");
  fp64_fma_probe_kernel<<<blocks, kVecThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(iters, 0.9999999, 1e-7,
                                                                                             out_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CFD_OK : cfd_internal_error(CFD_ERR_CUDA, "probe_fp64_fma: %s", cudaGetErrorString(e));
}

int cfd_cg_update_f64(size_t n, double alpha, const double* p_dev, const double* q_dev, double* x_dev, double* r_dev,
                      double* rr_dev, void* scratch_dev, cfd_stream_t stream) {
  if (n < 1 || !p_dev || !q_dev || !x_dev || !r_dev || !rr_dev || !scratch_dev ||
      misaligned(p_dev, q_dev, x_dev, r_dev) || misaligned(scratch_dev, scratch_dev, scratch_dev, scratch_dev) ||
      (reinterpret_cast<uintptr_t>(rr_dev) & 7))
    return cfd_internal_error(CFD_ERR_INVALID_ARG, "cg_update_f64: n = 0, NULL or misaligned pointer");
  update_f64_kernel<<<vec_blocks(n, update_f64_kernel), kVecThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, alpha, p_dev, q_dev, x_dev, r_dev, static_cast<double*>(scratch_dev), done_counter(scratch_dev), rr_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CFD_OK : cfd_internal_error(CFD_ERR_CUDA, "cg_update_f64: %s", cudaGetErrorString(e));
}

int cfd_cg_update_f32(size_t n, float alpha, const float* p_dev, const float* q_dev, float* x_dev, float* r_dev,
                      double* rr_dev, void* scratch_dev, cfd_stream_t stream) {
  if (n < 1 || !p_dev || !q_dev || !x_dev || !r_dev || !rr_dev || !scratch_dev ||
      misaligned(p_dev, q_dev, x_dev, r_dev) || misaligned(scratch_dev, scratch_dev, scratch_dev, scratch_dev) ||
      (reinterpret_cast<uintptr_t>(rr_dev) & 7))
    return cfd_internal_error(CFD_ERR_INVALID_ARG, "cg_update_f32: n = 0, NULL or misaligned pointer");
  update_f32_kernel<<<vec_blocks(n, update_f32_kernel), kVecThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, alpha, p_dev, q_dev, x_dev, r_dev, static_cast<double*>(scratch_dev), done_counter(scratch_dev), rr_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CFD_OK : cfd_internal_error(CFD_ERR_CUDA, "cg_update_f32: %s", cudaGetErrorString(e));
}

}  // extern "C"
