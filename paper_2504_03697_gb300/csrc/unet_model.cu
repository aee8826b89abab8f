// U-Net preconditioner model: layer graph, forward / backward, Adam, C-ABI.
//
// Architecture (a reading: the paper names no learned preconditioner; its
// future-work list includes "other preconditioners", Sec. 5):
//   level 0 (N^3):    L0a 3^3 1->16, L0b 3^3 16->16          (skip s0)
//   2x avg pool
//   level 1 (N^3/8):  L1a 3^3 16->32, L1b 3^3 32->32         (skip s1)
//   2x avg pool
//   level 2 (N^3/64): L2a 3^3 32->64, L2b 3^3 64->64
//   nearest 2x up, concat s1: L1c 3^3 (32+64)->32
//   nearest 2x up, concat s0: L0c 3^3 (16+32)->16
//   head 1^3 16->1
// No activation: the target of a preconditioner, A^-1, is linear, and a
// linear U-Net is a learned multigrid-like cycle (restriction by pooling,
// prolongation by up-sampling, learned smoothing convolutions).  Input and
// output are scaled by s = sqrt(V) / ||r|| (the network is linear, so the
// pair (r, e) trains it as (s r, s e)), and the output is projected to zero
// mean (the Neumann null space).
//
// Activations and activation gradients are BF16 octet planes (unet.h); master
// weights, gradients and Adam moments are FP32; the convolutions (forward
// and input gradients) run on the tensor cores (unet.cu); weight gradients
// are FP32 reductions on the CUDA cores, summed in a fixed order.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cfd.h"
#include "cfd_internal.h"
#include "unet.h"

namespace cfd {
namespace {

struct LayerSpec {
  int level;
  int c0, c1, cout, ks;
  bool packed;
};

constexpr int kNumLayers = 9;
constexpr LayerSpec kLayers[kNumLayers] = {
    {0, 1, 0, 16, 3, true},     // L0a  xin -> a0
    {0, 16, 0, 16, 3, false},   // L0b  a0 -> s0
    {1, 16, 0, 32, 3, false},   // L1a  p0 -> a1
    {1, 32, 0, 32, 3, false},   // L1b  a1 -> s1
    {2, 32, 0, 64, 3, false},   // L2a  p1 -> a2
    {2, 64, 0, 64, 3, false},   // L2b  a2 -> s2
    {1, 32, 64, 32, 3, false},  // L1c  s1 + u1 -> d1
    {0, 16, 32, 16, 3, false},  // L0c  s0 + u0 -> d0
    {0, 16, 0, 1, 1, false},    // head d0 -> z
};

int nout_pad(int c) { return c <= 16 ? 16 : (c <= 32 ? 32 : 64); }
int pad16(int c) { return (c + 15) / 16 * 16; }
int taps_of(int ks) { return ks * ks * ks; }

constexpr int kThreads = 256;
constexpr int kWgradChunks = 32;
constexpr int kWgradTcChunks = 160;  // partial-sum rows of the tensor-core weight gradient (>= the SM count)

__device__ __forceinline__ size_t gtid() { return size_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride() { return size_t(gridDim.x) * blockDim.x; }

int grid_for(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 8) b = 152 * 8;
  return int(b < 1 ? 1 : b);
}

// ---- elementwise kernels --------------------------------------------------

// fixed-order sum of nb partials by one block of kThreads threads
__device__ double block_sum(const double* partials, int nb) {
  __shared__ double sh[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += kThreads) s += partials[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (int(threadIdx.x) < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}


// partial sums of r^2 per block (for the input scale)
__global__ void sumsq_kernel(const double* r, size_t n, double* partials) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (size_t e = gtid(); e < n; e += gstride()) acc = fma(r[e], r[e], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < int(blockDim.x / 32); ++w) s += sh[w];
    partials[blockIdx.x] = s;
  }
}

// scale[0] = sqrt(V) / ||r|| (0 if r = 0), fixed-order sum of the partials
// (one block of kThreads threads)
__global__ void __launch_bounds__(kThreads) scale_kernel(const double* partials, int nparts, size_t V, double* scale) {
  const double s = block_sum(partials, nparts);
  if (threadIdx.x == 0) scale[0] = s > 0.0 ? sqrt(double(V) / s) : 0.0;
}

// scale[1] = mean of the head output (one block), for the projection below
__global__ void __launch_bounds__(kThreads) mean_kernel(const double* partials, int nparts, size_t V, double* scale) {
  const double s = block_sum(partials, nparts);
  if (threadIdx.x == 0) scale[1] = s / double(V);
}

__global__ void normalize_kernel(const double* r, size_t n, const double* scale, __nv_bfloat16* out) {
  const double s = scale[0];
  for (size_t e = gtid(); e < n; e += gstride()) out[e] = __float2bfloat16(float(r[e] * s));
}

__global__ void target_kernel(const double* e, size_t n, const double* scale, float* out) {
  const double s = scale[0];
  for (size_t i = gtid(); i < n; i += gstride()) out[i] = float(e[i] * s);
}

// z = out / s with its mean removed (two passes: partial sums, then shift)
__global__ void sum_f32_kernel(const float* z, size_t n, double* partials) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (size_t e = gtid(); e < n; e += gstride()) acc += double(z[e]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < int(blockDim.x / 32); ++w) s += sh[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void denorm_kernel(const float* z, size_t n, const double* scale, double* out) {
  const double sc = scale[0], mean = scale[1];
  const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
  for (size_t e = gtid(); e < n; e += gstride()) out[e] = (double(z[e]) - mean) * inv;
}

// loss = sum (z - t)^2 / V; gz = 2 (z - t) / V (BF16, one channel)
__global__ void loss_kernel(const float* z, const float* t, size_t n, __nv_bfloat16* gz, double* partials) {
  __shared__ double sh[32];
  double acc = 0.0;
  const float k = 2.0f / float(n);
  for (size_t e = gtid(); e < n; e += gstride()) {
    const float d = z[e] - t[e];
    gz[e] = __float2bfloat16(k * d);
    acc = fma(double(d), double(d), acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < int(blockDim.x / 32); ++w) s += sh[w];
    partials[blockIdx.x] = s / double(n);
  }
}

// A-norm loss: d = z - t; loss = d.(A d) / V, gz = 2 A d / V with A the
// Neumann 7-point pressure operator (n_c on the diagonal, -1 per neighbour;
// the operator of cfd_apply_poisson), FP32 stencil, FP64 loss partials.
__global__ void loss_anorm_kernel(const float* z, const float* t, int nx, int ny, int nz, __nv_bfloat16* gz,
                                  double* partials) {
  __shared__ double sh[32];
  const size_t n = size_t(nx) * ny * nz;
  const float k = 2.0f / float(n);
  double acc = 0.0;
  for (size_t e = gtid(); e < n; e += gstride()) {
    const int x = int(e % nx), y = int((e / nx) % ny), zc = int(e / (size_t(nx) * ny));
    const float dc = z[e] - t[e];
    float ad = 0.f;
    auto nbr = [&](size_t f) { ad += dc - (z[f] - t[f]); };
    if (x > 0) nbr(e - 1);
    if (x < nx - 1) nbr(e + 1);
    if (y > 0) nbr(e - nx);
    if (y < ny - 1) nbr(e + nx);
    if (zc > 0) nbr(e - size_t(nx) * ny);
    if (zc < nz - 1) nbr(e + size_t(nx) * ny);
    gz[e] = __float2bfloat16(k * ad);
    acc = fma(double(dc), double(ad), acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < int(blockDim.x / 32); ++w) s += sh[w];
    partials[blockIdx.x] = s / double(n);
  }
}

// Scale-invariant energy-norm loss ("cos"): with a = z.Az, b = z.At, T =
// t.At (FP32 stencils, FP64 sums), L = 1 - b / sqrt(a T), one minus the
// energy-norm cosine of z and t.  Flexible CG is invariant to a positive
// scale of the preconditioner, so only the direction of z is trained; the
// sign is kept (a negative multiple of t would make z.r < 0).  dL/dz =
// (c Az - At) / sqrt(a T) with c = b / a.
__device__ __forceinline__ float neumann_at(const float* f, size_t e, int x, int y, int zc, int nx, int ny, int nz) {
  const float c = f[e];
  float s = 0.f;
  if (x > 0) s += c - f[e - 1];
  if (x < nx - 1) s += c - f[e + 1];
  if (y > 0) s += c - f[e - nx];
  if (y < ny - 1) s += c - f[e + nx];
  if (zc > 0) s += c - f[e - size_t(nx) * ny];
  if (zc < nz - 1) s += c - f[e + size_t(nx) * ny];
  return s;
}

__global__ void cos_dots_kernel(const float* z, const float* t, int nx, int ny, int nz, double* partials) {
  __shared__ double sh[3][32];
  const size_t n = size_t(nx) * ny * nz;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (size_t e = gtid(); e < n; e += gstride()) {
    const int x = int(e % nx), y = int((e / nx) % ny), zc = int(e / (size_t(nx) * ny));
    const float az = neumann_at(z, e, x, y, zc, nx, ny, nz), at = neumann_at(t, e, x, y, zc, nx, ny, nz);
    s0 = fma(double(z[e]), double(az), s0);
    s1 = fma(double(z[e]), double(at), s1);
    s2 = fma(double(t[e]), double(at), s2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = s0;
    sh[1][threadIdx.x >> 5] = s1;
    sh[2][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < int(blockDim.x / 32); ++w) v += sh[threadIdx.x][w];
    partials[size_t(threadIdx.x) * gridDim.x + blockIdx.x] = v;
  }
}

// one block: sc[2] = c, sc[3] = 1 / sqrt(a T); partials[0] = L, partials[1 .. nb) = 0
__global__ void __launch_bounds__(kThreads) cos_finalize_kernel(double* partials, int nb, double* sc) {
  const double a = block_sum(partials, nb), b = block_sum(partials + nb, nb), T = block_sum(partials + 2 * nb, nb);
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) partials[i] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = a > 0.0 && T > 0.0;
    const double c = ok ? b / a : 0.0;
    sc[2] = c;
    sc[3] = ok ? 1.0 / sqrt(a * T) : 0.0;
    partials[0] = ok ? 1.0 - b / sqrt(a * T) : 1.0;
  }
}

__global__ void cos_grad_kernel(const float* z, const float* t, int nx, int ny, int nz, const double* sc,
                                __nv_bfloat16* gz) {
  const size_t n = size_t(nx) * ny * nz;
  const float c = float(sc[2]), k = float(sc[3]);
  for (size_t e = gtid(); e < n; e += gstride()) {
    const int x = int(e % nx), y = int((e / nx) % ny), zc = int(e / (size_t(nx) * ny));
    const float az = neumann_at(z, e, x, y, zc, nx, ny, nz), at = neumann_at(t, e, x, y, zc, nx, ny, nz);
    gz[e] = __float2bfloat16(k * (c * az - at));
  }
}

// Resampling kernels on octet planes (C a multiple of 8): one thread per
// (plane, voxel), 8 channels as one 16-byte vector, FP32 arithmetic.
__device__ __forceinline__ void ld8(const __nv_bfloat16* p, float (&f)[8]) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
  for (int k = 0; k < 8; ++k) f[k] = __bfloat162float(h[k]);
}
__device__ __forceinline__ void st8(__nv_bfloat16* p, const float (&f)[8]) {
  uint4 u;
  __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(&u);
#pragma unroll
  for (int k = 0; k < 8; ++k) h[k] = __float2bfloat16(f[k]);
  *reinterpret_cast<uint4*>(p) = u;
}

// 2x average pooling; fine grid (fx, fy, fz) all even
__global__ void pool2_kernel(const __nv_bfloat16* in, int fx, int fy, int fz, int C, __nv_bfloat16* out) {
  const int cx = fx / 2, cy = fy / 2, cz = fz / 2;
  const size_t nc = size_t(cx) * cy * cz, nf = size_t(fx) * fy * fz;
  const size_t n = nc * size_t(C / 8);
  for (size_t e = gtid(); e < n; e += gstride()) {
    const size_t p = e / nc, v = e % nc;
    const int x = int(v % cx), y = int((v / cx) % cy), z = int(v / (size_t(cx) * cy));
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int d = 0; d < 8; ++d) {
      const int xx = 2 * x + (d & 1), yy = 2 * y + ((d >> 1) & 1), zz = 2 * z + (d >> 2);
      float f[8];
      ld8(in + (p * nf + (size_t(zz) * fy + yy) * fx + xx) * 8, f);
#pragma unroll
      for (int k = 0; k < 8; ++k) s[k] += f[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] *= 0.125f;
    st8(out + e * 8, s);
  }
}

// adjoint of pooling: g_in[fine] += g_out[coarse] / 8
__global__ void pool2_adj_kernel(const __nv_bfloat16* gout, int fx, int fy, int fz, int C, __nv_bfloat16* gin) {
  const int cx = fx / 2, cy = fy / 2, cz = fz / 2;
  const size_t nc = size_t(cx) * cy * cz, nf = size_t(fx) * fy * fz;
  const size_t n = nf * size_t(C / 8);
  for (size_t e = gtid(); e < n; e += gstride()) {
    const size_t p = e / nf, v = e % nf;
    const int x = int(v % fx), y = int((v / fx) % fy), z = int(v / (size_t(fx) * fy));
    const size_t cv = (size_t(z / 2) * cy + y / 2) * cx + x / 2;
    float a[8], b[8];
    ld8(gin + e * 8, a);
    ld8(gout + (p * nc + cv) * 8, b);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] += 0.125f * b[k];
    st8(gin + e * 8, a);
  }
}

// nearest 2x up-sampling to the fine grid
__global__ void up2_kernel(const __nv_bfloat16* in, int fx, int fy, int fz, int C, __nv_bfloat16* out) {
  const int cx = fx / 2, cy = fy / 2, cz = fz / 2;
  const size_t nc = size_t(cx) * cy * cz, nf = size_t(fx) * fy * fz;
  const size_t n = nf * size_t(C / 8);
  for (size_t e = gtid(); e < n; e += gstride()) {
    const size_t p = e / nf, v = e % nf;
    const int x = int(v % fx), y = int((v / fx) % fy), z = int(v / (size_t(fx) * fy));
    const size_t cv = (size_t(z / 2) * cy + y / 2) * cx + x / 2;
    *reinterpret_cast<uint4*>(out + e * 8) = *reinterpret_cast<const uint4*>(in + (p * nc + cv) * 8);
  }
}

// adjoint of up-sampling: g_coarse = sum of the 8 fine children
__global__ void up2_adj_kernel(const __nv_bfloat16* gout, int fx, int fy, int fz, int C, __nv_bfloat16* gin) {
  const int cx = fx / 2, cy = fy / 2, cz = fz / 2;
  const size_t nc = size_t(cx) * cy * cz, nf = size_t(fx) * fy * fz;
  const size_t n = nc * size_t(C / 8);
  for (size_t e = gtid(); e < n; e += gstride()) {
    const size_t p = e / nc, v = e % nc;
    const int x = int(v % cx), y = int((v / cx) % cy), z = int(v / (size_t(cx) * cy));
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int d = 0; d < 8; ++d) {
      const int xx = 2 * x + (d & 1), yy = 2 * y + ((d >> 1) & 1), zz = 2 * z + (d >> 2);
      float f[8];
      ld8(gout + (p * nf + (size_t(zz) * fy + yy) * fx + xx) * 8, f);
#pragma unroll
      for (int k = 0; k < 8; ++k) s[k] += f[k];
    }
    st8(gin + e * 8, s);
  }
}

// ---- first layer and head on the CUDA cores -------------------------------
// The first layer (1 -> 16 channels, 27 taps) and the 1x1x1 head (16 -> 1)
// are too narrow to be tensor-core contractions: FP32 FMAs over the
// BF16-rounded weights, summed sequentially in tap / channel order.

// a0 = conv3x3x3(xin) + b: xin [V] BF16, w packed [16][32] BF16 (taps 0..26),
// out 16 channels as 2 octet planes.
__global__ void first_layer_kernel(const __nv_bfloat16* xin, int nx, int ny, int nz, const __nv_bfloat16* w,
                                   const float* bias, __nv_bfloat16* out) {
  // weights as 4 float4 per tap: one 16-byte shared load per 4 FMAs
  __shared__ float4 ws[27][4];
  __shared__ float bs[16];
  for (int i = threadIdx.x; i < 27 * 16; i += blockDim.x)
    reinterpret_cast<float*>(&ws[i / 16][0])[i % 16] = __bfloat162float(w[(i % 16) * 32 + i / 16]);
  if (threadIdx.x < 16) bs[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const size_t V = size_t(nx) * ny * nz;
  for (size_t v = gtid(); v < V; v += gstride()) {
    const unsigned vu = unsigned(v), row = vu / unsigned(nx);  // grids below 2^32 voxels
    const int x = int(vu - row * unsigned(nx)), z = int(row / unsigned(ny)), y = int(row - unsigned(z) * unsigned(ny));
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.f;
    int tap = 0;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx, ++tap) {
          const int xx = x + dx, yy = y + dy, zz = z + dz;
          if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
          const float xv = __bfloat162float(xin[(size_t(zz) * ny + yy) * nx + xx]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 wq = ws[tap][q];
            acc[4 * q] = fmaf(wq.x, xv, acc[4 * q]);
            acc[4 * q + 1] = fmaf(wq.y, xv, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(wq.z, xv, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(wq.w, xv, acc[4 * q + 3]);
          }
        }
    float o[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = acc[8 * h + k] + bs[8 * h + k];
      st8(out + (size_t(h) * V + v) * 8, o);
    }
  }
}

// z = w . d0 + b (FP32 [V]); d0 16 channels in 2 octet planes, w = row 0 of
// the head's [1][16][16] BF16 forward weights.
__global__ void head_kernel(const __nv_bfloat16* d0, size_t V, const __nv_bfloat16* w, const float* bias, float* z) {
  float wv[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) wv[c] = __bfloat162float(w[c]);
  const float b = bias[0];
  for (size_t v = gtid(); v < V; v += gstride()) {
    float a[8], c8[8];
    ld8(d0 + v * 8, a);
    ld8(d0 + (V + v) * 8, c8);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s = fmaf(wv[k], a[k], s);
#pragma unroll
    for (int k = 0; k < 8; ++k) s = fmaf(wv[8 + k], c8[k], s);
    z[v] = s + b;
  }
}

// input gradient of the head: g_d0[v][c] = w[c] gz[v] (one exact product,
// rounded to BF16), w from the forward weights.
__global__ void head_dgrad_kernel(const __nv_bfloat16* gz, size_t V, const __nv_bfloat16* w, __nv_bfloat16* gd0) {
  float wv[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) wv[c] = __bfloat162float(w[c]);
  for (size_t v = gtid(); v < V; v += gstride()) {
    const float g = __bfloat162float(gz[v]);
    float o[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = wv[8 * h + k] * g;
      st8(gd0 + (size_t(h) * V + v) * 8, o);
    }
  }
}

// ---- weight gradients (FP32, CUDA cores, fixed-order chunk reduction) ------

struct WgradArgs {
  int nx, ny, nz;
  const __nv_bfloat16* src0;
  int c0;
  const __nv_bfloat16* src1;
  int c1;
  int ks;
  const __nv_bfloat16* g;  // [V][cout]
  int cout;
  float* partial;          // [chunks][taps][cout][cin]
  float* bias_partial;     // [chunks][cout]
};

// grid (chunks, taps); each thread owns up to 16 (co, ci) pairs
__global__ void __launch_bounds__(kThreads) wgrad_kernel(const WgradArgs a) {
  __shared__ float gs[32][64];
  __shared__ float xs[32][96];
  const int tap = blockIdx.y, chunk = blockIdx.x;
  const int cin = a.c0 + a.c1;
  const int P = a.cout * cin;
  const size_t V = size_t(a.nx) * a.ny * a.nz;
  const size_t per = (V + gridDim.x - 1) / gridDim.x;
  const size_t v0 = size_t(chunk) * per, v1 = min(V, v0 + per);
  int dx = 0, dy = 0, dz = 0;
  if (a.ks == 3) {
    dx = tap % 3 - 1;
    dy = (tap / 3) % 3 - 1;
    dz = tap / 9 - 1;
  }
  float acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.f;
  float bacc = 0.f;
  __shared__ long long s_nb[32];
  for (size_t vb = v0; vb < v1; vb += 32) {
    if (threadIdx.x < 32) {
      const size_t v = vb + threadIdx.x;
      long long nb = -1;
      if (v < v1) {
        const int x = int(v % a.nx) + dx, y = int((v / a.nx) % a.ny) + dy, z = int(v / (size_t(a.nx) * a.ny)) + dz;
        if (x >= 0 && x < a.nx && y >= 0 && y < a.ny && z >= 0 && z < a.nz) nb = (long long)((size_t(z) * a.ny + y) * a.nx + x);
      }
      s_nb[threadIdx.x] = nb;
    }
    // output gradient rows: one 16-byte octet per work item (C >= 8), else elements
    if (a.cout >= 8) {
      for (int i = threadIdx.x; i < 32 * (a.cout / 8); i += kThreads) {
        const int vv = i % 32, q = i / 32;
        const size_t v = vb + vv;
        float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (v < v1) ld8(a.g + (size_t(q) * V + v) * 8, f);
#pragma unroll
        for (int k = 0; k < 8; ++k) gs[vv][8 * q + k] = f[k];
      }
    } else {
      for (int i = threadIdx.x; i < 32 * a.cout; i += kThreads) {
        const int vv = i % 32, co = i / 32;
        const size_t v = vb + vv;
        gs[vv][co] = v < v1 ? __bfloat162float(a.g[oct_index(v, co, a.cout, V)]) : 0.f;
      }
    }
    __syncthreads();
    const int oct0 = a.c0 >= 8 ? a.c0 / 8 : 0;
    if (a.c0 >= 8) {
      for (int i = threadIdx.x; i < 32 * (cin / 8); i += kThreads) {
        const int vv = i % 32, q = i / 32;
        const long long nb = s_nb[vv];
        float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (nb >= 0) {
          if (q < oct0) ld8(a.src0 + (size_t(q) * V + size_t(nb)) * 8, f);
          else ld8(a.src1 + (size_t(q - oct0) * V + size_t(nb)) * 8, f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) xs[vv][8 * q + k] = f[k];
      }
    } else {
      for (int i = threadIdx.x; i < 32 * cin; i += kThreads) {
        const int vv = i % 32, ci = i / 32;
        const long long nb = s_nb[vv];
        xs[vv][ci] = nb >= 0 ? __bfloat162float(a.src0[oct_index(size_t(nb), ci, a.c0, V)]) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int p = threadIdx.x + k * kThreads;
      if (p < P) {
        const int co = p / cin, ci = p % cin;
        float s = acc[k];
        for (int vv = 0; vv < 32; ++vv) s = fmaf(gs[vv][co], xs[vv][ci], s);
        acc[k] = s;
      }
    }
    if (tap == 0 && threadIdx.x < a.cout)
      for (int vv = 0; vv < 32; ++vv) bacc += gs[vv][threadIdx.x];
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int p = threadIdx.x + k * kThreads;
    if (p < P) a.partial[(size_t(chunk) * gridDim.y + tap) * P + p] = acc[k];
  }
  if (tap == 0 && threadIdx.x < a.cout) a.bias_partial[size_t(chunk) * a.cout + threadIdx.x] = bacc;
}

// Weight gradients of the two narrow layers, as voxel reductions (memory
// bound; no contraction worth the tensor cores):
//   first layer  dW[t][co] = sum_v g[v][co] x[v + s_t]   (one input channel)
//   head         dW[0][ci] = sum_v g[v] d[v][ci]          (one output channel)
// Block (chunk, group) sums a contiguous voxel range; per-thread FP32 sums,
// then a fixed-order block reduction, so the result does not depend on
// scheduling.  Partials in the [chunk][taps][cout][cin] layout of
// wgrad_reduce_kernel; bias partials [chunk][cout] from group 0.
constexpr int kNarrowChunks = 64;

template <int K>
__device__ __forceinline__ void block_sum_store(float (&v)[K], float* out) {
  __shared__ float sh[kThreads / 32][K];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[wid][k] = x;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    float x = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) x += sh[w][k];
    out[k] = x;
  }
  __syncthreads();
}

// grid (chunks, 9): group = the (dy, dz) of three taps dx = -1, 0, 1; x BF16
// [V] (one channel), g 16 channels in two octet planes
__global__ void __launch_bounds__(kThreads) wgrad_first_kernel(const __nv_bfloat16* x, const __nv_bfloat16* g, int nx,
                                                               int ny, int nz, float* partial, float* bias_partial) {
  const int chunk = blockIdx.x, grp = blockIdx.y;
  const int dy = grp % 3 - 1, dz = grp / 3 - 1;
  const size_t V = size_t(nx) * ny * nz;
  const size_t per = (V + gridDim.x - 1) / gridDim.x;
  const size_t v0 = size_t(chunk) * per, v1 = min(V, v0 + per);
  float acc[3][16], bacc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    acc[0][k] = acc[1][k] = acc[2][k] = 0.f;
    bacc[k] = 0.f;
  }
  for (size_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const int i = int(v % nx), j = int((v / nx) % ny), k = int(v / (size_t(nx) * ny));
    float glo[8], ghi[8], gv[16];
    ld8(g + v * 8, glo);
    ld8(g + (V + v) * 8, ghi);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      gv[c] = glo[c];
      gv[8 + c] = ghi[c];
    }
    const int jj = j + dy, kk = k + dz;
    float xs[3] = {0.f, 0.f, 0.f};
    if (jj >= 0 && jj < ny && kk >= 0 && kk < nz) {
      const size_t row = (size_t(kk) * ny + jj) * nx;
      if (i > 0) xs[0] = __bfloat162float(x[row + i - 1]);
      xs[1] = __bfloat162float(x[row + i]);
      if (i < nx - 1) xs[2] = __bfloat162float(x[row + i + 1]);
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      acc[0][c] = fmaf(xs[0], gv[c], acc[0][c]);
      acc[1][c] = fmaf(xs[1], gv[c], acc[1][c]);
      acc[2][c] = fmaf(xs[2], gv[c], acc[2][c]);
      bacc[c] += gv[c];
    }
  }
  __shared__ float out[48];
  float flat[48];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int c = 0; c < 16; ++c) flat[d * 16 + c] = acc[d][c];
  block_sum_store<48>(flat, out);
  for (int e = threadIdx.x; e < 48; e += blockDim.x) {
    const int d = e / 16, c = e % 16;
    const int tap = (dz + 1) * 9 + (dy + 1) * 3 + d;
    partial[(size_t(chunk) * 27 + tap) * 16 + c] = out[e];  // [chunk][tap][cout 16][cin 1]
  }
  if (grp == 0) {
    __shared__ float bout[16];
    block_sum_store<16>(bacc, bout);
    if (threadIdx.x < 16) bias_partial[size_t(chunk) * 16 + threadIdx.x] = bout[threadIdx.x];
  }
}

// grid (chunks): g BF16 [V] (one channel), d 16 channels in two octet planes
__global__ void __launch_bounds__(kThreads) wgrad_head_kernel(const __nv_bfloat16* d, const __nv_bfloat16* g, size_t V,
                                                              float* partial, float* bias_partial) {
  const int chunk = blockIdx.x;
  const size_t per = (V + gridDim.x - 1) / gridDim.x;
  const size_t v0 = size_t(chunk) * per, v1 = min(V, v0 + per);
  float acc[17];
#pragma unroll
  for (int c = 0; c < 17; ++c) acc[c] = 0.f;
  for (size_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const float gv = __bfloat162float(g[v]);
    float dlo[8], dhi[8];
    ld8(d + v * 8, dlo);
    ld8(d + (V + v) * 8, dhi);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      acc[c] = fmaf(gv, dlo[c], acc[c]);
      acc[8 + c] = fmaf(gv, dhi[c], acc[8 + c]);
    }
    acc[16] += gv;
  }
  __shared__ float out[17];
  block_sum_store<17>(acc, out);
  if (threadIdx.x < 16) partial[size_t(chunk) * 16 + threadIdx.x] = out[threadIdx.x];  // [chunk][1][1][16]
  if (threadIdx.x == 0) bias_partial[chunk] = out[16];
}

// grad[i] += sum over chunks (fixed order); i over taps * P, then bias
__global__ void wgrad_reduce_kernel(const float* partial, const float* bias_partial, int chunks, size_t n, int cout,
                                    float* grad, float* bias_grad) {
  for (size_t i = gtid(); i < n; i += gstride()) {
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += partial[size_t(c) * n + i];
    grad[i] += s;
  }
  if (blockIdx.x == 0 && int(threadIdx.x) < cout) {
    float s = 0.f;
    for (int c = 0; c < chunks; ++c) s += bias_partial[size_t(c) * cout + threadIdx.x];
    bias_grad[threadIdx.x] += s;
  }
}

// [27][nout][cin_pad] -> [cin_pad/16][27] blocks of nout x 16 K-major core
// matrices (byte (o/8) 256 + h 128 + (o%8) 16 within a block), one 16-byte
// chunk per work item
__global__ void to_smem_order_kernel(const __nv_bfloat16* src, int nout, int cin_pad, __nv_bfloat16* dst) {
  const size_t chunks = size_t(27) * nout * (cin_pad / 8);
  for (size_t e = gtid(); e < chunks; e += gstride()) {
    const int c8 = int(e % (cin_pad / 8));
    const int o = int((e / (cin_pad / 8)) % nout);
    const int tap = int(e / (size_t(cin_pad / 8) * nout));
    const int cb = c8 / 2, h = c8 % 2;
    const size_t byte = (size_t(cb) * 27 + tap) * size_t(nout) * 32 + size_t(o >> 3) * 256 + size_t(h) * 128 +
                        size_t(o & 7) * 16;
    *reinterpret_cast<uint4*>(reinterpret_cast<char*>(dst) + byte) =
        *reinterpret_cast<const uint4*>(src + (size_t(tap) * nout + o) * cin_pad + 8 * c8);
  }
}

// ---- optimiser and weight packing -------------------------------------------

__global__ void adam_kernel(float* w, float* m, float* v, const float* g, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2, float gscale) {
  for (size_t i = gtid(); i < n; i += gstride()) {
    const float gi = g[i] * gscale;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// forward layout [taps][nout][cin_pad] (or packed [nout][32]) from master [taps][cout][cin]
__global__ void pack_fwd_kernel(const float* wm, int taps, int cout, int cin, int nout, int cin_pad, int packed,
                                __nv_bfloat16* out) {
  const size_t n = packed ? size_t(nout) * 32 : size_t(taps) * nout * cin_pad;
  for (size_t e = gtid(); e < n; e += gstride()) {
    float val = 0.f;
    if (packed) {
      const int co = int(e / 32), t = int(e % 32);
      if (co < cout && t < taps) val = wm[size_t(t) * cout * cin + size_t(co) * cin];
    } else {
      const int ci = int(e % cin_pad);
      const int co = int((e / cin_pad) % nout);
      const int t = int(e / (size_t(cin_pad) * nout));
      if (co < cout && ci < cin) val = wm[(size_t(t) * cout + co) * cin + ci];
    }
    out[e] = __float2bfloat16(val);
  }
}

// input-gradient layout: out' = input channels [o0, o0 + on), in' = output
// channels, taps flipped: w'[t'][o'][i'] = w[taps-1-t'][i'][o0 + o']
__global__ void pack_dgrad_kernel(const float* wm, int taps, int cout, int cin, int o0, int on, int nout, int in_pad,
                                  __nv_bfloat16* out) {
  const size_t n = size_t(taps) * nout * in_pad;
  for (size_t e = gtid(); e < n; e += gstride()) {
    const int ip = int(e % in_pad);
    const int op = int((e / in_pad) % nout);
    const int t = int(e / (size_t(in_pad) * nout));
    float val = 0.f;
    if (op < on && ip < cout) val = wm[(size_t(taps - 1 - t) * cout + ip) * cin + (o0 + op)];
    out[e] = __float2bfloat16(val);
  }
}

// ---- flexible CG (FP64 vectors, FP64 fixed-order reductions) ---------------

struct FpcgScalars {
  double rz;     // z_k . r_k
  double alpha;
  double beta;
  double rr;     // r . r (recursive or true, whichever was computed last)
  double pq;
  double bb;     // ||b||^2 after mean removal
  double mean;   // mean of b (removed)
  int flag;      // 1: p.q <= 0 or non-finite; 2: z.r = 0 or non-finite
  int pad;
};

constexpr int kDotBlocks = 152 * 4;

// per-block partial sums of a.b (sum of a when b is null) and of a.c (when c
// is non-null), at partials[block] and partials[gridDim.x + block]
__global__ void __launch_bounds__(kThreads) dot2_kernel(const double* a, const double* b, const double* c, size_t n,
                                                        double* partials) {
  __shared__ double sh[2][32];
  double s0 = 0.0, s1 = 0.0;
  for (size_t e = gtid(); e < n; e += gstride()) {
    const double ae = a[e];
    s0 = fma(ae, b ? b[e] : 1.0, s0);
    if (c) s1 = fma(ae, c[e], s1);
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
    for (int w = 0; w < kThreads / 32; ++w) {
      t0 += sh[0][w];
      t1 += sh[1][w];
    }
    partials[blockIdx.x] = t0;
    partials[gridDim.x + blockIdx.x] = t1;
  }
}

enum FpcgOp : int { kOpMean = 0, kOpBB = 1, kOpRZ = 2, kOpAlpha = 3, kOpRR = 4, kOpBeta = 5 };

__global__ void __launch_bounds__(kThreads) fpcg_scalar_kernel(int op, const double* partials, int nb, size_t n,
                                                               FpcgScalars* sc) {
  const double s0 = block_sum(partials, nb);
  const double s1 = (op == kOpBeta) ? block_sum(partials + nb, nb) : 0.0;
  if (threadIdx.x != 0) return;
  switch (op) {
    case kOpMean: sc->mean = s0 / double(n); break;
    case kOpBB: sc->bb = s0; sc->rr = s0; break;
    case kOpRZ:
      sc->rz = s0;
      if (s0 == 0.0 || !isfinite(s0)) sc->flag = 2;
      break;
    case kOpAlpha:
      sc->pq = s0;
      if (!(s0 > 0.0) || !isfinite(s0)) {
        sc->flag = 1;
        sc->alpha = 0.0;
      } else {
        sc->alpha = sc->rz / s0;
      }
      break;
    case kOpRR: sc->rr = s0; break;
    case kOpBeta: {
      // Polak-Ribiere: beta = z_{k+1} . (r_{k+1} - r_k) / (z_k . r_k), with
      // r_{k+1} - r_k = -alpha q_k.  z.r < 0 (a preconditioner that is not
      // positive definite) is allowed: alpha = z.r / p.q is then negative and
      // still the exact line search along p, since r.p = r.z.
      if (s0 == 0.0 || !isfinite(s0) || !isfinite(s1)) {
        sc->flag = 2;
        sc->beta = 0.0;
      } else {
        sc->beta = -sc->alpha * s1 / sc->rz;
        sc->rz = s0;
      }
      break;
    }
  }
}

__global__ void sub_mean_kernel(const double* b, size_t n, const FpcgScalars* sc, double* out) {
  const double m = sc->mean;
  for (size_t e = gtid(); e < n; e += gstride()) out[e] = b[e] - m;
}

// r = b - t (t = A x), or r = b when t is null
__global__ void residual_kernel(const double* b, const double* t, size_t n, double* r) {
  for (size_t e = gtid(); e < n; e += gstride()) r[e] = t ? b[e] - t[e] : b[e];
}

// x += alpha p; r -= alpha q; partials of r.r
__global__ void __launch_bounds__(kThreads) xr_update_kernel(double* x, double* r, const double* p, const double* q,
                                                             size_t n, const FpcgScalars* sc, double* partials) {
  __shared__ double sh[32];
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
    for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    partials[blockIdx.x] = t;
  }
}

// p = z + beta p (beta = 0 on a restart: p = z)
__global__ void direction_kernel(const double* z, double* p, size_t n, const FpcgScalars* sc, int restart) {
  const double be = restart ? 0.0 : sc->beta;
  for (size_t e = gtid(); e < n; e += gstride()) p[e] = restart ? z[e] : fma(be, p[e], z[e]);
}

}  // namespace
}  // namespace cfd

using namespace cfd;

// ---------------------------------------------------------------------------
// Model object
// ---------------------------------------------------------------------------
struct cfd_unet {
  int nx, ny, nz;
  cudaStream_t stream;
  char* ws;
  size_t bytes;
  int64_t nparams;
  // parameters (FP32), one contiguous block per array
  float *w, *m, *v, *g;
  size_t woff[kNumLayers], boff[kNumLayers];  // offsets of weights / bias of each layer
  // BF16 weight copies
  __nv_bfloat16* wf[kNumLayers];       // forward
  __nv_bfloat16* wfc[kNumLayers];      // forward, shared-memory order (3x3x3 layers 1..7)
  __nv_bfloat16* wdc[kNumLayers][2];   // input gradient, shared-memory order
  __nv_bfloat16* wd[kNumLayers][2];    // input gradient (two output slices for L1c)
  // activations
  __nv_bfloat16 *xin, *a0, *s0, *p0, *a1, *s1, *p1, *a2, *s2, *u1, *d1, *u0, *d0;
  float *z, *tgt;
  // gradients
  __nv_bfloat16 *gz, *g_d0, *g_s0, *g_u0, *g_d1, *g_s1, *g_u1, *g_s2, *g_a2, *g_p1, *g_a1, *g_p0, *g_a0;
  // scratch
  float *wpart, *bpart;
  float *wtc, *btc;  // partial sums of the tensor-core weight gradient
  double *parts, *scale, *lossp;
  int* err;
  // flexible CG vectors and scalars
  double *cg_b, *cg_r, *cg_z, *cg_p, *cg_q, *cg_parts;
  FpcgScalars* cg_sc;
  // tensor table for cfd_unet_read_tensor (activations and their gradients)
  __nv_bfloat16* tens[26];
  size_t tens_count[26];
  int loss_kind;  // CFD_UNET_LOSS_*
  int wgrad_mode; // CFD_UNET_WGRAD_*
  int conv_mode;  // CFD_UNET_CONV_*: how the tiled convolutions stage weights and inputs
  int adam_t;
  int64_t launches;
};

namespace {

struct UNetLayout {
  size_t total;
  size_t off[64];
  int k;
};

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

int64_t param_count() {
  int64_t n = 0;
  for (const auto& L : kLayers) n += int64_t(taps_of(L.ks)) * L.cout * (L.c0 + L.c1) + L.cout;
  return n;
}

// Walk the buffer list once to size it (ptrs == nullptr) or to assign it.
size_t carve(cfd_unet* u, int nx, int ny, int nz, char* base) {
  size_t off = 0;
  auto take = [&](size_t b) -> char* {
    char* p = base ? base + off : nullptr;
    off = al256(off + b);
    return p;
  };
  const size_t V0 = size_t(nx) * ny * nz, V1 = V0 / 8, V2 = V0 / 64;
  const int64_t np = param_count();
  float* w = reinterpret_cast<float*>(take(size_t(np) * 4));
  float* m = reinterpret_cast<float*>(take(size_t(np) * 4));
  float* v = reinterpret_cast<float*>(take(size_t(np) * 4));
  float* g = reinterpret_cast<float*>(take(size_t(np) * 4));
  if (u) { u->w = w; u->m = m; u->v = v; u->g = g; }
  for (int l = 0; l < kNumLayers; ++l) {
    const LayerSpec& L = kLayers[l];
    const int cin = L.c0 + L.c1, taps = taps_of(L.ks);
    const size_t fwd = L.packed ? size_t(nout_pad(L.cout)) * 32 : size_t(taps) * nout_pad(L.cout) * pad16(cin);
    __nv_bfloat16* wf = reinterpret_cast<__nv_bfloat16*>(take(fwd * 2));
    __nv_bfloat16* wd0 = nullptr;
    __nv_bfloat16* wd1 = nullptr;
    if (l != 0) {
      if (l == 6) {  // L1c: input-gradient output split into 32 + 64 channels
        wd0 = reinterpret_cast<__nv_bfloat16*>(take(size_t(taps) * 32 * pad16(L.cout) * 2));
        wd1 = reinterpret_cast<__nv_bfloat16*>(take(size_t(taps) * 64 * pad16(L.cout) * 2));
      } else {
        wd0 = reinterpret_cast<__nv_bfloat16*>(take(size_t(taps) * nout_pad(cin) * pad16(L.cout) * 2));
      }
    }
    // copies in the tiled kernel's shared-memory order for the 3x3x3 layers
    __nv_bfloat16 *wfc = nullptr, *wdc0 = nullptr, *wdc1 = nullptr;
    if (l >= 1 && l <= 7) {
      wfc = reinterpret_cast<__nv_bfloat16*>(take(fwd * 2));
      if (l == 6) {
        wdc0 = reinterpret_cast<__nv_bfloat16*>(take(size_t(taps) * 32 * pad16(L.cout) * 2));
        wdc1 = reinterpret_cast<__nv_bfloat16*>(take(size_t(taps) * 64 * pad16(L.cout) * 2));
      } else {
        wdc0 = reinterpret_cast<__nv_bfloat16*>(take(size_t(taps) * nout_pad(cin) * pad16(L.cout) * 2));
      }
    }
    if (u) {
      u->wf[l] = wf; u->wd[l][0] = wd0; u->wd[l][1] = wd1;
      u->wfc[l] = wfc; u->wdc[l][0] = wdc0; u->wdc[l][1] = wdc1;
    }
  }
  auto act = [&](size_t vox, int c) { return reinterpret_cast<__nv_bfloat16*>(take(vox * size_t(c) * 2)); };
  __nv_bfloat16* bufs[26] = {
      act(V0, 1),  act(V0, 16), act(V0, 16), act(V1, 16), act(V1, 32), act(V1, 32), act(V2, 32),
      act(V2, 64), act(V2, 64), act(V1, 64), act(V1, 32), act(V0, 32), act(V0, 16),
      act(V0, 1),  act(V0, 16), act(V0, 16), act(V0, 32), act(V1, 32), act(V1, 32), act(V1, 64),
      act(V2, 64), act(V2, 64), act(V2, 32), act(V1, 32), act(V1, 16), act(V0, 16)};
  float* z = reinterpret_cast<float*>(take(V0 * 4));
  float* tgt = reinterpret_cast<float*>(take(V0 * 4));
  // weight-gradient partials: largest taps * cout * cin over the layers
  size_t maxp = 0;
  for (const auto& L : kLayers) maxp = std::max(maxp, size_t(taps_of(L.ks)) * L.cout * (L.c0 + L.c1));
  float* wpart = reinterpret_cast<float*>(take(size_t(kWgradChunks) * maxp * 4));
  float* bpart = reinterpret_cast<float*>(take(size_t(kWgradChunks) * 64 * 4));
  float* wtc = reinterpret_cast<float*>(take(size_t(kWgradTcChunks) * maxp * 4));
  float* btc = reinterpret_cast<float*>(take(size_t(kWgradTcChunks) * 64 * 4));
  double* parts = reinterpret_cast<double*>(take(size_t(152 * 8) * 8));
  double* scale = reinterpret_cast<double*>(take(64));
  double* lossp = reinterpret_cast<double*>(take(size_t(3 * 152 * 8) * 8));
  int* err = reinterpret_cast<int*>(take(64));
  double* cgv[5];
  for (int i = 0; i < 5; ++i) cgv[i] = reinterpret_cast<double*>(take(V0 * 8));
  double* cg_parts = reinterpret_cast<double*>(take(size_t(2 * kDotBlocks) * 8));
  FpcgScalars* cg_sc = reinterpret_cast<FpcgScalars*>(take(sizeof(FpcgScalars)));
  if (u) {
    u->cg_b = cgv[0]; u->cg_r = cgv[1]; u->cg_z = cgv[2]; u->cg_p = cgv[3]; u->cg_q = cgv[4];
    u->cg_parts = cg_parts; u->cg_sc = cg_sc;
    const size_t vox[26] = {V0, V0, V0, V1, V1, V1, V2, V2, V2, V1, V1, V0, V0,
                            V0, V0, V0, V0, V1, V1, V1, V2, V2, V2, V1, V1, V0};
    const int ch[26] = {1, 16, 16, 16, 32, 32, 32, 64, 64, 64, 32, 32, 16,
                        1, 16, 16, 32, 32, 32, 64, 64, 64, 32, 32, 16, 16};
    for (int i = 0; i < 26; ++i) {
      u->tens[i] = bufs[i];
      u->tens_count[i] = vox[i] * size_t(ch[i]);
    }
    u->xin = bufs[0]; u->a0 = bufs[1]; u->s0 = bufs[2]; u->p0 = bufs[3]; u->a1 = bufs[4]; u->s1 = bufs[5];
    u->p1 = bufs[6]; u->a2 = bufs[7]; u->s2 = bufs[8]; u->u1 = bufs[9]; u->d1 = bufs[10]; u->u0 = bufs[11];
    u->d0 = bufs[12];
    u->gz = bufs[13]; u->g_d0 = bufs[14]; u->g_s0 = bufs[15]; u->g_u0 = bufs[16]; u->g_d1 = bufs[17];
    u->g_s1 = bufs[18]; u->g_u1 = bufs[19]; u->g_s2 = bufs[20]; u->g_a2 = bufs[21]; u->g_p1 = bufs[22];
    u->g_a1 = bufs[23]; u->g_p0 = bufs[24]; u->g_a0 = bufs[25];
    u->z = z; u->tgt = tgt; u->wpart = wpart; u->bpart = bpart; u->wtc = wtc; u->btc = btc;
    u->parts = parts; u->scale = scale;
    u->lossp = lossp; u->err = err;
    size_t o = 0;
    for (int l = 0; l < kNumLayers; ++l) {
      const LayerSpec& L = kLayers[l];
      u->woff[l] = o;
      o += size_t(taps_of(L.ks)) * L.cout * (L.c0 + L.c1);
      u->boff[l] = o;
      o += size_t(L.cout);
    }
  }
  return off;
}

thread_local char g_unet_err[256] = "no error";

int uerr(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_unet_err, sizeof(g_unet_err), fmt, ap);
  va_end(ap);
  cfd_internal_error(code, "%s", g_unet_err);
  return code;
}

int uck(cfd_unet*, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CFD_OK;
  return uerr(CFD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// count one kernel launch and check it
int klaunch(cfd_unet* u, const char* what) {
  ++u->launches;
  return uck(u, cudaGetLastError(), what);
}

void level_dims(const cfd_unet* u, int level, int& x, int& y, int& z) {
  x = u->nx >> level;
  y = u->ny >> level;
  z = u->nz >> level;
}

int conv(cfd_unet* u, int layer, const __nv_bfloat16* src0, const __nv_bfloat16* src1, __nv_bfloat16* dst0,
         __nv_bfloat16* dst1, int split, float* dst_f32) {
  const LayerSpec& L = kLayers[layer];
  ConvArgs a{};
  level_dims(u, L.level, a.nx, a.ny, a.nz);
  a.src0 = src0; a.c0 = L.c0; a.src1 = src1; a.c1 = L.c1;
  a.ks = L.ks; a.packed = L.packed ? 1 : 0;
  a.w = u->wf[layer];
  a.w_cm = u->conv_mode == CFD_UNET_CONV_REGISTERS ? nullptr : u->wfc[layer];
  a.stages = u->conv_mode == CFD_UNET_CONV_TWO_STAGE ? 2 : (u->conv_mode == CFD_UNET_CONV_PERSISTENT ? 3 : 1);
  a.bias = u->w + u->boff[layer];
  a.cout = L.cout;
  a.dst0 = dst0; a.dst1 = dst1; a.split = split; a.dst_f32 = dst_f32;
  a.err = u->err;
  ++u->launches;
  return uck(u, launch_conv3d(a, nout_pad(L.cout), u->stream), "conv");
}

// input gradient of layer `layer`: g_out -> (dst0 channels [o0, o0+on) ...)
int conv_dgrad(cfd_unet* u, int layer, int slice, const __nv_bfloat16* gout, int o_count, __nv_bfloat16* dst0,
               __nv_bfloat16* dst1, int split) {
  const LayerSpec& L = kLayers[layer];
  ConvArgs a{};
  level_dims(u, L.level, a.nx, a.ny, a.nz);
  a.src0 = gout; a.c0 = L.cout; a.src1 = nullptr; a.c1 = 0;
  a.ks = L.ks; a.packed = 0;
  a.w = u->wd[layer][slice];
  a.w_cm = u->conv_mode == CFD_UNET_CONV_REGISTERS ? nullptr : u->wdc[layer][slice];
  a.stages = u->conv_mode == CFD_UNET_CONV_TWO_STAGE ? 2 : (u->conv_mode == CFD_UNET_CONV_PERSISTENT ? 3 : 1);
  a.bias = nullptr;
  a.cout = o_count;
  a.dst0 = dst0; a.dst1 = dst1; a.split = split; a.dst_f32 = nullptr;
  a.err = u->err;
  ++u->launches;
  return uck(u, launch_conv3d(a, nout_pad(o_count), u->stream), "conv dgrad");
}

int wgrad(cfd_unet* u, int layer, const __nv_bfloat16* src0, const __nv_bfloat16* src1, const __nv_bfloat16* gout) {
  const LayerSpec& L = kLayers[layer];
  if (u->wgrad_mode == CFD_UNET_WGRAD_TENSOR && L.ks == 3 && !L.packed) {
    // the 3x3x3 layers with 16-channel multiples: tensor cores
    int fx, fy, fz, chunks = 0;
    level_dims(u, L.level, fx, fy, fz);
    const cudaError_t e = launch_wgrad_tc(src0, L.c0, src1, L.c1, gout, L.cout, fx, fy, fz, u->wtc, u->btc,
                                          kWgradTcChunks, &chunks, u->err, u->stream);
    if (e == cudaSuccess) {
      ++u->launches;
      const size_t n = size_t(27) * L.cout * (L.c0 + L.c1);
      wgrad_reduce_kernel<<<grid_for(n), kThreads, 0, u->stream>>>(u->wtc, u->btc, chunks, n, L.cout,
                                                                   u->g + u->woff[layer], u->g + u->boff[layer]);
      return klaunch(u, "wgrad reduce");
    }
    if (e != cudaErrorNotSupported) return uck(u, e, "tensor-core weight gradient");
  }
  if ((layer == 0 && L.c0 == 1 && L.cout == 16 && L.ks == 3) || (layer == 8 && L.cout == 1 && L.c0 == 16 && L.ks == 1)) {
    int fx, fy, fz;
    level_dims(u, L.level, fx, fy, fz);
    if (layer == 0)
      wgrad_first_kernel<<<dim3(kNarrowChunks, 9), kThreads, 0, u->stream>>>(src0, gout, fx, fy, fz, u->wpart, u->bpart);
    else
      wgrad_head_kernel<<<kNarrowChunks, kThreads, 0, u->stream>>>(src0, gout, size_t(fx) * fy * fz, u->wpart, u->bpart);
    int rc = klaunch(u, "narrow-layer weight gradient");
    if (rc) return rc;
    const size_t n = size_t(taps_of(L.ks)) * L.cout * L.c0;
    wgrad_reduce_kernel<<<grid_for(n), kThreads, 0, u->stream>>>(u->wpart, u->bpart, kNarrowChunks, n, L.cout,
                                                                 u->g + u->woff[layer], u->g + u->boff[layer]);
    return klaunch(u, "wgrad reduce");
  }
  WgradArgs a{};
  level_dims(u, L.level, a.nx, a.ny, a.nz);
  a.src0 = src0; a.c0 = L.c0; a.src1 = src1; a.c1 = L.c1; a.ks = L.ks;
  a.g = gout; a.cout = L.cout; a.partial = u->wpart; a.bias_partial = u->bpart;
  const int taps = taps_of(L.ks);
  wgrad_kernel<<<dim3(kWgradChunks, taps), kThreads, 0, u->stream>>>(a);
  int rc = klaunch(u, "wgrad");
  if (rc) return rc;
  const size_t n = size_t(taps) * L.cout * (L.c0 + L.c1);
  wgrad_reduce_kernel<<<grid_for(n), kThreads, 0, u->stream>>>(u->wpart, u->bpart, kWgradChunks, n, L.cout,
                                                               u->g + u->woff[layer], u->g + u->boff[layer]);
  return klaunch(u, "wgrad reduce");
}

int pack_weights(cfd_unet* u) {
  for (int l = 0; l < kNumLayers; ++l) {
    const LayerSpec& L = kLayers[l];
    const int cin = L.c0 + L.c1, taps = taps_of(L.ks);
    const size_t nf = L.packed ? size_t(nout_pad(L.cout)) * 32 : size_t(taps) * nout_pad(L.cout) * pad16(cin);
    pack_fwd_kernel<<<grid_for(nf), kThreads, 0, u->stream>>>(u->w + u->woff[l], taps, L.cout, cin, nout_pad(L.cout),
                                                              pad16(cin), L.packed ? 1 : 0, u->wf[l]);
    int rc = klaunch(u, "pack");
    if (rc) return rc;
    if (l == 0) continue;
    if (l == 6) {
      pack_dgrad_kernel<<<grid_for(size_t(taps) * 32 * pad16(L.cout)), kThreads, 0, u->stream>>>(
          u->w + u->woff[l], taps, L.cout, cin, 0, 32, 32, pad16(L.cout), u->wd[l][0]);
      pack_dgrad_kernel<<<grid_for(size_t(taps) * 64 * pad16(L.cout)), kThreads, 0, u->stream>>>(
          u->w + u->woff[l], taps, L.cout, cin, 32, 64, 64, pad16(L.cout), u->wd[l][1]);
    } else {
      pack_dgrad_kernel<<<grid_for(size_t(taps) * nout_pad(cin) * pad16(L.cout)), kThreads, 0, u->stream>>>(
          u->w + u->woff[l], taps, L.cout, cin, 0, cin, nout_pad(cin), pad16(L.cout), u->wd[l][0]);
    }
    rc = klaunch(u, "pack dgrad");
    if (rc) return rc;
    if (l <= 7) {
      auto cm = [&](const __nv_bfloat16* src, int nout, int cin_pad, __nv_bfloat16* dst) {
        to_smem_order_kernel<<<grid_for(size_t(27) * nout * cin_pad / 8), kThreads, 0, u->stream>>>(src, nout, cin_pad,
                                                                                                     dst);
        return klaunch(u, "weights to shared-memory order");
      };
      rc = cm(u->wf[l], nout_pad(L.cout), pad16(cin), u->wfc[l]);
      if (!rc && l == 6) {
        rc = cm(u->wd[l][0], 32, pad16(L.cout), u->wdc[l][0]);
        if (!rc) rc = cm(u->wd[l][1], 64, pad16(L.cout), u->wdc[l][1]);
      } else if (!rc) {
        rc = cm(u->wd[l][0], nout_pad(cin), pad16(L.cout), u->wdc[l][0]);
      }
      if (rc) return rc;
    }
  }
  return CFD_OK;
}

// forward pass from u->xin to u->z (FP32 head output)
int forward(cfd_unet* u) {
  int fx, fy, fz;
  int rc = CFD_OK;
  auto ok = [&](int r) { if (r && !rc) rc = r; return rc == CFD_OK; };
  level_dims(u, 0, fx, fy, fz);
  first_layer_kernel<<<grid_for(size_t(fx) * fy * fz), kThreads, 0, u->stream>>>(u->xin, fx, fy, fz, u->wf[0],
                                                                                  u->w + u->boff[0], u->a0);
  if (!ok(klaunch(u, "first layer"))) return rc;
  if (!ok(conv(u, 1, u->a0, nullptr, u->s0, nullptr, 16, nullptr))) return rc;
  level_dims(u, 0, fx, fy, fz);
  pool2_kernel<<<grid_for(size_t(fx) * fy * fz * 2), kThreads, 0, u->stream>>>(u->s0, fx, fy, fz, 16, u->p0);
  if (!ok(klaunch(u, "pool"))) return rc;
  if (!ok(conv(u, 2, u->p0, nullptr, u->a1, nullptr, 32, nullptr))) return rc;
  if (!ok(conv(u, 3, u->a1, nullptr, u->s1, nullptr, 32, nullptr))) return rc;
  level_dims(u, 1, fx, fy, fz);
  pool2_kernel<<<grid_for(size_t(fx) * fy * fz * 4), kThreads, 0, u->stream>>>(u->s1, fx, fy, fz, 32, u->p1);
  if (!ok(klaunch(u, "pool"))) return rc;
  if (!ok(conv(u, 4, u->p1, nullptr, u->a2, nullptr, 64, nullptr))) return rc;
  if (!ok(conv(u, 5, u->a2, nullptr, u->s2, nullptr, 64, nullptr))) return rc;
  level_dims(u, 1, fx, fy, fz);
  up2_kernel<<<grid_for(size_t(fx) * fy * fz * 64), kThreads, 0, u->stream>>>(u->s2, fx, fy, fz, 64, u->u1);
  if (!ok(klaunch(u, "up"))) return rc;
  if (!ok(conv(u, 6, u->s1, u->u1, u->d1, nullptr, 32, nullptr))) return rc;
  level_dims(u, 0, fx, fy, fz);
  up2_kernel<<<grid_for(size_t(fx) * fy * fz * 32), kThreads, 0, u->stream>>>(u->d1, fx, fy, fz, 32, u->u0);
  if (!ok(klaunch(u, "up"))) return rc;
  if (!ok(conv(u, 7, u->s0, u->u0, u->d0, nullptr, 16, nullptr))) return rc;
  const size_t V0 = size_t(u->nx) * u->ny * u->nz;
  head_kernel<<<grid_for(V0), kThreads, 0, u->stream>>>(u->d0, V0, u->wf[8], u->w + u->boff[8], u->z);
  ok(klaunch(u, "head"));
  return rc;
}

// backward pass from u->gz (dL/dz, BF16) accumulating weight gradients into u->g
int backward(cfd_unet* u) {
  int rc = CFD_OK;
  auto ok = [&](int r) { if (r && !rc) rc = r; return rc == CFD_OK; };
  int fx, fy, fz;
  // head
  if (!ok(wgrad(u, 8, u->d0, nullptr, u->gz))) return rc;
  {
    const size_t V0 = size_t(u->nx) * u->ny * u->nz;
    head_dgrad_kernel<<<grid_for(V0), kThreads, 0, u->stream>>>(u->gz, V0, u->wf[8], u->g_d0);
    if (!ok(klaunch(u, "head dgrad"))) return rc;
  }
  // L0c: input = s0 (16) + u0 (32)
  if (!ok(wgrad(u, 7, u->s0, u->u0, u->g_d0))) return rc;
  if (!ok(conv_dgrad(u, 7, 0, u->g_d0, 48, u->g_s0, u->g_u0, 16))) return rc;
  level_dims(u, 0, fx, fy, fz);
  up2_adj_kernel<<<grid_for(size_t(fx / 2) * (fy / 2) * (fz / 2) * 32), kThreads, 0, u->stream>>>(u->g_u0, fx, fy, fz, 32,
                                                                                                    u->g_d1);
  if (!ok(klaunch(u, "up adjoint"))) return rc;
  // L1c: input = s1 (32) + u1 (64)
  if (!ok(wgrad(u, 6, u->s1, u->u1, u->g_d1))) return rc;
  if (!ok(conv_dgrad(u, 6, 0, u->g_d1, 32, u->g_s1, nullptr, 32))) return rc;
  if (!ok(conv_dgrad(u, 6, 1, u->g_d1, 64, u->g_u1, nullptr, 64))) return rc;
  level_dims(u, 1, fx, fy, fz);
  up2_adj_kernel<<<grid_for(size_t(fx / 2) * (fy / 2) * (fz / 2) * 64), kThreads, 0, u->stream>>>(u->g_u1, fx, fy, fz, 64,
                                                                                                    u->g_s2);
  if (!ok(klaunch(u, "up adjoint"))) return rc;
  // level 2
  if (!ok(wgrad(u, 5, u->a2, nullptr, u->g_s2))) return rc;
  if (!ok(conv_dgrad(u, 5, 0, u->g_s2, 64, u->g_a2, nullptr, 64))) return rc;
  if (!ok(wgrad(u, 4, u->p1, nullptr, u->g_a2))) return rc;
  if (!ok(conv_dgrad(u, 4, 0, u->g_a2, 32, u->g_p1, nullptr, 32))) return rc;
  level_dims(u, 1, fx, fy, fz);
  pool2_adj_kernel<<<grid_for(size_t(fx) * fy * fz * 32), kThreads, 0, u->stream>>>(u->g_p1, fx, fy, fz, 32, u->g_s1);
  if (!ok(klaunch(u, "pool adjoint"))) return rc;
  // level 1
  if (!ok(wgrad(u, 3, u->a1, nullptr, u->g_s1))) return rc;
  if (!ok(conv_dgrad(u, 3, 0, u->g_s1, 32, u->g_a1, nullptr, 32))) return rc;
  if (!ok(wgrad(u, 2, u->p0, nullptr, u->g_a1))) return rc;
  if (!ok(conv_dgrad(u, 2, 0, u->g_a1, 16, u->g_p0, nullptr, 16))) return rc;
  level_dims(u, 0, fx, fy, fz);
  pool2_adj_kernel<<<grid_for(size_t(fx) * fy * fz * 16), kThreads, 0, u->stream>>>(u->g_p0, fx, fy, fz, 16, u->g_s0);
  if (!ok(klaunch(u, "pool adjoint"))) return rc;
  // level 0
  if (!ok(wgrad(u, 1, u->a0, nullptr, u->g_s0))) return rc;
  if (!ok(conv_dgrad(u, 1, 0, u->g_s0, 16, u->g_a0, nullptr, 16))) return rc;
  ok(wgrad(u, 0, u->xin, nullptr, u->g_a0));
  return rc;
}

int input_scale(cfd_unet* u, const double* r) {
  const size_t V = size_t(u->nx) * u->ny * u->nz;
  const int nb = grid_for(V);
  sumsq_kernel<<<nb, kThreads, 0, u->stream>>>(r, V, u->parts);
  int rc = klaunch(u, "sumsq");
  if (rc) return rc;
  scale_kernel<<<1, kThreads, 0, u->stream>>>(u->parts, nb, V, u->scale);
  rc = klaunch(u, "scale");
  if (rc) return rc;
  normalize_kernel<<<grid_for(V), kThreads, 0, u->stream>>>(r, V, u->scale, u->xin);
  return klaunch(u, "normalize");
}

// deterministic host-side initialisation: uniform(-a, a), a = sqrt(3 / fan_in)
void init_params(std::vector<float>& p, uint64_t seed) {
  uint64_t s = seed * 0x9E3779B97F4A7C15ull + 0x1234567ull;
  auto next = [&]() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return double(z >> 11) * (1.0 / 9007199254740992.0);
  };
  size_t o = 0;
  for (const auto& L : kLayers) {
    const int cin = L.c0 + L.c1, taps = taps_of(L.ks);
    const double a = std::sqrt(3.0 / double(cin * taps));
    const size_t nw = size_t(taps) * L.cout * cin;
    for (size_t i = 0; i < nw; ++i) p[o + i] = float((2.0 * next() - 1.0) * a);
    o += nw;
    for (int i = 0; i < L.cout; ++i) p[o + size_t(i)] = 0.f;
    o += size_t(L.cout);
  }
}

}  // namespace

bool cfd::unet_view(const cfd_unet* u, UNetView* v) {
  if (!u || !v) return false;
  v->nx = u->nx;
  v->ny = u->ny;
  v->nz = u->nz;
  v->xin = u->xin;
  v->z = u->z;
  v->err = u->err;
  v->conv_mode = u->conv_mode;
  return true;
}

int cfd::unet_forward_on(cfd_unet* u, cudaStream_t s, int* kernels) {
  if (!u) return uerr(CFD_ERR_INVALID_ARG, "unet: NULL handle");
  const cudaStream_t keep = u->stream;
  const int64_t l0 = u->launches;
  u->stream = s;
  const int rc = forward(u);
  u->stream = keep;
  if (kernels) *kernels = int(u->launches - l0);
  return rc;
}

extern "C" {

int cfd_unet_workspace_bytes(int nx, int ny, int nz, size_t* bytes) {
  if (nx < 4 || ny < 4 || nz < 4 || nx % 4 || ny % 4 || nz % 4 || !bytes)
    return uerr(CFD_ERR_INVALID_ARG, "unet: grid sizes must be multiples of 4 (>= 4)");
  *bytes = carve(nullptr, nx, ny, nz, nullptr);
  return CFD_OK;
}

int cfd_unet_create(int nx, int ny, int nz, void* dev_ws, size_t bytes, cfd_stream_t stream, uint64_t seed,
                    cfd_unet** out) {
  size_t need = 0;
  int rc = cfd_unet_workspace_bytes(nx, ny, nz, &need);
  if (rc) return rc;
  if (!out || !dev_ws || (reinterpret_cast<uintptr_t>(dev_ws) & 255))
    return uerr(CFD_ERR_INVALID_ARG, "unet: out NULL or workspace NULL / not 256-byte aligned");
  if (bytes < need) return uerr(CFD_ERR_WORKSPACE_TOO_SMALL, "unet: workspace %zu < %zu", bytes, need);
  cfd_unet* u = new (std::nothrow) cfd_unet();
  if (!u) return uerr(CFD_ERR_INVALID_ARG, "unet: out of host memory");
  u->nx = nx; u->ny = ny; u->nz = nz;
  u->stream = reinterpret_cast<cudaStream_t>(stream);
  u->ws = static_cast<char*>(dev_ws);
  u->bytes = bytes;
  u->nparams = param_count();
  u->conv_mode = CFD_UNET_CONV_BULK;
  carve(u, nx, ny, nz, u->ws);
  std::vector<float> p(size_t(u->nparams));
  init_params(p, seed);
  rc = uck(u, cudaMemcpyAsync(u->w, p.data(), p.size() * 4, cudaMemcpyHostToDevice, u->stream), "copy params");
  if (!rc) rc = uck(u, cudaMemsetAsync(u->m, 0, p.size() * 4, u->stream), "memset");
  if (!rc) rc = uck(u, cudaMemsetAsync(u->v, 0, p.size() * 4, u->stream), "memset");
  if (!rc) rc = uck(u, cudaMemsetAsync(u->err, 0, 4, u->stream), "memset");
  if (!rc) rc = pack_weights(u);
  if (!rc) rc = uck(u, cudaStreamSynchronize(u->stream), "synchronize");
  if (rc) {
    delete u;
    return rc;
  }
  *out = u;
  return CFD_OK;
}

void cfd_unet_destroy(cfd_unet* u) { delete u; }

int64_t cfd_unet_param_count(const cfd_unet* u) { return u ? u->nparams : param_count(); }

int cfd_unet_grid(const cfd_unet* u, int* nx, int* ny, int* nz) {
  if (!u || !nx || !ny || !nz) return uerr(CFD_ERR_INVALID_ARG, "unet: NULL argument");
  *nx = u->nx;
  *ny = u->ny;
  *nz = u->nz;
  return CFD_OK;
}

int cfd_unet_get_params(cfd_unet* u, float* host, int64_t n) {
  if (!u || !host || n != u->nparams) return uerr(CFD_ERR_INVALID_ARG, "unet: bad parameter buffer");
  int rc = uck(u, cudaMemcpyAsync(host, u->w, size_t(n) * 4, cudaMemcpyDeviceToHost, u->stream), "copy params");
  if (!rc) rc = uck(u, cudaStreamSynchronize(u->stream), "synchronize");
  return rc;
}

int cfd_unet_set_params(cfd_unet* u, const float* host, int64_t n) {
  if (!u || !host || n != u->nparams) return uerr(CFD_ERR_INVALID_ARG, "unet: bad parameter buffer");
  int rc = uck(u, cudaMemcpyAsync(u->w, host, size_t(n) * 4, cudaMemcpyHostToDevice, u->stream), "copy params");
  if (!rc) rc = pack_weights(u);
  if (!rc) rc = uck(u, cudaStreamSynchronize(u->stream), "synchronize");
  return rc;
}

int cfd_unet_apply(cfd_unet* u, const double* r_dev, double* z_dev) {
  if (!u || !r_dev || !z_dev) return uerr(CFD_ERR_INVALID_ARG, "unet: NULL argument");
  const size_t V = size_t(u->nx) * u->ny * u->nz;
  int rc = input_scale(u, r_dev);
  if (!rc) rc = forward(u);
  if (rc) return rc;
  const int nb = grid_for(V);
  sum_f32_kernel<<<nb, kThreads, 0, u->stream>>>(u->z, V, u->parts);
  rc = klaunch(u, "sum");
  if (rc) return rc;
  mean_kernel<<<1, kThreads, 0, u->stream>>>(u->parts, nb, V, u->scale);
  rc = klaunch(u, "mean");
  if (rc) return rc;
  denorm_kernel<<<grid_for(V), kThreads, 0, u->stream>>>(u->z, V, u->scale, z_dev);
  return klaunch(u, "denorm");
}

int cfd_unet_train_step(cfd_unet* u, const double* r_dev, const double* e_dev, int npairs, float lr, float* loss) {
  if (!u || !r_dev || !e_dev || npairs < 1) return uerr(CFD_ERR_INVALID_ARG, "unet: bad training arguments");
  const size_t V = size_t(u->nx) * u->ny * u->nz;
  const int nb = grid_for(V);
  int rc = uck(u, cudaMemsetAsync(u->g, 0, size_t(u->nparams) * 4, u->stream), "memset grads");
  std::vector<double> lp = std::vector<double>(size_t(nb));
  double total = 0.0;
  for (int k = 0; k < npairs && !rc; ++k) {
    const double* r = r_dev + size_t(k) * V;
    const double* e = e_dev + size_t(k) * V;
    rc = input_scale(u, r);
    if (rc) break;
    target_kernel<<<grid_for(V), kThreads, 0, u->stream>>>(e, V, u->scale, u->tgt);
    rc = klaunch(u, "target");
    if (!rc) rc = forward(u);
    if (rc) break;
    if (u->loss_kind == CFD_UNET_LOSS_COS) {
      cos_dots_kernel<<<nb, kThreads, 0, u->stream>>>(u->z, u->tgt, u->nx, u->ny, u->nz, u->lossp);
      rc = klaunch(u, "loss dots");
      if (!rc) {
        cos_finalize_kernel<<<1, kThreads, 0, u->stream>>>(u->lossp, nb, u->scale);
        rc = klaunch(u, "loss finalize");
      }
      if (!rc) cos_grad_kernel<<<nb, kThreads, 0, u->stream>>>(u->z, u->tgt, u->nx, u->ny, u->nz, u->scale, u->gz);
    } else if (u->loss_kind == CFD_UNET_LOSS_ANORM) {
      loss_anorm_kernel<<<nb, kThreads, 0, u->stream>>>(u->z, u->tgt, u->nx, u->ny, u->nz, u->gz, u->lossp);
    } else {
      loss_kernel<<<nb, kThreads, 0, u->stream>>>(u->z, u->tgt, V, u->gz, u->lossp);
    }
    if (!rc) rc = klaunch(u, "loss");
    if (!rc) rc = backward(u);
    if (!rc) rc = uck(u, cudaMemcpyAsync(lp.data(), u->lossp, size_t(nb) * 8, cudaMemcpyDeviceToHost, u->stream), "copy loss");
    if (!rc) rc = uck(u, cudaStreamSynchronize(u->stream), "synchronize");
    for (int i = 0; i < nb && !rc; ++i) total += lp[size_t(i)];
  }
  if (rc) return rc;
  ++u->adam_t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, float(u->adam_t)), c2 = 1.f - std::pow(b2, float(u->adam_t));
  adam_kernel<<<grid_for(size_t(u->nparams)), kThreads, 0, u->stream>>>(u->w, u->m, u->v, u->g, size_t(u->nparams), lr,
                                                                         b1, b2, 1e-8f, c1, c2, 1.f / float(npairs));
  rc = klaunch(u, "adam");
  if (!rc) rc = pack_weights(u);
  int herr = 0;
  if (!rc) rc = uck(u, cudaMemcpyAsync(&herr, u->err, 4, cudaMemcpyDeviceToHost, u->stream), "copy err");
  if (!rc) rc = uck(u, cudaStreamSynchronize(u->stream), "synchronize");
  if (!rc && herr) rc = uerr(CFD_ERR_TIMEOUT, "unet: a tensor-core wait timed out");
  if (loss) *loss = float(total / npairs);
  return rc;
}

int cfd_unet_set_conv_mode(cfd_unet* u, int mode) {
  if (!u || mode < CFD_UNET_CONV_REGISTERS || mode > CFD_UNET_CONV_PERSISTENT)
    return uerr(CFD_ERR_INVALID_ARG, "unet: NULL handle or unknown convolution mode");
  u->conv_mode = mode;
  return CFD_OK;
}

int cfd_unet_set_wgrad_mode(cfd_unet* u, int mode) {
  if (!u || (mode != CFD_UNET_WGRAD_TENSOR && mode != CFD_UNET_WGRAD_CUDA_CORES))
    return uerr(CFD_ERR_INVALID_ARG, "unet: NULL handle or unknown weight-gradient mode");
  u->wgrad_mode = mode;
  return CFD_OK;
}

int cfd_unet_set_loss(cfd_unet* u, int kind) {
  if (!u || kind < CFD_UNET_LOSS_MSE || kind > CFD_UNET_LOSS_COS) return uerr(CFD_ERR_INVALID_ARG, "unet: bad loss kind");
  u->loss_kind = kind;
  return CFD_OK;
}

int cfd_unet_read_tensor(cfd_unet* u, int which, void* host, int64_t count) {
  if (!u || !host) return uerr(CFD_ERR_INVALID_ARG, "unet: NULL argument");
  const size_t V = size_t(u->nx) * u->ny * u->nz;
  const void* src = nullptr;
  size_t bytes = 0;
  if (which >= 0 && which < 26) {
    src = u->tens[which];
    bytes = u->tens_count[which] * 2;
    if (size_t(count) != u->tens_count[which]) return uerr(CFD_ERR_INVALID_ARG, "unet: tensor %d has %zu elements", which, u->tens_count[which]);
  } else if (which == CFD_UNET_T_OUT || which == CFD_UNET_T_TARGET) {
    src = which == CFD_UNET_T_OUT ? static_cast<const void*>(u->z) : static_cast<const void*>(u->tgt);
    bytes = V * 4;
    if (size_t(count) != V) return uerr(CFD_ERR_INVALID_ARG, "unet: tensor %d has %zu elements", which, V);
  } else if (which == CFD_UNET_T_GRAD || which == CFD_UNET_T_ADAM_M || which == CFD_UNET_T_ADAM_V) {
    src = which == CFD_UNET_T_GRAD ? u->g : (which == CFD_UNET_T_ADAM_M ? u->m : u->v);
    bytes = size_t(u->nparams) * 4;
    if (count != u->nparams) return uerr(CFD_ERR_INVALID_ARG, "unet: tensor %d has %lld elements", which, (long long)u->nparams);
  } else {
    return uerr(CFD_ERR_INVALID_ARG, "unet: unknown tensor %d", which);
  }
  int rc = uck(u, cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, u->stream), "copy tensor");
  if (!rc) rc = uck(u, cudaStreamSynchronize(u->stream), "synchronize");
  return rc;
}

int cfd_unet_fpcg_solve(cfd_unet* u, const double* b_dev, double* x_dev, double rtol, int32_t max_iters,
                        cfd_solve_stats* stats) {
  if (!u || !b_dev || !x_dev) return uerr(CFD_ERR_INVALID_ARG, "fpcg: NULL argument");
  if (!(rtol > 0.0 && rtol < 1.0) || max_iters < 0) return uerr(CFD_ERR_INVALID_ARG, "fpcg: rtol in (0, 1), max_iters >= 0");
  const GridDims gd{u->nx, u->ny, u->nz};
  const size_t n = gd.count();
  if (max_iters == 0) max_iters = 20 * std::max(u->nx, std::max(u->ny, u->nz));
  const int tz = solve_tile_depth(gd.mz);
  cudaStream_t s = u->stream;
  FpcgScalars h{};
  int rc = CFD_OK;
  auto launched = [&](const char* what) { if (!rc) rc = klaunch(u, what); return rc == CFD_OK; };
  auto scalar = [&](int op, int nb) {
    fpcg_scalar_kernel<<<1, kThreads, 0, s>>>(op, u->cg_parts, nb, n, u->cg_sc);
    return launched("fpcg scalar");
  };
  auto dot = [&](const double* a, const double* b, const double* c) {
    dot2_kernel<<<kDotBlocks, kThreads, 0, s>>>(a, b, c, n, u->cg_parts);
    return launched("fpcg dot");
  };
  auto apply_a = [&](const double* x, double* y) {
    if (!rc) rc = uck(u, launch_apply_poisson(gd, x, y, tz, s, &u->launches), "fpcg apply");
    return rc == CFD_OK;
  };
  auto read_scalars = [&]() {
    if (!rc) rc = uck(u, cudaMemcpyAsync(&h, u->cg_sc, sizeof(h), cudaMemcpyDeviceToHost, s), "copy scalars");
    if (!rc) rc = uck(u, cudaStreamSynchronize(s), "synchronize");
    return rc == CFD_OK;
  };
  // z = M(r): the network, or the identity on the plain-CG fallback
  bool plain = false;
  auto precondition = [&]() {
    if (rc) return false;
    if (plain) {
      rc = uck(u, cudaMemcpyAsync(u->cg_z, u->cg_r, n * 8, cudaMemcpyDeviceToDevice, s), "copy z");
    } else {
      rc = cfd_unet_apply(u, u->cg_r, u->cg_z);
    }
    return rc == CFD_OK;
  };
  // restart from the true residual of the current x: r = b - A x, z = M(r), p = z
  auto restart = [&](bool zero_x) {
    if (zero_x) {
      if (!rc) rc = uck(u, cudaMemsetAsync(x_dev, 0, n * 8, s), "memset x");
      residual_kernel<<<grid_for(n), kThreads, 0, s>>>(u->cg_b, nullptr, n, u->cg_r);
    } else {
      apply_a(x_dev, u->cg_q);
      residual_kernel<<<grid_for(n), kThreads, 0, s>>>(u->cg_b, u->cg_q, n, u->cg_r);
    }
    launched("fpcg residual");
    precondition();
    dot(u->cg_z, u->cg_r, nullptr);
    scalar(kOpRZ, kDotBlocks);
    direction_kernel<<<grid_for(n), kThreads, 0, s>>>(u->cg_z, u->cg_p, n, u->cg_sc, 1);
    return launched("fpcg direction");
  };

  // b <- b - mean(b); ||b||^2
  if (!rc) rc = uck(u, cudaMemsetAsync(u->cg_sc, 0, sizeof(FpcgScalars), s), "memset scalars");
  dot(b_dev, nullptr, nullptr);
  scalar(kOpMean, kDotBlocks);
  sub_mean_kernel<<<grid_for(n), kThreads, 0, s>>>(b_dev, n, u->cg_sc, u->cg_b);
  launched("fpcg mean");
  dot(u->cg_b, u->cg_b, nullptr);
  scalar(kOpBB, kDotBlocks);
  if (!read_scalars()) return rc;
  const double bb = h.bb;
  const double tol2 = rtol * rtol * bb;
  int iters = 0, plain_iters = 0, restarts = 0, status = CFD_OK;
  double rel = 0.0;
  if (bb == 0.0) {
    if (!rc) rc = uck(u, cudaMemsetAsync(x_dev, 0, n * 8, s), "memset x");
  } else {
    constexpr int kMaxRestarts = 8;
    constexpr int kStagnation = 50;  // iterations without halving the best residual
    restart(true);
    double best = bb;
    int since_best = 0;
    while (!rc) {
      if (!read_scalars()) break;
      if (h.flag) {
        // breakdown of the preconditioned recurrence (p.q <= 0, z.r = 0 or
        // non-finite): continue as plain CG from the current iterate
        if (plain) { status = CFD_ERR_BREAKDOWN; break; }
        plain = true;
        ++restarts;
        if (!rc) rc = uck(u, cudaMemsetAsync(&u->cg_sc->flag, 0, sizeof(int), s), "memset flag");
        restart(false);
        continue;
      }
      if (iters >= max_iters) { status = CFD_ERR_NOT_CONVERGED; break; }
      // one flexible CG iteration
      apply_a(u->cg_p, u->cg_q);
      dot(u->cg_p, u->cg_q, nullptr);
      scalar(kOpAlpha, kDotBlocks);
      xr_update_kernel<<<kDotBlocks, kThreads, 0, s>>>(x_dev, u->cg_r, u->cg_p, u->cg_q, n, u->cg_sc, u->cg_parts);
      launched("fpcg update");
      scalar(kOpRR, kDotBlocks);
      ++iters;
      if (plain) ++plain_iters;
      if (!read_scalars()) break;
      if (h.flag) continue;
      if (h.rr <= tol2) {
        // judge by the FP64 true residual; restart from it if the recursion drifted
        apply_a(x_dev, u->cg_q);
        residual_kernel<<<grid_for(n), kThreads, 0, s>>>(u->cg_b, u->cg_q, n, u->cg_r);
        launched("fpcg residual");
        dot(u->cg_r, u->cg_r, nullptr);
        scalar(kOpRR, kDotBlocks);
        if (!read_scalars()) break;
        if (h.rr <= tol2) break;
        if (++restarts > kMaxRestarts) { status = CFD_ERR_NOT_CONVERGED; break; }
        precondition();
        dot(u->cg_z, u->cg_r, nullptr);
        scalar(kOpRZ, kDotBlocks);
        direction_kernel<<<grid_for(n), kThreads, 0, s>>>(u->cg_z, u->cg_p, n, u->cg_sc, 1);
        launched("fpcg direction");
        continue;
      }
      if (h.rr < 0.25 * best) {
        best = h.rr;
        since_best = 0;
      } else if (!plain && ++since_best >= kStagnation) {
        plain = true;  // stagnation of the learned preconditioner: plain CG
        ++restarts;
        restart(false);
        continue;
      }
      // z = M(r); beta (Polak-Ribiere); p = z + beta p
      precondition();
      dot(u->cg_z, u->cg_r, u->cg_q);
      scalar(kOpBeta, kDotBlocks);
      direction_kernel<<<grid_for(n), kThreads, 0, s>>>(u->cg_z, u->cg_p, n, u->cg_sc, 0);
      launched("fpcg direction");
    }
    if (rc) return rc;
    // final true residual
    apply_a(x_dev, u->cg_q);
    residual_kernel<<<grid_for(n), kThreads, 0, s>>>(u->cg_b, u->cg_q, n, u->cg_r);
    launched("fpcg residual");
    dot(u->cg_r, u->cg_r, nullptr);
    scalar(kOpRR, kDotBlocks);
    if (!read_scalars()) return rc;
    rel = std::sqrt(h.rr / bb);
    if (status == CFD_OK && !(h.rr <= tol2)) status = CFD_ERR_NOT_CONVERGED;
  }
  if (rc) return rc;
  int herr = 0;
  rc = uck(u, cudaMemcpyAsync(&herr, u->err, 4, cudaMemcpyDeviceToHost, s), "copy err");
  if (!rc) rc = uck(u, cudaStreamSynchronize(s), "synchronize");
  if (rc) return rc;
  if (herr) status = CFD_ERR_TIMEOUT;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iters = iters;
    stats->outer_iters = plain_iters;
    stats->restarts = restarts;
    stats->status = status;
    stats->rel_resid = rel;
    stats->b_norm = std::sqrt(bb);
  }
  if (status != CFD_OK)
    uerr(status, "fpcg: status %d after %d iterations (relative residual %.3e)", status, iters, rel);
  return status;
}

int64_t cfd_unet_launch_count(const cfd_unet* u) { return u ? u->launches : 0; }

const char* cfd_unet_last_error(void) { return g_unet_err; }

}  // extern "C"
