// Learned 3D-convolutional preconditioner: BF16 tensor-core (tcgen05)
// convolution kernels, U-Net forward / backward, Adam.
//
// The paper (Sec. 3.1) preconditions its pressure CG with DIC or Jacobi and
// names "other preconditioners" as future work (Sec. 5).  This file provides
// a learned one: a 3-level U-Net z = U(r) applied inside flexible CG.
//
// Convolution = implicit GEMM on the 5th-generation tensor cores: one CTA
// computes a tile of 128 output voxels x Cout channels; the K dimension runs
// over (tap, 16-channel block).  For every K chunk all 128 threads gather
// the shifted input rows (channels-last BF16, zero outside the grid) and the
// weight rows into a shared-memory stage laid out as K-major core matrices,
// one thread issues tcgen05.mma (M = 128, N = Cout, K = 16, FP32
// accumulation in tensor memory) and commits it to the stage's mbarrier, so
// gathering the next stages overlaps the running MMAs (4-stage ring).  The
// epilogue reads the accumulator with tcgen05.ld, adds the bias and stores
// BF16 (or FP32).  Every mbarrier wait is bounded.
//
// Layer building blocks (all convolutions stride 1):
//   * 3x3x3 or 1x1x1 convolution, input = one tensor or the channel
//     concatenation of two (skip connections, read in place), output
//     optionally split over two tensors by channel (backward of a concat);
//   * a tap-packed mode for single-channel inputs (the first layer: K = 27
//     taps padded to 32 instead of 27 x 16);
//   * 2x average pooling and nearest 2x up-sampling (and their adjoints).

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "cfd_internal.h"
#include "tc_common.cuh"
#include "unet.h"

namespace cfd {

namespace {

constexpr int kConvThreads = 128;  // one thread per output row of the tile
constexpr int kConvStages = 4;
constexpr unsigned long long kConvWaitNs = 1000000000ull;

__device__ __forceinline__ void store16B(unsigned char* dst, uint4 v) { *reinterpret_cast<uint4*>(dst) = v; }

// Row of 16 BF16 K-values for the A operand of voxel v, tap offset
// (dx, dy, dz), channel block cb; zero outside the grid or past Cin.
__device__ __forceinline__ void gather_row(const ConvArgs& a, int x, int y, int z, bool valid, int tap, int cb,
                                           uint4& lo, uint4& hi) {
  lo = make_uint4(0, 0, 0, 0);
  hi = lo;
  if (!valid) return;
  if (a.packed) {
    // 16 taps of the single input channel: taps 16 cb .. 16 cb + 15
    __nv_bfloat16 vals[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int t = 16 * cb + j;
      __nv_bfloat16 val = __float2bfloat16(0.f);
      if (t < 27) {
        const int xx = x + (t % 3) - 1, yy = y + (t / 3) % 3 - 1, zz = z + t / 9 - 1;
        if (xx >= 0 && xx < a.nx && yy >= 0 && yy < a.ny && zz >= 0 && zz < a.nz)
          val = a.src0[(size_t(zz) * a.ny + yy) * a.nx + xx];
      }
      vals[j] = val;
    }
    lo = *reinterpret_cast<uint4*>(&vals[0]);
    hi = *reinterpret_cast<uint4*>(&vals[8]);
    return;
  }
  int dx = 0, dy = 0, dz = 0;
  if (a.ks == 3) {
    dx = tap % 3 - 1;
    dy = (tap / 3) % 3 - 1;
    dz = tap / 9 - 1;
  }
  const int xx = x + dx, yy = y + dy, zz = z + dz;
  if (xx < 0 || xx >= a.nx || yy < 0 || yy >= a.ny || zz < 0 || zz >= a.nz) return;
  const size_t nb = (size_t(zz) * a.ny + yy) * a.nx + xx;
  const int c = 16 * cb;
  const __nv_bfloat16* src;
  int cs, cc;
  if (c < a.c0) {
    src = a.src0;
    cs = a.c0;
    cc = c;
  } else {
    src = a.src1;
    cs = a.c1;
    cc = c - a.c0;
  }
  if (cs % 16 == 0) {
    const uint4* p = reinterpret_cast<const uint4*>(src + nb * cs + cc);
    lo = p[0];
    hi = p[1];
  } else {
    // narrow source (fewer than 16 channels): element loads, zero padding
    __nv_bfloat16 vals[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) vals[j] = (cc + j < cs) ? src[nb * cs + cc + j] : __float2bfloat16(0.f);
    lo = *reinterpret_cast<uint4*>(&vals[0]);
    hi = *reinterpret_cast<uint4*>(&vals[8]);
  }
}

template <int NOUT>
__global__ void __launch_bounds__(kConvThreads) conv3d_tc_kernel(const ConvArgs a) {
  constexpr int kA = 128 * 16 * 2;          // A stage bytes
  constexpr int kB = NOUT * 16 * 2;         // B stage bytes
  constexpr int kStage = kA + kB;
  constexpr uint32_t kTmemCols = NOUT < 32 ? 32 : NOUT;
  __shared__ __align__(1024) unsigned char smem[kConvStages * kStage];
  __shared__ __align__(8) uint64_t bar[kConvStages];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;

  const int t = threadIdx.x;
  const size_t V = size_t(a.nx) * a.ny * a.nz;
  const size_t v = size_t(blockIdx.x) * 128 + t;
  const bool valid = v < V;
  int x = 0, y = 0, z = 0;
  if (valid) {
    x = int(v % a.nx);
    y = int((v / a.nx) % a.ny);
    z = int(v / (size_t(a.nx) * a.ny));
  }
  const int cin_pad = (a.c0 + a.c1 + 15) / 16 * 16;
  const int cblocks = a.packed ? 2 : cin_pad / 16;
  const int taps = a.packed ? 1 : a.ks * a.ks * a.ks;
  const int chunks = taps * cblocks;

  if (t == 0) {
    for (int s = 0; s < kConvStages; ++s) tc::mbar_init(&bar[s], 1);
    tc::mbar_fence_init();
    s_fail = 0;
  }
  if (t < 32) tc::tmem_alloc(&s_tmem, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc::idesc_bf16_f32(128, NOUT);

  for (int k = 0; k < chunks; ++k) {
    const int s = k % kConvStages;
    unsigned char* sa = smem + s * kStage;
    unsigned char* sb = sa + kA;
    if (k >= kConvStages) {
      // the MMA that read this stage (chunk k - stages) must be complete
      if (!tc::mbar_wait(&bar[s], unsigned((k / kConvStages - 1) & 1), kConvWaitNs)) s_fail = 1;
    }
    const int tap = k / cblocks, cb = k % cblocks;
    uint4 lo, hi;
    gather_row(a, x, y, z, valid, tap, cb, lo, hi);
    store16B(sa + tc::core_offset(t, 0), lo);
    store16B(sa + tc::core_offset(t, 1), hi);
    if (t < NOUT) {
      const __nv_bfloat16* wr = a.packed ? a.w + size_t(t) * 32 + 16 * cb
                                         : a.w + (size_t(tap) * NOUT + t) * cin_pad + 16 * cb;
      const uint4* wp = reinterpret_cast<const uint4*>(wr);
      store16B(sb + tc::core_offset(t, 0), wp[0]);
      store16B(sb + tc::core_offset(t, 1), wp[1]);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (s_fail) break;
    tc::fence_after_sync();
    if (t == 0) {
      tc::mma_bf16(tmem, tc::smem_desc(tc::smem_addr(sa), 128, 256), tc::smem_desc(tc::smem_addr(sb), 128, 256), idesc,
                   k > 0);
      tc::mma_commit(&bar[s]);
    }
  }
  // all MMAs done: wait for the last commit (tracks every earlier MMA)
  if (!s_fail && chunks > 0) {
    const int s = (chunks - 1) % kConvStages;
    if (!tc::mbar_wait(&bar[s], unsigned(((chunks - 1) / kConvStages) & 1), kConvWaitNs)) s_fail = 1;
  }
  __syncthreads();
  tc::fence_after_sync();
  if (s_fail) {
    if (t == 0) atomicExch(a.err, 1);
  } else {
    const int w = t / 32;
#pragma unroll
    for (int c0 = 0; c0 < NOUT; c0 += 16) {
      float acc[16];
      tc::tmem_ld16(tmem + (uint32_t(w * 32) << 16) + uint32_t(c0), acc);
      if (valid) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + j;
          if (c >= a.cout) break;
          float val = acc[j] + (a.bias ? a.bias[c] : 0.f);
          if (a.dst_f32) {
            a.dst_f32[v * a.cout + c] = val;
          } else if (c < a.split) {
            a.dst0[v * a.split + c] = __float2bfloat16(val);
          } else {
            a.dst1[v * (a.cout - a.split) + (c - a.split)] = __float2bfloat16(val);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t < 32) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

cudaError_t launch_conv3d(const ConvArgs& a, int nout_pad, cudaStream_t s) {
  const size_t V = size_t(a.nx) * a.ny * a.nz;
  const unsigned grid = unsigned((V + 127) / 128);
  switch (nout_pad) {
    case 16: conv3d_tc_kernel<16><<<grid, kConvThreads, 0, s>>>(a); break;
    case 32: conv3d_tc_kernel<32><<<grid, kConvThreads, 0, s>>>(a); break;
    case 64: conv3d_tc_kernel<64><<<grid, kConvThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace cfd

// ---------------------------------------------------------------------------
// C-ABI: one convolution (the U-Net building block), for direct checks.
// ---------------------------------------------------------------------------
extern "C" int cfd_conv3d_bf16(int nx, int ny, int nz, const void* src0, int c0, const void* src1, int c1, int ks,
                               const void* weights, const float* bias, int cout, int nout_pad, void* dst_bf16,
                               float* dst_f32, int* err_dev, void* stream) {
  using namespace cfd;
  if (nx < 1 || ny < 1 || nz < 1 || !src0 || c0 < 1 || c1 < 0 || (c1 > 0 && !src1) || (ks != 1 && ks != 3) ||
      !weights || cout < 1 || cout > nout_pad || (nout_pad != 16 && nout_pad != 32 && nout_pad != 64) ||
      (!dst_bf16 && !dst_f32) || !err_dev)
    return cfd_internal_error(-1, "conv3d: invalid arguments");
  if (c1 > 0 && c0 % 16 != 0) return cfd_internal_error(-1, "conv3d: the first source of a concatenation needs 16k channels");
  ConvArgs a{};
  a.nx = nx; a.ny = ny; a.nz = nz;
  a.src0 = static_cast<const __nv_bfloat16*>(src0);
  a.c0 = c0;
  a.src1 = static_cast<const __nv_bfloat16*>(src1);
  a.c1 = c1;
  a.ks = ks;
  a.packed = (c0 == 1 && c1 == 0 && ks == 3) ? 1 : 0;
  a.w = static_cast<const __nv_bfloat16*>(weights);
  a.bias = bias;
  a.cout = cout;
  a.dst0 = static_cast<__nv_bfloat16*>(dst_bf16);
  a.dst1 = nullptr;
  a.split = cout;
  a.dst_f32 = dst_f32;
  a.err = err_dev;
  const cudaError_t e = launch_conv3d(a, nout_pad, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cfd_internal_error(-2, "conv3d launch: %s", cudaGetErrorString(e));
  return 0;
}
