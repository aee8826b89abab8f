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
// the shifted input rows (BF16 octet planes, zero outside the grid) and the
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
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

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
  const size_t V = size_t(a.nx) * a.ny * a.nz;
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
  if (cs % 8 == 0) {
    // two octet planes: channels cc .. cc + 7 and cc + 8 .. cc + 15
    lo = *reinterpret_cast<const uint4*>(src + oct_index(nb, cc, cs, V));
    if (cc + 8 < cs) hi = *reinterpret_cast<const uint4*>(src + oct_index(nb, cc + 8, cs, V));
  } else {
    // narrow source (fewer than 8 channels): element loads, zero padding
    __nv_bfloat16 vals[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) vals[j] = (cc + j < cs) ? src[oct_index(nb, cc + j, cs, V)] : __float2bfloat16(0.f);
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
            a.dst0[oct_index(v, c, a.split, V)] = __float2bfloat16(val);
          } else {
            a.dst1[oct_index(v, c - a.split, a.cout - a.split, V)] = __float2bfloat16(val);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t < 32) tc::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Tiled 3x3x3 convolution: one TMA-staged input tile per 16-channel block,
// every tap read in place by shifting the A descriptor.
//
// A CTA owns an output box of xc x ty x tz voxels.  For each 16-channel
// block, two TMA loads bring the input box with a one-voxel halo ((xc + 2) x
// (ty + 2) x (tz + 2) voxels, zero outside the grid) into two shared-memory
// planes, one per 8-channel K-half; voxel (x, y, z) of the box is "row" r =
// (z (ty + 2) + y)(xc + 2) + x at byte r * 16 of each plane.  Read with a
// stride byte offset of 128 (8-row groups back to back) and a leading byte
// offset of the plane distance, any 128 consecutive rows form a valid K-major
// A operand, so the operand of tap (dx, dy, dz) for output rows [s, s + 128)
// is simply rows [s + dz (ty+2)(xc+2) + dy (xc+2) + dx, ...): one tile load
// serves all 27 taps.  Output rows are taken in M-blocks of 128 consecutive
// rows (one x-line each when xc = 126 ... 128, "line mode"; otherwise
// consecutive rows from the first interior row); rows that fall on halo
// voxels are computed and discarded.  M-block j accumulates in TMEM columns
// [j NOUT, (j + 1) NOUT).  The weights of the channel block (27 taps x NOUT
// rows x 16) are copied to shared memory as K-major core matrices.
// ---------------------------------------------------------------------------

constexpr int kTileMaxMB = 8;
constexpr int kTileSmemMax = 210 * 1024;  // dynamic shared memory cap (static use is about 1 KB)

struct ConvTileArgs {
  CUtensorMap map0;            // src0 [nz][ny][nx][c0], box {8, bx, by, bz}
  CUtensorMap map1;            // src1 (concatenation) or unused
  const __nv_bfloat16* src0;   // the same tensors (octet planes), for row copies
  const __nv_bfloat16* src1;
  int nx, ny, nz;
  int c0, c1;
  int xc, ty, tz;              // output box
  int bx, by, bz;              // input box (output box + halo)
  int line_mode;
  int mb;                      // M-blocks per CTA
  int plane;                   // bytes between the two K-half planes (16-multiple)
  int tiles_x, tiles_y;
  const __nv_bfloat16* w;      // [27][NOUT][cin_pad]
  const __nv_bfloat16* w_cm;   // or null: [cb][27] x (NOUT x 16 K-major core matrices)
  int cin_pad;
  const float* bias;
  int cout;
  __nv_bfloat16* dst0;
  __nv_bfloat16* dst1;
  int split;
  int* err;
};

__device__ __forceinline__ int tile_block_start(const ConvTileArgs& a, int j) {
  if (a.line_mode) return ((1 + j / a.ty) * a.by + 1 + j % a.ty) * a.bx + 1;
  return (a.by + 1) * a.bx + 1 + 128 * j;
}

template <int NOUT>
__global__ void __launch_bounds__(kConvThreads) conv3d_tile_kernel(const __grid_constant__ ConvTileArgs a) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar_tma, bar_mma;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  __shared__ int s_start[kTileMaxMB];  // first row of each M-block
  constexpr int kBTap = NOUT * 32;  // bytes of one tap's B operand
  unsigned char* plane0 = dsm;
  unsigned char* plane1 = dsm + a.plane;
  unsigned char* sb = dsm + 2 * a.plane;

  const int t = threadIdx.x;
  const int tx = blockIdx.x % a.tiles_x;
  const int ty_ = (blockIdx.x / a.tiles_x) % a.tiles_y;
  const int tz_ = blockIdx.x / (a.tiles_x * a.tiles_y);
  const int x0 = tx * a.xc, y0 = ty_ * a.ty, z0 = tz_ * a.tz;
  const int cb0 = a.c0 / 16;
  const int ncb = cb0 + a.c1 / 16;
  const uint32_t tmem_cols = (a.mb * NOUT <= 32) ? 32u : (a.mb * NOUT <= 64 ? 64u : (a.mb * NOUT <= 128 ? 128u : (a.mb * NOUT <= 256 ? 256u : 512u)));
  const unsigned box_bytes = unsigned(a.bx) * a.by * a.bz * 16;

  if (t == 0) {
    tc::mbar_init(&bar_tma, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_fence_init();
    s_fail = 0;
  }
  if (t < kTileMaxMB) s_start[t] = t < a.mb ? tile_block_start(a, t) : 0;
  if (t < 32) tc::tmem_alloc(&s_tmem, tmem_cols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc::idesc_bf16_f32(128, NOUT);
  const int row_z = a.by * a.bx;

  bool tma_pending = false;
  for (int cb = 0; cb < ncb; ++cb) {
    if (cb > 0) {
      // the MMAs of the previous channel block read these buffers
      if (!tc::mbar_wait(&bar_mma, unsigned((cb - 1) & 1), kConvWaitNs)) s_fail = 1;
    }
    // weights of this channel block: [tap][NOUT][16] as K-major core matrices
    for (int i = t; i < 27 * NOUT * 2; i += kConvThreads) {
      const int h = i & 1, o = (i >> 1) % NOUT, tap = (i >> 1) / NOUT;
      const uint4 v = *reinterpret_cast<const uint4*>(a.w + (size_t(tap) * NOUT + o) * a.cin_pad + 16 * cb + 8 * h);
      store16B(sb + tap * kBTap + tc::core_offset(o, h), v);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (s_fail) break;
    if (t == 0) {
      const void* map = cb < cb0 ? static_cast<const void*>(&a.map0) : static_cast<const void*>(&a.map1);
      const int oct = 2 * (cb < cb0 ? cb : cb - cb0);
      tc::mbar_expect_tx(&bar_tma, 2 * box_bytes);
      tc::tma_load_5d(plane0, map, 0, x0 - 1, y0 - 1, z0 - 1, oct, &bar_tma);
      tc::tma_load_5d(plane1, map, 0, x0 - 1, y0 - 1, z0 - 1, oct + 1, &bar_tma);
    }
    tma_pending = true;
    if (!tc::mbar_wait(&bar_tma, unsigned(cb & 1), kConvWaitNs)) {
      s_fail = 1;
      break;
    }
    tma_pending = false;
    tc::fence_after_sync();
    if (t == 0) {
      // One thread issues 27 x mb MMAs; the descriptors differ only in their
      // start-address field (address >> 4 in the low bits), so they are
      // formed by adding row / tap offsets to two base descriptors.
      const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(plane0), uint32_t(a.plane), 128);
      const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(sb), 128, 256);
      int st[kTileMaxMB];
#pragma unroll
      for (int j = 0; j < kTileMaxMB; ++j) st[j] = s_start[j];
      int tap = 0;
      for (int dz = -1; dz <= 1; ++dz) {
        for (int dy = -1; dy <= 1; ++dy) {
          for (int dx = -1; dx <= 1; ++dx, ++tap) {
            const int off = dz * row_z + dy * a.bx + dx;
            const uint64_t bdesc = bdesc0 + uint64_t(tap * (kBTap >> 4));
            const bool acc = (cb | tap) != 0;
#pragma unroll
            for (int j = 0; j < kTileMaxMB; ++j)
              if (j < a.mb) tc::mma_bf16(tmem + uint32_t(j * NOUT), adesc0 + uint64_t(st[j] + off), bdesc, idesc, acc);
          }
        }
      }
      tc::mma_commit(&bar_mma);
    }
  }
  __syncthreads();
  if (!s_fail && ncb > 0) {
    if (!tc::mbar_wait(&bar_mma, unsigned((ncb - 1) & 1), kConvWaitNs)) s_fail = 1;
  }
  __syncthreads();
  tc::fence_after_sync();
  if (s_fail) {
    if (t == 0) atomicExch(a.err, 1);
    // let a copy still in flight land before the CTA's shared memory goes away
    if (tma_pending) tc::mbar_wait(&bar_tma, unsigned((ncb - 1) & 1), kConvWaitNs);
  } else {
    const int w = t / 32;
    const int bxby = a.bx * a.by;
    const size_t Vt = size_t(a.nx) * a.ny * a.nz;
    for (int j = 0; j < a.mb; ++j) {
      const int row = s_start[j] + t;  // this thread's TMEM lane = row t of block j
      const int zq = row / bxby, rem = row - zq * bxby;
      const int yq = rem / a.bx, xq = rem - yq * a.bx;
      const int gx = x0 + xq - 1, gy = y0 + yq - 1, gz = z0 + zq - 1;
      const bool valid = xq >= 1 && xq <= a.xc && yq >= 1 && yq <= a.ty && zq >= 1 && zq <= a.tz && gx < a.nx &&
                         gy < a.ny && gz < a.nz;
      const size_t v = (size_t(gz) * a.ny + gy) * a.nx + gx;
#pragma unroll
      for (int c0 = 0; c0 < NOUT; c0 += 16) {
        float acc[16];
        tc::tmem_ld16(tmem + (uint32_t(w * 32) << 16) + uint32_t(j * NOUT + c0), acc);
        if (valid && c0 < a.cout) {
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int cbase = c0 + 8 * half;
            if (cbase >= a.cout) break;
            __nv_bfloat16 o8[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) o8[k] = __float2bfloat16(acc[8 * half + k] + (a.bias ? a.bias[cbase + k] : 0.f));
            __nv_bfloat16* dst = cbase < a.split ? a.dst0 + oct_index(v, cbase, a.split, Vt)
                                                 : a.dst1 + oct_index(v, cbase - a.split, a.cout - a.split, Vt);
            *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(o8);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t < 32) tc::tmem_dealloc(tmem, tmem_cols);
}

// Two-stage pipelined variant for weights already in the shared-memory
// order (w_cm): one thread streams channel block cb + 1 (two TMA plane copies
// and one bulk copy of its 27 weight tiles) into the other stage while the
// tensor core runs the 27 x mb MMAs of block cb; the stage is refilled once
// the MMAs that read it have committed.  Other threads wait for the epilogue.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_addr(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_addr(bar))
               : "memory");
}

template <int NOUT, int STAGES>
__global__ void __launch_bounds__(kConvThreads) conv3d_tile_pipe_kernel(const __grid_constant__ ConvTileArgs a) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar_full[STAGES], bar_mma[STAGES];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  __shared__ int s_start[kTileMaxMB];
  constexpr int kBTap = NOUT * 32;
  constexpr unsigned kBBytes = 27u * kBTap;
  const size_t stage_bytes = 2 * size_t(a.plane) + kBBytes;

  const int t = threadIdx.x;
  const int tx = blockIdx.x % a.tiles_x;
  const int ty_ = (blockIdx.x / a.tiles_x) % a.tiles_y;
  const int tz_ = blockIdx.x / (a.tiles_x * a.tiles_y);
  const int x0 = tx * a.xc, y0 = ty_ * a.ty, z0 = tz_ * a.tz;
  const int cb0 = a.c0 / 16;
  const int ncb = cb0 + a.c1 / 16;
  const uint32_t tmem_cols = (a.mb * NOUT <= 32) ? 32u : (a.mb * NOUT <= 64 ? 64u : (a.mb * NOUT <= 128 ? 128u : (a.mb * NOUT <= 256 ? 256u : 512u)));
  const unsigned box_bytes = unsigned(a.bx) * a.by * a.bz * 16;

  if (t == 0) {
    for (int q = 0; q < STAGES; ++q) {
      tc::mbar_init(&bar_full[q], 1);
      tc::mbar_init(&bar_mma[q], 1);
    }
    tc::mbar_fence_init();
    s_fail = 0;
  }
  if (t < kTileMaxMB) s_start[t] = t < a.mb ? tile_block_start(a, t) : 0;
  if (t < 32) tc::tmem_alloc(&s_tmem, tmem_cols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  if (t == 0) {
    const uint32_t idesc = tc::idesc_bf16_f32(128, NOUT);
    const int row_z = a.by * a.bx;
    int st[kTileMaxMB];
#pragma unroll
    for (int j = 0; j < kTileMaxMB; ++j) st[j] = s_start[j];
    // stage of channel block q: q % STAGES; its use count: q / STAGES
    auto issue = [&](int cb) {
      const int sg = cb % STAGES;
      unsigned char* base = dsm + size_t(sg) * stage_bytes;
      const void* map = cb < cb0 ? static_cast<const void*>(&a.map0) : static_cast<const void*>(&a.map1);
      const int oct = 2 * (cb < cb0 ? cb : cb - cb0);
      tc::mbar_expect_tx(&bar_full[sg], 2 * box_bytes + kBBytes);
      tc::tma_load_5d(base, map, 0, x0 - 1, y0 - 1, z0 - 1, oct, &bar_full[sg]);
      tc::tma_load_5d(base + a.plane, map, 0, x0 - 1, y0 - 1, z0 - 1, oct + 1, &bar_full[sg]);
      bulk_copy_g2s(base + 2 * size_t(a.plane), a.w_cm + size_t(cb) * (kBBytes / 2), kBBytes, &bar_full[sg]);
    };
    int issued = 0, consumed = 0;
    bool fail = false;
    issue(0);
    issued = 1;
    for (int cb = 0; cb < ncb && !fail; ++cb) {
      if (STAGES > 1 && cb + 1 < ncb) {
        // the stage of cb + 1 was last read by the MMAs of cb + 1 - STAGES
        const int prev = cb + 1 - STAGES;
        if (prev >= 0 &&
            !tc::mbar_wait(&bar_mma[prev % STAGES], unsigned((prev / STAGES) & 1), kConvWaitNs)) {
          fail = true;
          break;
        }
        issue(cb + 1);
        issued = cb + 2;
      }
      if (!tc::mbar_wait(&bar_full[cb % STAGES], unsigned((cb / STAGES) & 1), kConvWaitNs)) {
        fail = true;
        break;
      }
      consumed = cb + 1;
      tc::fence_after_sync();
      unsigned char* base = dsm + size_t(cb % STAGES) * stage_bytes;
      const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(base), uint32_t(a.plane), 128);
      const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(base + 2 * size_t(a.plane)), 128, 256);
      int tap = 0;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx, ++tap) {
            const int off = dz * row_z + dy * a.bx + dx;
            const uint64_t bdesc = bdesc0 + uint64_t(tap * (kBTap >> 4));
            const bool acc = (cb | tap) != 0;
#pragma unroll
            for (int j = 0; j < kTileMaxMB; ++j)
              if (j < a.mb) tc::mma_bf16(tmem + uint32_t(j * NOUT), adesc0 + uint64_t(st[j] + off), bdesc, idesc, acc);
          }
      tc::mma_commit(&bar_mma[cb % STAGES]);
      if (STAGES == 1 && cb + 1 < ncb) {
        // one stage: the next block's copies wait for these MMAs
        if (!tc::mbar_wait(&bar_mma[0], unsigned(cb & 1), kConvWaitNs)) {
          fail = true;
          break;
        }
        issue(cb + 1);
        issued = cb + 2;
      }
    }
    if (!fail && ncb > 0) {
      if (!tc::mbar_wait(&bar_mma[(ncb - 1) % STAGES], unsigned(((ncb - 1) / STAGES) & 1), kConvWaitNs)) fail = true;
    }
    if (fail) {
      s_fail = 1;
      // let copies still in flight land before the CTA's shared memory goes away
      for (int cb = consumed; cb < issued; ++cb)
        tc::mbar_wait(&bar_full[cb % STAGES], unsigned((cb / STAGES) & 1), kConvWaitNs);
      if (consumed > 0)
        tc::mbar_wait(&bar_mma[(consumed - 1) % STAGES], unsigned(((consumed - 1) / STAGES) & 1), kConvWaitNs);
    }
  }
  __syncthreads();
  tc::fence_after_sync();
  if (s_fail) {
    if (t == 0) atomicExch(a.err, 1);
  } else {
    const int w = t / 32;
    const int bxby = a.bx * a.by;
    const size_t Vt = size_t(a.nx) * a.ny * a.nz;
    for (int j = 0; j < a.mb; ++j) {
      const int row = s_start[j] + t;
      const int zq = row / bxby, rem = row - zq * bxby;
      const int yq = rem / a.bx, xq = rem - yq * a.bx;
      const int gx = x0 + xq - 1, gy = y0 + yq - 1, gz = z0 + zq - 1;
      const bool valid = xq >= 1 && xq <= a.xc && yq >= 1 && yq <= a.ty && zq >= 1 && zq <= a.tz && gx < a.nx &&
                         gy < a.ny && gz < a.nz;
      const size_t v = (size_t(gz) * a.ny + gy) * a.nx + gx;
#pragma unroll
      for (int c0 = 0; c0 < NOUT; c0 += 16) {
        float acc[16];
        tc::tmem_ld16(tmem + (uint32_t(w * 32) << 16) + uint32_t(j * NOUT + c0), acc);
        if (valid && c0 < a.cout) {
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int cbase = c0 + 8 * half;
            if (cbase >= a.cout) break;
            __nv_bfloat16 o8[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) o8[k] = __float2bfloat16(acc[8 * half + k] + (a.bias ? a.bias[cbase + k] : 0.f));
            __nv_bfloat16* dst = cbase < a.split ? a.dst0 + oct_index(v, cbase, a.split, Vt)
                                                 : a.dst1 + oct_index(v, cbase - a.split, a.cout - a.split, Vt);
            *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(o8);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t < 32) tc::tmem_dealloc(tmem, tmem_cols);
}

// Persistent warp-specialised variant (weights in shared-memory order, as
// the pipelined kernel): one CTA per SM walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; warp 0 copies each (tile, channel block)
// unit into one of kWsStages shared-memory stages: the input box's x-rows of
// the two octet planes as contiguous bulk copies (one per row, up to 130
// voxels of 16 bytes; the box image is the one the TMA copies of the other
// kernels produce, with zeros outside the grid written by the warp) and the
// block's weights as one bulk copy; one lane of warp 1
// waits for a unit, issues its 27 x mb MMAs into one of two TMEM
// accumulators (tiles alternate between them) and commits to the stage's
// "empty" barrier, and after a tile's last block also to the accumulator's
// "full" barrier; warps 2-5 (one TMEM lane quarter each) read a finished
// accumulator, add the bias, store, and release it.  So the copies of the
// next unit, the MMAs of this one and the epilogue of the previous tile
// overlap.  The MMAs of a tile are those of the other kernels in the same
// order, so the results are bitwise equal.  Every wait is bounded; on a
// timeout the CTA lets its copies and MMAs in flight finish, sets *err and
// returns.
constexpr int kWsStages = 2;
constexpr int kWsThreads = 192;

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(b)) : "memory");
}

template <int NOUT>
__global__ void __launch_bounds__(kWsThreads, 1) conv3d_tile_ws_kernel(const __grid_constant__ ConvTileArgs a,
                                                                       int ntiles, unsigned stage_bytes) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar_full[kWsStages], bar_empty[kWsStages], bar_tfull[2], bar_tempty[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_start[kTileMaxMB];
  __shared__ volatile int s_fail;
  __shared__ volatile int s_issued, s_consumed, s_mma;  // units copied / awaited / whose MMAs were issued
  constexpr int kBTap = NOUT * 32;
  constexpr unsigned kBBytes = 27u * kBTap;
  const int t = threadIdx.x, warp = t / 32, lane = t % 32;
  const int cb0 = a.c0 / 16;
  const int ncb = cb0 + a.c1 / 16;
  const int acc_cols = a.mb * NOUT;
  const int need = 2 * acc_cols;
  const uint32_t tmem_cols = need <= 32 ? 32u : (need <= 64 ? 64u : (need <= 128 ? 128u : (need <= 256 ? 256u : 512u)));
  const int my_tiles = ntiles > int(blockIdx.x) ? (ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  const int units = my_tiles * ncb;
  auto origin = [&](int tl, int& x0, int& y0, int& z0) {
    const int g = int(blockIdx.x) + tl * int(gridDim.x);
    const int tx = g % a.tiles_x, ty_ = (g / a.tiles_x) % a.tiles_y, tz_ = g / (a.tiles_x * a.tiles_y);
    x0 = tx * a.xc;
    y0 = ty_ * a.ty;
    z0 = tz_ * a.tz;
  };

  if (t == 0) {
    for (int q = 0; q < kWsStages; ++q) {
      tc::mbar_init(&bar_full[q], 1);
      tc::mbar_init(&bar_empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&bar_tfull[q], 1);
      tc::mbar_init(&bar_tempty[q], 4);
    }
    tc::mbar_fence_init();
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    s_mma = 0;
  }
  if (t < kTileMaxMB) s_start[t] = t < a.mb ? tile_block_start(a, t) : 0;
  if (warp == 0) tc::tmem_alloc(&s_tmem, tmem_cols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {  // producer: the whole warp
    const int nrow = a.by * a.bz;  // x-rows of the input box per plane
    const size_t V = size_t(a.nx) * a.ny * a.nz;
    for (int u = 0; u < units; ++u) {
      const int sg = u % kWsStages;
      int ok = 1;
      if (lane == 0 && u >= kWsStages &&
          !tc::mbar_wait(&bar_empty[sg], unsigned(((u / kWsStages) - 1) & 1), kConvWaitNs))
        ok = 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok || s_fail) {
        if (lane == 0) s_fail = 1;
        break;
      }
      const int tl = u / ncb, cb = u % ncb;
      int x0, y0, z0;
      origin(tl, x0, y0, z0);
      unsigned char* base = dsm + size_t(sg) * stage_bytes;
      const __nv_bfloat16* src = cb < cb0 ? a.src0 : a.src1;
      const int oct = 2 * (cb < cb0 ? cb : cb - cb0);
      // the box's x-rows: voxels [xs, xs + bx) of row (y, z); the part inside
      // the grid, [vx0, vx1), is one contiguous run of 16-byte voxels in each
      // octet plane; the rest (and rows outside the grid) is zero
      const int xs = x0 - 1;
      const int vx0 = xs > 0 ? xs : 0, vx1 = xs + a.bx < a.nx ? xs + a.bx : a.nx;
      const int nvalid = vx1 > vx0 ? vx1 - vx0 : 0;
      auto row_valid = [&](int rr, int& gy, int& gz) {
        gy = y0 - 1 + rr % a.by;
        gz = z0 - 1 + rr / a.by;
        return nvalid > 0 && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
      };
      int nrows_valid = 0;
      for (int q = lane; q < 2 * nrow; q += 32) {
        const int h = q / nrow, rr = q % nrow;
        int gy, gz;
        const bool v = row_valid(rr, gy, gz);
        uint4* row = reinterpret_cast<uint4*>(base + h * size_t(a.plane) + size_t(rr) * a.bx * 16);
        const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
        if (!v) {
          for (int x = 0; x < a.bx; ++x) row[x] = z4;
        } else {
          for (int x = 0; x < vx0 - xs; ++x) row[x] = z4;
          for (int x = vx1 - xs; x < a.bx; ++x) row[x] = z4;
          nrows_valid += 1;
        }
      }
      for (int o = 16; o > 0; o >>= 1) nrows_valid += __shfl_down_sync(0xffffffffu, nrows_valid, o);
      tc::fence_proxy_async_smem();  // the zero fill is read by the tensor cores
      __syncwarp();
      if (lane == 0) tc::mbar_expect_tx(&bar_full[sg], unsigned(nrows_valid) * unsigned(nvalid) * 16u + kBBytes);
      __syncwarp();
      for (int q = lane; q < 2 * nrow; q += 32) {
        const int h = q / nrow, rr = q % nrow;
        int gy, gz;
        if (!row_valid(rr, gy, gz)) continue;
        unsigned char* dst = base + h * size_t(a.plane) + (size_t(rr) * a.bx + size_t(vx0 - xs)) * 16;
        const __nv_bfloat16* from = src + ((size_t(oct + h) * V + (size_t(gz) * a.ny + gy) * a.nx + vx0) * 8);
        bulk_copy_g2s(dst, from, unsigned(nvalid) * 16u, &bar_full[sg]);
      }
      if (lane == 0) {
        bulk_copy_g2s(base + 2 * size_t(a.plane), a.w_cm + size_t(cb) * (kBBytes / 2), kBBytes, &bar_full[sg]);
        s_issued = u + 1;
      }
      __syncwarp();
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = tc::idesc_bf16_f32(128, NOUT);
      const int row_z = a.by * a.bx;
      int st[kTileMaxMB];
#pragma unroll
      for (int j = 0; j < kTileMaxMB; ++j) st[j] = s_start[j];
      for (int u = 0; u < units && !s_fail; ++u) {
        const int sg = u % kWsStages, tl = u / ncb, cb = u % ncb, b = tl & 1;
        if (!tc::mbar_wait(&bar_full[sg], unsigned((u / kWsStages) & 1), kConvWaitNs)) {
          s_fail = 1;
          break;
        }
        s_consumed = u + 1;
        if (cb == 0 && tl >= 2 && !tc::mbar_wait(&bar_tempty[b], unsigned(((tl >> 1) - 1) & 1), kConvWaitNs)) {
          s_fail = 1;
          break;
        }
        tc::fence_after_sync();
        unsigned char* base = dsm + size_t(sg) * stage_bytes;
        const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(base), uint32_t(a.plane), 128);
        const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(base + 2 * size_t(a.plane)), 128, 256);
        const uint32_t dcol = tmem + uint32_t(b * acc_cols);
        int tap = 0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx, ++tap) {
              const int off = dz * row_z + dy * a.bx + dx;
              const uint64_t bdesc = bdesc0 + uint64_t(tap * (kBTap >> 4));
              const bool acc = (cb | tap) != 0;
#pragma unroll
              for (int j = 0; j < kTileMaxMB; ++j)
                if (j < a.mb) tc::mma_bf16(dcol + uint32_t(j * NOUT), adesc0 + uint64_t(st[j] + off), bdesc, idesc, acc);
            }
        tc::mma_commit(&bar_empty[sg]);
        if (cb == ncb - 1) tc::mma_commit(&bar_tfull[b]);
        s_mma = u + 1;
      }
    }
  } else {  // epilogue: warps 2-5, TMEM lane quarter q
    const int q = warp & 3, e = q * 32 + lane;
    const int bxby = a.bx * a.by;
    const size_t Vt = size_t(a.nx) * a.ny * a.nz;
    // the voxel of TMEM lane e in M-block j, relative to the tile origin
    // (the same for every tile), and the bias of the output channels
    int rel[kTileMaxMB];
#pragma unroll
    for (int j = 0; j < kTileMaxMB; ++j) {
      rel[j] = -1;
      if (j < a.mb) {
        const int row = s_start[j] + e;
        const int zq = row / bxby, rem = row - zq * bxby;
        const int yq = rem / a.bx, xq = rem - yq * a.bx;
        if (xq >= 1 && xq <= a.xc && yq >= 1 && yq <= a.ty && zq >= 1 && zq <= a.tz)
          rel[j] = ((zq - 1) * 256 + (yq - 1)) * 256 + (xq - 1);  // z, y, x offsets (each < 256)
      }
    }
    float bias[NOUT];
#pragma unroll
    for (int c = 0; c < NOUT; ++c) bias[c] = a.bias && c < a.cout ? a.bias[c] : 0.f;
    for (int tl = 0; tl < my_tiles; ++tl) {
      const int b = tl & 1;
      bool ok = !s_fail && tc::mbar_wait(&bar_tfull[b], unsigned((tl >> 1) & 1), kConvWaitNs);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) s_fail = 1;
        break;
      }
      tc::fence_after_sync();
      int x0, y0, z0;
      origin(tl, x0, y0, z0);
#pragma unroll
      for (int j = 0; j < kTileMaxMB; ++j) {
        if (j >= a.mb) break;
        const int r = rel[j];
        const int gx = x0 + (r & 255), gy = y0 + ((r >> 8) & 255), gz = z0 + (r >> 16);
        const bool valid = r >= 0 && gx < a.nx && gy < a.ny && gz < a.nz;
        const size_t v = (size_t(gz) * a.ny + gy) * a.nx + gx;
#pragma unroll
        for (int c0 = 0; c0 < NOUT; c0 += 16) {
          float acc[16];
          tc::tmem_ld16(tmem + (uint32_t(q * 32) << 16) + uint32_t(b * acc_cols + j * NOUT + c0), acc);
          if (valid && c0 < a.cout) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              const int cbase = c0 + 8 * half;
              if (cbase >= a.cout) break;
              __nv_bfloat16 o8[8];
#pragma unroll
              for (int k = 0; k < 8; ++k) o8[k] = __float2bfloat16(acc[8 * half + k] + bias[cbase + k]);
              __nv_bfloat16* dst = cbase < a.split ? a.dst0 + oct_index(v, cbase, a.split, Vt)
                                                   : a.dst1 + oct_index(v, cbase - a.split, a.cout - a.split, Vt);
              *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(o8);
            }
          }
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_tempty[b]);
    }
  }
  __syncthreads();
  if (s_fail && t == 0) {
    // copies issued but not awaited, and the MMAs issued last, finish before
    // the shared memory and TMEM are released
    for (int u = s_consumed; u < s_issued; ++u)
      tc::mbar_wait(&bar_full[u % kWsStages], unsigned((u / kWsStages) & 1), kConvWaitNs);
    if (s_mma > 0)
      tc::mbar_wait(&bar_empty[(s_mma - 1) % kWsStages], unsigned(((s_mma - 1) / kWsStages) & 1), kConvWaitNs);
    atomicExch(a.err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return encode;
}

// octet-plane BF16 tensor of C channels: dims {8, nx, ny, nz, C / 8}, box
// {8, bx, by, bz, 1} (one plane, contiguous x-runs of bx * 16 bytes)
bool encode_oct_map(CUtensorMap* m, const __nv_bfloat16* base, int C, int nx, int ny, int nz, int bx, int by, int bz) {
  auto encode = tensor_map_encoder();
  if (!encode || C % 8 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) || bx > 256 || by > 256 || bz > 256) return false;
  cuuint64_t dims[5] = {8, cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(nz), cuuint64_t(C / 8)};
  const cuuint64_t row = 16;  // bytes per voxel and plane
  // byte strides of dims 1..4 (x, y, z, plane); dim 0 (8 channels) is dense
  cuuint64_t strides[4] = {row, row * nx, row * nx * ny, row * nx * ny * nz};
  cuuint32_t box[5] = {8, cuuint32_t(bx), cuuint32_t(by), cuuint32_t(bz), 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Output box of the tiled kernel for an nx-wide grid: full x-lines of up to
// 128 voxels (line mode for 126..128) or consecutive 128-row blocks.
int plane_bytes(const ConvTileArgs& t, int ty, int tz) {
  const int rows = t.bx * (ty + 2) * (tz + 2);
  const int slack = t.line_mode ? 0 : 128 + t.bx * (ty + 2) + t.bx + 1;
  return ((rows + slack) * 16 + 127) / 128 * 128;
}

// tmem: TMEM columns the tile's accumulators may take (512, or 256 when
// the persistent kernel double-buffers them); smem_cap: bytes of all stages.
bool pick_tile(ConvTileArgs& t, int nout, int stages, int tmem = 512, size_t smem_cap = 200 * 1024) {
  t.xc = t.nx >= 128 ? 128 : t.nx;
  t.bx = t.xc + 2;
  t.line_mode = t.xc == 128 ? 1 : 0;
  const int max_mb = std::min(kTileMaxMB, tmem / nout);
  int best_ty = 1, best_tz = 1, best_mb = 0;
  double best_eff = -1.0;
  for (int tz = 1; tz <= 4; tz *= 2) {
    for (int ty = 1; ty <= 8; ty *= 2) {
      if (ty > t.ny || tz > t.nz) continue;
      int mb;
      if (t.line_mode) {
        mb = ty * tz;
      } else {
        const int by = ty + 2, first = (by + 1) * t.bx + 1, last = (tz * by + ty) * t.bx + t.xc;
        mb = (last - first + 1 + 127) / 128;
      }
      if (mb > max_mb) continue;
      const int rows = t.bx * (ty + 2) * (tz + 2);
      const size_t smem = size_t(stages) * (2 * size_t(plane_bytes(t, ty, tz)) + size_t(27) * nout * 32);
      if (smem > smem_cap) continue;
      // useful outputs per unit of (MMA rows + loaded rows)
      const double eff = double(t.xc * ty * tz) / double(mb * 128 * 27 + rows * 4);
      if (eff > best_eff + 1e-12) {
        best_eff = eff;
        best_ty = ty;
        best_tz = tz;
        best_mb = mb;
      }
    }
  }
  if (best_mb == 0) return false;
  t.ty = best_ty;
  t.tz = best_tz;
  t.by = t.ty + 2;
  t.bz = t.tz + 2;
  t.mb = best_mb;
  // plane: the box rows plus slack for M-blocks that run past the last row
  // (contiguous mode reads up to 127 rows + one z-slab beyond it)
  t.plane = plane_bytes(t, t.ty, t.tz);
  t.tiles_x = (t.nx + t.xc - 1) / t.xc;
  t.tiles_y = (t.ny + t.ty - 1) / t.ty;
  return true;
}

template <int NOUT>
cudaError_t launch_tile(const ConvArgs& a, cudaStream_t s, bool& taken) {
  taken = false;
  ConvTileArgs t{};
  t.nx = a.nx; t.ny = a.ny; t.nz = a.nz;
  t.c0 = a.c0; t.c1 = a.c1;
  const bool bulk = a.w_cm != nullptr && !(reinterpret_cast<uintptr_t>(a.w_cm) & 15);
  const bool ws = bulk && a.stages == 3;  // persistent warp-specialised kernel
  const int stages = bulk ? (a.stages == 2 ? 2 : 1) : 1;
  if (ws) {
    // two stages of 1024-aligned (planes + weights), two TMEM accumulators
    if (!pick_tile(t, NOUT, kWsStages, 256, size_t(kTileSmemMax) - 2 * 1024)) return cudaSuccess;
  } else if (!pick_tile(t, NOUT, stages)) {
    return cudaSuccess;
  }
  if (!encode_oct_map(&t.map0, a.src0, a.c0, a.nx, a.ny, a.nz, t.bx, t.by, t.bz)) return cudaSuccess;
  t.src0 = a.src0;
  t.src1 = a.src1;
  if (a.c1 > 0 && !encode_oct_map(&t.map1, a.src1, a.c1, a.nx, a.ny, a.nz, t.bx, t.by, t.bz)) return cudaSuccess;
  t.w = a.w;
  t.w_cm = bulk ? a.w_cm : nullptr;
  t.cin_pad = (a.c0 + a.c1 + 15) / 16 * 16;
  t.bias = a.bias;
  t.cout = a.cout;
  t.dst0 = a.dst0; t.dst1 = a.dst1; t.split = a.split;
  t.err = a.err;
  const unsigned grid_tiles = unsigned(t.tiles_x) * unsigned(t.tiles_y) * unsigned((t.nz + t.tz - 1) / t.tz);
  if (ws) {
    const unsigned stage_bytes = unsigned((2 * size_t(t.plane) + size_t(27) * NOUT * 32 + 1023) / 1024 * 1024);
    const size_t req = size_t(kWsStages) * stage_bytes;
    if (req > size_t(kTileSmemMax)) return cudaSuccess;
    static int ws_configured = 0;
    if (!ws_configured) {
      cudaError_t e =
          cudaFuncSetAttribute(conv3d_tile_ws_kernel<NOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmemMax);
      if (e != cudaSuccess) return e;
      ws_configured = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one CTA per SM (the shared memory of two stages), at most one per tile
    const unsigned grid = std::min(grid_tiles, unsigned(sms > 0 ? sms : 1));
    conv3d_tile_ws_kernel<NOUT><<<grid, kWsThreads, req, s>>>(t, int(grid_tiles), stage_bytes);
    taken = true;
    return cudaGetLastError();
  }
  const size_t smem = size_t(stages) * (2 * size_t(t.plane) + size_t(27) * NOUT * 32);
  // TMEM: at most 512 / cols CTAs may share an SM; pad the shared-memory
  // request so that no more than that many fit
  const int need = t.mb * NOUT;
  const int cols = need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : (need <= 256 ? 256 : 512)));
  const int max_ctas = 512 / cols;
  size_t req = smem;
  const size_t sm_total = 228 * 1024;
  if ((req + 1024) * size_t(max_ctas + 1) <= sm_total) req = sm_total / size_t(max_ctas + 1) - 1024 + 16;
  if (req > kTileSmemMax) return cudaSuccess;
  static int configured = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(conv3d_tile_kernel<NOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(conv3d_tile_pipe_kernel<NOUT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(conv3d_tile_pipe_kernel<NOUT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmemMax);
    if (e != cudaSuccess) return e;
    configured = 1;
  }
  const unsigned grid = grid_tiles;
  if (bulk && stages == 2)
    conv3d_tile_pipe_kernel<NOUT, 2><<<grid, kConvThreads, req, s>>>(t);
  else if (bulk)
    conv3d_tile_pipe_kernel<NOUT, 1><<<grid, kConvThreads, req, s>>>(t);
  else
    conv3d_tile_kernel<NOUT><<<grid, kConvThreads, req, s>>>(t);
  taken = true;
  return cudaGetLastError();
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Weight gradient of a stride-1 3x3x3 convolution on the tensor cores:
//   dW[t][co][ci] = sum over voxels v of g[v][co] in[v + s_t][ci],
// a contraction over K = voxels for each tap t (zero input outside the grid).
//
// A CTA stages an output box of g and the same box of the input, both with a
// one-voxel halo (TMA, zero fill outside the grid), as 8-channel planes:
// voxel row r = (z by + y) bx + x of the box holds 8 channels in 16 bytes, so
// 8 consecutive rows of one plane are an MN-major core matrix (8 K-rows of
// 8 MN-elements), the next 8 rows the next core matrix along K (128 bytes on)
// and the next plane the next core matrix along M or N (one plane on).  The
// 16 interior voxels of an x-line are the K = 16 block of one MMA; tap t
// reads the input rows shifted by its row offset (the descriptor start), as
// in the forward kernel.  M = 128 covers the operand with more channels
// (its unused M-groups read staged shared memory and are discarded), N the
// other channel count.  Each CTA accumulates its taps in TMEM over all its
// boxes and writes FP32 partial sums [chunk][tap][cout][cin] (and the bias
// gradient, the sum of g, from the staged boxes); a fixed-order reduction
// over the chunks follows, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
constexpr int kWgThreads = 128;
constexpr int kWgSlots = 16;               // planes staged: the A operand's 16 M-groups of 8 channels
constexpr int kWgXc = 16;                  // interior voxels per x-line of a box (one K block)
constexpr int kWgSmemMax = 208 * 1024;

struct WgradTcArgs {
  CUtensorMap map_g;   // g [V][cout] octet planes, box {8, bx, by, bz}
  CUtensorMap map0;    // input src0 (c0 channels)
  CUtensorMap map1;    // input src1 (c1 channels) or unused
  int c0, c1, cout;
  int bx, by, bz, ty, tz;
  int tiles_x, tiles_y, tiles;
  int plane;           // bytes between staged planes (128-multiple)
  int a_in;            // 1: A = input planes (M = cin), B = g planes (N = cout); 0: the other way
  int n_a, n_b;        // planes of A and B
  int taps_per_group;
  int chunks;
  float* partial;      // [chunks][27][cout][cin]
  float* bias_partial; // [chunks][cout]
  int* err;
};

template <int N>
__global__ void __launch_bounds__(kWgThreads) wgrad_tc_kernel(const __grid_constant__ WgradTcArgs a) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t bar_tma, bar_mma;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  __shared__ int s_off[27];      // row offset of each tap in the staged box
  __shared__ float s_bias[96];   // bias partial sums of warps 1..3
  const int t = threadIdx.x;
  const int chunk = blockIdx.x, group = blockIdx.y;
  const int tap0 = group * a.taps_per_group;
  const int ntap = min(a.taps_per_group, 27 - tap0);
  unsigned char* A = dsm;
  unsigned char* B = dsm + size_t(a.n_a) * a.plane;
  unsigned char* in_planes = a.a_in ? A : B;
  unsigned char* g_planes = a.a_in ? B : A;
  const int cin = a.c0 + a.c1;
  const unsigned box_bytes = unsigned(a.bx) * a.by * a.bz * 16;
  constexpr uint32_t kCols = 512;

  const int row_z = a.bx * a.by;
  if (t == 0) {
    tc::mbar_init(&bar_tma, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_fence_init();
    s_fail = 0;
  }
  if (t < 27) s_off[t] = (t / 9 - 1) * row_z + ((t / 3) % 3 - 1) * a.bx + (t % 3 - 1);
  if (t < 32) tc::tmem_alloc(&s_tmem, kCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  // kind::f16, D FP32, A and B BF16, both MN-major (transpose bits 15, 16)
  const uint32_t idesc = tc::idesc_bf16_f32(128, N) | (1u << 15) | (1u << 16);
  // bias gradient: thread 32 + j of warps 1..3 sums channel j % cout over the
  // rows r of each box with r % parts == j / cout (a fixed split)
  const int bj = t - 32, parts = 96 / a.cout;
  const bool bias_thread = group == 0 && bj >= 0 && bj < parts * a.cout;
  float bacc = 0.f;
  int nbox = 0;
  bool tma_pending = false;
  for (int box = chunk; box < a.tiles; box += a.chunks, ++nbox) {
    const int tx = box % a.tiles_x, tyi = (box / a.tiles_x) % a.tiles_y, tzi = box / (a.tiles_x * a.tiles_y);
    const int x0 = tx * kWgXc, y0 = tyi * a.ty, z0 = tzi * a.tz;
    if (nbox > 0 && !tc::mbar_wait(&bar_mma, unsigned((nbox - 1) & 1), kConvWaitNs)) s_fail = 1;
    __syncthreads();  // every thread is past the previous box (bias sums) and saw s_fail
    if (s_fail) break;
    if (t == 0) {
      tc::mbar_expect_tx(&bar_tma, unsigned(a.n_a + a.n_b) * box_bytes);
      const int p0 = a.c0 / 8;
      for (int p = 0; p < cin / 8; ++p)
        tc::tma_load_5d(in_planes + size_t(p) * a.plane, p < p0 ? static_cast<const void*>(&a.map0)
                                                                : static_cast<const void*>(&a.map1),
                        0, x0 - 1, y0 - 1, z0 - 1, p < p0 ? p : p - p0, &bar_tma);
      for (int p = 0; p < a.cout / 8; ++p)
        tc::tma_load_5d(g_planes + size_t(p) * a.plane, &a.map_g, 0, x0 - 1, y0 - 1, z0 - 1, p, &bar_tma);
    }
    tma_pending = true;
    if (!tc::mbar_wait(&bar_tma, unsigned(nbox & 1), kConvWaitNs)) {
      s_fail = 1;
      break;
    }
    tma_pending = false;
    tc::fence_after_sync();
    if (bias_thread) {
      // g summed over the interior voxels of the box (zero outside the grid),
      // beside the MMA issue of thread 0
      const int co = bj % a.cout, part = bj / a.cout;
      const unsigned char* gp = g_planes + size_t(co / 8) * a.plane + (co % 8) * 2;
      int i = 0;
      for (int zb = 1; zb <= a.tz; ++zb)
        for (int yb = 1; yb <= a.ty; ++yb) {
          const int r0 = (zb * a.by + yb) * a.bx + 1;
          for (int xb = 0; xb < kWgXc; ++xb, ++i)
            if (i % parts == part)
              bacc += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(gp + size_t(r0 + xb) * 16));
        }
    }
    if (t == 0) {
      // leading byte offset 128 (K: the next 8 voxel rows), stride byte offset
      // one plane (M / N: the next 8 channels); starts move by whole rows
      const uint64_t adesc0 = tc::smem_desc(tc::smem_addr(A), 128, uint32_t(a.plane));
      const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(B), 128, uint32_t(a.plane));
      for (int zb = 1; zb <= a.tz; ++zb) {
        for (int yb = 1; yb <= a.ty; ++yb) {
          const int r = (zb * a.by + yb) * a.bx + 1;  // first interior voxel of the x-line
          const bool acc = nbox > 0 || zb > 1 || yb > 1;
          for (int k = 0; k < ntap; ++k) {
            const int off = s_off[tap0 + k];
            const int ra = a.a_in ? r + off : r, rb = a.a_in ? r : r + off;
            tc::mma_bf16(tmem + uint32_t(k * N), adesc0 + uint64_t(ra), bdesc0 + uint64_t(rb), idesc, acc);
          }
        }
      }
      tc::mma_commit(&bar_mma);
    }
  }
  __syncthreads();
  if (!s_fail && nbox > 0 && !tc::mbar_wait(&bar_mma, unsigned((nbox - 1) & 1), kConvWaitNs)) s_fail = 1;
  __syncthreads();
  tc::fence_after_sync();
  if (s_fail) {
    if (t == 0) atomicExch(a.err, 1);
    if (tma_pending) tc::mbar_wait(&bar_tma, unsigned(nbox & 1), kConvWaitNs);  // let a copy in flight land
  } else {
    const int w = t / 32;
    const int mreal = a.a_in ? cin : a.cout;
    for (int k = 0; k < ntap; ++k) {
      const int tap = tap0 + k;
#pragma unroll
      for (int c = 0; c < N; c += 16) {
        float v[16];
        tc::tmem_ld16(tmem + (uint32_t(w * 32) << 16) + uint32_t(k * N + c), v);
        if (t < mreal) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int co = a.a_in ? c + j : t, ci = a.a_in ? t : c + j;
            a.partial[((size_t(chunk) * 27 + tap) * a.cout + co) * cin + ci] = nbox > 0 ? v[j] : 0.f;
          }
        }
      }
    }
    if (bias_thread) s_bias[bj] = bacc;
  }
  __syncthreads();
  if (!s_fail && group == 0 && t < a.cout) {
    float b = 0.f;
    for (int p = 0; p < parts; ++p) b += s_bias[p * a.cout + t];  // parts in a fixed order
    a.bias_partial[size_t(chunk) * a.cout + t] = b;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t < 32) tc::tmem_dealloc(tmem, kCols);
}

template <int N>
cudaError_t launch_wgrad_tc_n(const WgradTcArgs& a, unsigned groups, size_t smem, cudaStream_t s) {
  static int configured = 0;
  if (!configured) {
    const cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmemMax);
    if (e != cudaSuccess) return e;
    configured = 1;
  }
  wgrad_tc_kernel<N><<<dim3(unsigned(a.chunks), groups), kWgThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wgrad_tc(const __nv_bfloat16* src0, int c0, const __nv_bfloat16* src1, int c1,
                            const __nv_bfloat16* g, int cout, int nx, int ny, int nz, float* partial,
                            float* bias_partial, int max_chunks, int* chunks_out, int* err, cudaStream_t s) {
  const int cin = c0 + c1;
  if (c0 % 8 || c1 % 8 || cout % 8 || cin < 16 || cout < 16 || cin > 128 || cout > 128 || (c1 > 0 && !src1) ||
      max_chunks < 1)
    return cudaErrorNotSupported;
  WgradTcArgs a{};
  a.c0 = c0;
  a.c1 = c1;
  a.cout = cout;
  a.a_in = cin >= cout ? 1 : 0;
  const int n = a.a_in ? cout : cin;
  if (n != 16 && n != 32 && n != 64) return cudaErrorNotSupported;
  a.n_a = (a.a_in ? cin : cout) / 8;
  a.n_b = n / 8;
  if (a.n_a + a.n_b > kWgSlots) return cudaErrorNotSupported;
  // box: 16 interior columns, ty x tz interior lines; the 16 staged planes
  // must fit in shared memory; most interior voxels per staged voxel
  a.bx = kWgXc + 2;
  int best_ty = 1, best_tz = 1;
  double best = -1.0;
  for (int tz = 1; tz <= 8; ++tz)
    for (int ty = 1; ty <= 8; ++ty) {
      if (ty > ny || tz > nz) continue;
      const int rows = a.bx * (ty + 2) * (tz + 2);
      const size_t plane = size_t(rows * 16 + 127) / 128 * 128;
      if (plane * kWgSlots > size_t(kWgSmemMax)) continue;
      const double eff = double(ty * tz) / double((ty + 2) * (tz + 2));
      if (eff > best + 1e-12) {
        best = eff;
        best_ty = ty;
        best_tz = tz;
      }
    }
  if (best < 0) return cudaErrorNotSupported;
  a.ty = best_ty;
  a.tz = best_tz;
  a.by = a.ty + 2;
  a.bz = a.tz + 2;
  a.plane = (a.bx * a.by * a.bz * 16 + 127) / 128 * 128;
  a.tiles_x = (nx + kWgXc - 1) / kWgXc;
  a.tiles_y = (ny + a.ty - 1) / a.ty;
  a.tiles = a.tiles_x * a.tiles_y * ((nz + a.tz - 1) / a.tz);
  if (!encode_oct_map(&a.map_g, g, cout, nx, ny, nz, a.bx, a.by, a.bz)) return cudaErrorNotSupported;
  if (!encode_oct_map(&a.map0, src0, c0, nx, ny, nz, a.bx, a.by, a.bz)) return cudaErrorNotSupported;
  if (c1 > 0 && !encode_oct_map(&a.map1, src1, c1, nx, ny, nz, a.bx, a.by, a.bz)) return cudaErrorNotSupported;
  a.taps_per_group = std::min(27, 512 / n);
  const int groups = (27 + a.taps_per_group - 1) / a.taps_per_group;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  a.chunks = std::max(1, std::min({a.tiles, max_chunks, std::max(1, sms / groups)}));
  a.partial = partial;
  a.bias_partial = bias_partial;
  a.err = err;
  const size_t smem = size_t(a.plane) * kWgSlots;
  cudaError_t e;
  switch (n) {
    case 16: e = launch_wgrad_tc_n<16>(a, unsigned(groups), smem, s); break;
    case 32: e = launch_wgrad_tc_n<32>(a, unsigned(groups), smem, s); break;
    default: e = launch_wgrad_tc_n<64>(a, unsigned(groups), smem, s); break;
  }
  if (e == cudaSuccess && chunks_out) *chunks_out = a.chunks;
  return e;
}

bool conv3d_tile_eligible(const ConvArgs& a) {
  return a.ks == 3 && !a.packed && a.c0 % 16 == 0 && a.c1 % 16 == 0 && !a.dst_f32 && a.cout % 8 == 0 &&
         a.split % 8 == 0 && !(reinterpret_cast<uintptr_t>(a.w) & 15) && !(reinterpret_cast<uintptr_t>(a.dst0) & 15) &&
         !(a.dst1 && (reinterpret_cast<uintptr_t>(a.dst1) & 15));
}

cudaError_t launch_conv3d(const ConvArgs& a, int nout_pad, cudaStream_t s) {
  const size_t V = size_t(a.nx) * a.ny * a.nz;
  if (conv3d_tile_eligible(a) && !a.no_tile) {
    bool taken = false;
    cudaError_t e = cudaSuccess;
    switch (nout_pad) {
      case 16: e = launch_tile<16>(a, s, taken); break;
      case 32: e = launch_tile<32>(a, s, taken); break;
      case 64: e = launch_tile<64>(a, s, taken); break;
      default: break;
    }
    if (e != cudaSuccess || taken) return e;
  }
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
