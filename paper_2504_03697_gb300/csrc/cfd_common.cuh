// Shared device-side definitions of the cavity projection path (sm_103a).
//
// Staggered (MAC) grid, Sec. 3.1 of arXiv 2504.03697: velocity components on
// cell faces, pressure at cell centres.  Arrays are x-fastest.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cfd {

constexpr int kMaxPartials = 8;  // scalars one grid reduction can carry

// Control block of one persistent solve: grid-barrier counters and the
// reduced scalars published by the last block to arrive.
struct __align__(64) SolveCtrl {
  unsigned int arrive;
  unsigned int gen;
  int error;            // CFD_ERR_* of a device-side failure, 0 if none
  int pad0;
  double red[kMaxPartials];
};

// Per-solve statistics written by the device (mirrors cfd_solve_stats).
struct DevSolveStats {
  int iters;
  int outer_iters;
  int restarts;
  int status;
  double rel_resid;
  double b_norm;
};

// Per-step statistics slot (pressure + three diffusion solves).
struct DevStepStats {
  DevSolveStats p;
  DevSolveStats d[3];
};

// Status codes shared with include/cfd.h
constexpr int kOk = 0;
constexpr int kErrNotConverged = -3;
constexpr int kErrBreakdown = -4;
constexpr int kErrTimeout = -5;

__host__ __device__ inline size_t idx3(int i, int j, int k, int mx, int my) {
  return (size_t(k) * my + j) * mx + i;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_s32(const int* p) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------------------
// Deterministic block reduction of NV doubles (fixed shuffle tree, then warp
// totals summed in warp order).  Result valid in thread 0.  `scratch` holds
// at least 32 * NV doubles.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) scratch[warp * NV + a] = v[a];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double s = scratch[a];
      for (int w = 1; w < nwarps; ++w) s += scratch[w * NV + a];
      v[a] = s;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Grid-wide reduction + barrier for a cooperatively launched (all blocks
// co-resident) persistent kernel.
//
// Every block contributes NV partial sums; the last block to arrive sums the
// per-block partials in block order (deterministic, independent of arrival
// order), publishes the totals in ctrl->red and releases the others.  Every
// wait is bounded: after `timeout_ns` a waiter records CFD_ERR_TIMEOUT in
// ctrl->error and all blocks return false; they also return false as soon as
// any block has recorded an error.  On success the totals are in out[].
// ---------------------------------------------------------------------------
template <int NV>
__device__ bool grid_allreduce(double (&v)[NV], double (&out)[NV], SolveCtrl* ctrl, double* partials,
                               double* scratch, unsigned long long timeout_ns) {
  __shared__ int s_flag;
  __shared__ unsigned int s_gen;
  block_reduce<NV>(v, scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) partials[size_t(blockIdx.x) * kMaxPartials + a] = v[a];
    s_gen = ld_volatile_u32(&ctrl->gen);
    __threadfence();
    unsigned int ticket = atomicAdd(&ctrl->arrive, 1u);
    s_flag = (ticket == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (s_flag) {
    // last block: fixed-order sum of all block partials
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) acc[a] = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
      for (int a = 0; a < NV; ++a) acc[a] += __ldcg(&partials[size_t(b) * kMaxPartials + a]);
    }
    block_reduce<NV>(acc, scratch);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) ctrl->red[a] = acc[a];
      ctrl->arrive = 0u;
      __threadfence();
      atomicAdd(&ctrl->gen, 1u);
    }
  } else if (threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    int ok = 1;
    unsigned int ns = 32;
    while (ld_volatile_u32(&ctrl->gen) == s_gen) {
      if (ld_volatile_s32(&ctrl->error) != 0) { ok = 0; break; }
      if (global_ns() - t0 > timeout_ns) {
        atomicCAS(&ctrl->error, 0, kErrTimeout);
        ok = 0;
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns <<= 1;
    }
    s_flag = ok ? 2 : 3;
  }
  __syncthreads();
  if (s_flag == 3) return false;
  __threadfence();
#pragma unroll
  for (int a = 0; a < NV; ++a) out[a] = __ldcg(&ctrl->red[a]);
  __syncthreads();  // s_flag is rewritten by the next call
  return true;
}

}  // namespace cfd
