// Shared device-side definitions of the cavity projection path (sm_103a).
//
// Staggered (MAC) grid, Sec. 3.1 of arXiv 2504.03697: velocity components on
// cell faces, pressure at cell centres.  Arrays are x-fastest.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cfd {

constexpr int kMaxPartials = 8;  // scalars one grid reduction can carry

// Control block of one persistent solve (zeroed by the host before each
// launch): the grid all-reduce counter and the error flag.
struct __align__(64) SolveCtrl {
  unsigned int arrive;  // monotonic arrival counter of the grid all-reduce
  int error;            // CFD_ERR_* of a device-side failure, 0 if none
  int pad[14];
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

__device__ __forceinline__ void red_add_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------------------
// Grid-wide all-reduce + barrier for a cooperatively launched persistent
// kernel (all blocks co-resident).
//
// Each block publishes NV partial sums in a double-buffered array (buffer
// round & 1) and arrives on a monotonically increasing counter with a
// release reduction.  Once the counter reaches (round + 1) * gridDim.x,
// every block sums all block partials itself, in block order with the same
// thread/tree shape, so every block obtains bitwise the same totals and the
// result does not depend on arrival order.  Double buffering is enough: a
// block can only overwrite buffer (round & 1) again after the next round's
// barrier, which every block reaches only after finishing this round's sum.
//
// Memory ordering: partial stores, then red.release on the counter; the
// waiting thread 0 acquires the counter; bar.sync carries that to the other
// threads, which read the partials through L2 (ld.global.cg).
//
// Every wait is bounded: after timeout_ns the waiter records
// CFD_ERR_TIMEOUT in ctrl->error and returns false; any block that sees a
// recorded error also returns false.  `round` is the caller's per-block
// count of completed all-reduces (identical in every block).
// ---------------------------------------------------------------------------
template <int NV>
__device__ bool grid_allreduce(double (&v)[NV], double (&out)[NV], SolveCtrl* ctrl, double* partials,
                               double* scratch, unsigned long long timeout_ns, unsigned int& round) {
  __shared__ int s_ok;
  __shared__ double s_bcast[kMaxPartials];
  block_reduce<NV>(v, scratch);
  double* buf = partials + size_t(round & 1u) * gridDim.x * kMaxPartials;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) buf[size_t(blockIdx.x) * kMaxPartials + a] = v[a];
    red_add_release_gpu(&ctrl->arrive, 1u);
    const unsigned int target = (round + 1u) * gridDim.x;
    const unsigned long long t0 = global_ns();
    int ok = 1;
    unsigned int polls = 0;
    while (int(ld_acquire_gpu(&ctrl->arrive) - target) < 0) {
      if ((++polls & 63u) == 0) {
        if (ld_volatile_s32(&ctrl->error) != 0) { ok = 0; break; }
        if (global_ns() - t0 > timeout_ns) {
          atomicCAS(&ctrl->error, 0, kErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  ++round;
  __syncthreads();
  if (!s_ok) return false;
  double acc[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) acc[a] = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int a = 0; a < NV; ++a) acc[a] += __ldcg(&buf[size_t(b) * kMaxPartials + a]);
  }
  block_reduce<NV>(acc, scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) s_bcast[a] = acc[a];
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < NV; ++a) out[a] = s_bcast[a];
  return true;
}

}  // namespace cfd
