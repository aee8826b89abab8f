// Shared device-side definitions of the cavity projection path (sm_103a).
//
// Staggered (MAC) grid, Sec. 3.1 of arXiv 2504.03697: velocity components on
// cell faces, pressure at cell centres.  Arrays are x-fastest.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cfd {

constexpr int kMaxPartials = 8;   // scalars one grid reduction can carry
constexpr int kFlatMaxBlocks = 1024;  // up to this grid size every block reads every partial
constexpr int kGroupSize = 32;      // blocks per group of the two-level all-reduce
constexpr int kMaxGroups = 128;     // groups (so at most 4096 blocks)

// Control block of one persistent solve (zeroed by the host before each
// launch): the grid all-reduce counters and the error flag.
struct __align__(64) SolveCtrl {
  unsigned int arrive;  // monotonic arrival counter (flat) / group-sum counter (two-level)
  int error;            // CFD_ERR_* of a device-side failure, 0 if none
  int pad[14];
  unsigned int group[kMaxGroups];  // monotonic per-group arrival counters (two-level)
};

// Doubles of the partial-sum scratch a grid of `blocks` blocks needs:
// double-buffered block partials, then double-buffered group partials.
__host__ __device__ constexpr size_t partials_doubles(int blocks) {
  return 2 * size_t(blocks) * kMaxPartials + 2 * size_t(kMaxGroups) * kMaxPartials;
}

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

__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Bounded wait (thread 0) until the monotonic counter reaches target.
// Returns false, recording CFD_ERR_TIMEOUT, once timeout_ns have passed
// (checked on the first unsatisfied poll and every 64 polls after it, so a
// limit of 0 gives up at once), and also when another block has recorded an
// error.
__device__ __forceinline__ bool wait_counter(SolveCtrl* ctrl, const unsigned int* counter, unsigned int target,
                                             unsigned long long timeout_ns) {
  const unsigned long long t0 = global_ns();
  unsigned int polls = 0;
  while (int(ld_acquire_gpu(counter) - target) < 0) {
    if ((polls++ & 63u) == 0) {
      if (ld_volatile_s32(&ctrl->error) != 0) return false;
      if (global_ns() - t0 >= timeout_ns) {
        atomicCAS(&ctrl->error, 0, kErrTimeout);
        return false;
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Grid-wide all-reduce + barrier for a cooperatively launched persistent
// kernel (all blocks co-resident).  Every block obtains bitwise the same
// totals, independent of arrival order: all sums run in a fixed order with
// a fixed thread/tree shape.
//
// Flat form (grid <= kFlatMaxBlocks): each block stores its NV partials in a
// double-buffered array (buffer round & 1), arrives on a monotonic counter
// with a release reduction, waits until the counter reaches
// (round + 1) * grid, then sums all block partials itself.
//
// Two-level form (larger grids): blocks arrive on their group's counter
// (groups of kGroupSize consecutive blocks) with an acq_rel atomic; the last
// arriver of a group sums the group's partials in block order, stores the
// group partial and arrives on the top counter; every block waits for all
// groups and sums the group partials in group order.  This keeps the reads
// per all-reduce linear in the grid size.
//
// Double buffering is enough: a buffer is written again two rounds later,
// after a barrier that every block reaches only once it has read this round.
// Memory ordering: partial stores precede a release (red.release or the
// release half of atom.acq_rel) on the counter they arrive at; readers
// acquire that counter in thread 0, bar.sync carries it to the block, and
// partials are read through L2 (ld.global.cg).
//
// Every wait is bounded (wait_counter).  `round` is the caller's per-block
// count of completed all-reduces (identical in every block).
// ---------------------------------------------------------------------------
// The blocks of one problem inside a (possibly multi-problem) launch: this
// block's index among them and their count.  Independent problems of one
// launch never synchronise with each other.
struct VBlock {
  int bid;
  int nb;
};

template <int NV>
__device__ bool grid_allreduce(double (&v)[NV], double (&out)[NV], SolveCtrl* ctrl, double* partials,
                               double* scratch, unsigned long long timeout_ns, unsigned int& round, VBlock vb) {
  __shared__ int s_ok;
  __shared__ int s_last;
  __shared__ double s_bcast[kMaxPartials];
  block_reduce<NV>(v, scratch);
  const unsigned int G = unsigned(vb.nb);
  const unsigned int r = round++;
  double* buf = partials + size_t(r & 1u) * G * kMaxPartials;
  double acc[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) acc[a] = 0.0;

  if (G <= unsigned(kFlatMaxBlocks)) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) buf[size_t(vb.bid) * kMaxPartials + a] = v[a];
      red_add_release_gpu(&ctrl->arrive, 1u);
      s_ok = wait_counter(ctrl, &ctrl->arrive, (r + 1u) * G, timeout_ns) ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) return false;
    // warp 0 sums the block partials (each lane a fixed strided subset, then
    // a fixed shuffle tree) and broadcasts: one block barrier instead of the
    // two of a block-wide reduction
    if (threadIdx.x < 32) {
      for (unsigned int b = threadIdx.x; b < G; b += 32) {
#pragma unroll
        for (int a = 0; a < NV; ++a) acc[a] += __ldcg(&buf[size_t(b) * kMaxPartials + a]);
      }
#pragma unroll
      for (int a = 0; a < NV; ++a) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[a] += __shfl_down_sync(0xffffffffu, acc[a], off);
      }
      if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < NV; ++a) s_bcast[a] = acc[a];
      }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < NV; ++a) out[a] = s_bcast[a];
    return true;
  } else {
    const unsigned int ngroups = (G + kGroupSize - 1) / kGroupSize;
    const unsigned int g = unsigned(vb.bid) / kGroupSize;
    const unsigned int g0 = g * kGroupSize;
    const unsigned int gsize = (G - g0) < unsigned(kGroupSize) ? (G - g0) : unsigned(kGroupSize);
    double* gbuf = partials + 2 * size_t(G) * kMaxPartials + size_t(r & 1u) * kMaxGroups * kMaxPartials;
    if (threadIdx.x == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) buf[size_t(vb.bid) * kMaxPartials + a] = v[a];
      const unsigned int old = atom_add_acq_rel_gpu(&ctrl->group[g], 1u);
      s_last = (old == (r + 1u) * gsize - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
      // last of its group: sum the group's block partials in block order
      double gacc[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) gacc[a] = 0.0;
      if (threadIdx.x < gsize) {
#pragma unroll
        for (int a = 0; a < NV; ++a) gacc[a] = __ldcg(&buf[size_t(g0 + threadIdx.x) * kMaxPartials + a]);
      }
      block_reduce<NV>(gacc, scratch);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < NV; ++a) gbuf[size_t(g) * kMaxPartials + a] = gacc[a];
        red_add_release_gpu(&ctrl->arrive, 1u);
      }
    }
    if (threadIdx.x == 0) s_ok = wait_counter(ctrl, &ctrl->arrive, (r + 1u) * ngroups, timeout_ns) ? 1 : 0;
    __syncthreads();
    if (!s_ok) return false;
    for (unsigned int q = threadIdx.x; q < ngroups; q += blockDim.x) {
#pragma unroll
      for (int a = 0; a < NV; ++a) acc[a] += __ldcg(&gbuf[size_t(q) * kMaxPartials + a]);
    }
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
