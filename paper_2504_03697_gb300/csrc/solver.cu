// Host side of the persistent conjugate-gradient solves (sm_103a): launch
// shapes, occupancy, cooperative launches, TMA tensor maps.  The kernels
// live in solver_impl.cuh and are instantiated by solver_k_*.cu; the
// method and its row evaluation are described there.

#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>

#include "solver_impl.cuh"
#include "solver_kernels.h"

namespace cfd {

namespace {

int tiles_of(GridDims g, int tz) { return make_tiles(g.mx, g.my, g.mz, tz).count(); }

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

CgKernel cg_kernel_for(int precond, int rtz, bool multi = false) {
  if (multi) return cg_kernel_multi(precond);
  return precond ? cg_kernel_jacobi(rtz) : cg_kernel_plain(rtz);
}

Cg1Kernel cg1_kernel_for(int rtz) { return cg1_kernel(rtz); }

bool cg1_allowed(const CgArgs& a) { return a.variant == 0 && a.precond == 0 && a.e0 && a.e1 && a.e2; }

}  // namespace

// Co-resident blocks per SM of one kernel variant (both preconditioner
// instantiations), capped at 4.
int variant_blocks_per_sm(int rtz) {
  int per_sm = 1 << 30;
  for (int p = 0; p < 2; ++p) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cg_kernel_for(p, rtz), kSolveThreads, 0);
    per_sm = b < per_sm ? b : per_sm;
  }
  return per_sm > 4 ? 4 : per_sm;
}

// Co-resident blocks per SM of the single-reduction variant.
int cg1_blocks_per_sm(int rtz) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cg1_kernel_for(rtz), kSolveThreads, 0);
  return b > 4 ? 4 : b;
}

int cg_max_coresident_blocks(int kind_is_ir) {
  int best = 0;
  for (int rtz : {0, 1, 2, 4, 8}) {
    const int b = variant_blocks_per_sm(rtz);
    best = b > best ? b : best;
  }
  if (kind_is_ir) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ir_kernel_single(), kSolveThreads, 0);
    b = b > 8 ? 8 : b;
    best = b > best ? b : best;
  }
  return best * num_sms();
}

// Launch shape of one solve: blocks per SM and tile depth.  Requested values
// (> 0) are honoured (clamped to what the kernel variant can keep
// co-resident); otherwise the register path is preferred with the fewest
// blocks that fits it (fewest all-reduce participants), and the memory path
// falls back to the deepest tile that still gives every SM two tiles, with
// as many blocks per SM as fit (latency hiding).
SolveShape pick_solve_shape(GridDims g, int max_blocks, int bps_req, int tz_req) {
  const int sms = num_sms();
  auto consider = [&](int bps, int tz, bool allow_reg) {
    const int tiles = tiles_of(g, tz);
    const int reg_cap = variant_blocks_per_sm(tz) * sms;
    const int mem_cap = variant_blocks_per_sm(0) * sms;
    int blocks = bps * sms;
    blocks = blocks < max_blocks ? blocks : max_blocks;
    int b_reg = blocks < reg_cap ? blocks : reg_cap;
    b_reg = b_reg < tiles ? b_reg : tiles;
    b_reg = b_reg > 0 ? b_reg : 1;
    const int tpb = (tiles + b_reg - 1) / b_reg;
    if (allow_reg && tpb * tz <= kRegCells) return SolveShape{b_reg, tz, tz};
    int b_mem = blocks < mem_cap ? blocks : mem_cap;
    b_mem = b_mem > 0 ? b_mem : 1;
    return SolveShape{b_mem, tz, 0};
  };
  if (bps_req > 0 || tz_req > 0) {
    const int bps = bps_req > 0 ? bps_req : 1;
    int tz = tz_req > 0 ? tz_req : 2;
    tz = tz < 2 ? 1 : (tz < 4 ? 2 : (tz < 8 ? 4 : 8));
    return consider(bps, tz, true);
  }
  for (int bps = 1; bps <= 4; bps <<= 1) {
    for (int tz = kMaxTz; tz >= 1; tz >>= 1) {
      const SolveShape s = consider(bps, tz, true);
      if (s.rtz > 0) return s;
    }
  }
  for (int tz = kMaxTz; tz > 1; tz >>= 1)
    if (tiles_of(g, tz) >= 2 * sms) return consider(4, tz, false);
  return consider(4, 1, false);
}

// The tile-resident single-reduction kernel serves the automatic shape when
// its tiles fill more than half of the SMs and fit one per SM: below that
// the smaller tiles of the register path spread the FP64 work over more SMs.
// Its blocks take a whole SM's registers each, so it runs only on a device
// that no other cooperative grid shares.
int cgt_blocks_for(GridDims g, const LaunchGeom& lg) {
  if (lg.bps_req > 0 || lg.tz_req > 0 || lg.shared) return 0;
  static int per_sm = -1;
  if (per_sm < 0) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cgt_kernel(), cgt_threads(), 0);
    per_sm = b;
  }
  const int sms = num_sms();
  const int tiles = cgt_tiles(g);
  if (g.count() >= (size_t(1) << 20) - 1) return 0;  // halo indices are packed in 20 bits
  if (per_sm < 1 || tiles > sms || tiles > lg.blocks || 2 * tiles <= sms) return 0;
  return tiles;
}

cudaError_t launch_cg(const CgArgs& a_in, const LaunchGeom& lg, cudaStream_t s, int64_t* launches) {
  CgArgs a = a_in;
  if (const int tiles = cg1_allowed(a) ? cgt_blocks_for(a.g, lg) : 0) {
    a.tz = kCgtTileDepth;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tiles);
    cfg.blockDim = dim3(cgt_threads());
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t err = cudaLaunchKernelEx(&cfg, cgt_kernel(), a);
    if (launches) *launches += 1;
    return err;
  }
  SolveShape sh = pick_solve_shape(a.g, lg.blocks, lg.bps_req, lg.tz_req);
  a.tz = sh.tz;
  // the single-reduction kernel must keep the whole grid co-resident too: the
  // memory path shrinks the grid to its capacity, the register path (whose
  // tiles per block are fixed by the grid size) falls back to the textbook
  // kernel instead
  bool single = cg1_allowed(a);
  if (single) {
    const int cap = cg1_blocks_per_sm(sh.rtz) * num_sms();
    if (sh.blocks > cap) {
      if (sh.rtz > 0) single = false;
      else sh.blocks = cap;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sh.blocks);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t err = single ? cudaLaunchKernelEx(&cfg, cg1_kernel_for(sh.rtz), a)
                                    : cudaLaunchKernelEx(&cfg, cg_kernel_for(a.precond, sh.rtz), a,
                                                         (const CgArgs*)nullptr, (const int*)nullptr, 0);
  if (launches) *launches += 1;
  return err;
}

int batch_blocks_per_sm() {
  int b = 0, b0 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cg_kernel_for(1, 0, true), kSolveThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, cg_kernel_for(0, 0, true), kSolveThreads, 0);
  b = b0 < b ? b0 : b;
  return b > 4 ? 4 : b;
}

int batch_num_sms() { return num_sms(); }

static cudaError_t launch_coop(void (*kern)(const CgArgs, const CgArgs*, const int*, int), const CgArgs* t,
                               const int* starts, int nprob, int blocks, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, CgArgs{}, t, starts, nprob);
}

cudaError_t launch_cg_multi(const CgArgs* d_table, const int* d_starts, int nprob, int total_blocks, int precond,
                            cudaStream_t s, int64_t* launches) {
  if (launches) *launches += 1;
  return launch_coop(cg_kernel_for(precond, 0, true), d_table, d_starts, nprob, total_blocks, s);
}

int solve_tile_depth_for(GridDims g, int blocks) {
  for (int tz = kMaxTz; tz > 1; tz >>= 1)
    if (tiles_of(g, tz) >= 2 * blocks) return tz;
  return 1;
}

cudaError_t launch_apply_poisson(GridDims g, const double* x, double* y, int tz, cudaStream_t s,
                                 int64_t* launches) {
  if (tz < 1 || tz > kMaxTz) tz = 4;
  const int tiles = tiles_of(g, tz);
  apply_poisson_kernel<<<tiles, kSolveThreads, 0, s>>>(g, x, y, tz);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

bool encode_f32_grid_map(CUtensorMap* map, const float* base, int mx, int my, int mz) {
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
  // TMA: row stride a multiple of 16 bytes, 16-byte aligned base; the box is
  // only used on grids at least as large as it
  if (!encode || mx % 4 != 0 || mx < kTmaBoxW || my < kTmaBoxH || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  cuuint64_t dims[3] = {cuuint64_t(mx), cuuint64_t(my), cuuint64_t(mz)};
  cuuint64_t strides[2] = {cuuint64_t(mx) * 4, cuuint64_t(mx) * cuuint64_t(my) * 4};
  cuuint32_t box[3] = {cuuint32_t(kTmaBoxW), cuuint32_t(kTmaBoxH), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_ir(const IrArgs& a_in, const LaunchGeom& lg, cudaStream_t s, int64_t* launches) {
  IrArgs a = a_in;
  const int sms = num_sms();
  a.use_tma = 0;
  if (a.kind == kOpPressure && !lg.no_tma && encode_f32_grid_map(&a.map_r32, a.r32, a.g.mx, a.g.my, a.g.mz) &&
      encode_f32_grid_map(&a.map_p0, a.p0_32, a.g.mx, a.g.my, a.g.mz) &&
      encode_f32_grid_map(&a.map_p1, a.p1_32, a.g.mx, a.g.my, a.g.mz)) {
    a.use_tma = 1;
    const int cols = ((a.g.mx + kTileX - 1) / kTileX) * ((a.g.my + kTileY - 1) / kTileY);
    a.tma_zl = 8;
    for (int zl = 64; zl >= 8; zl >>= 1)
      if (cols * ((a.g.mz + zl - 1) / zl) >= 4 * sms) {
        a.tma_zl = zl;
        break;
      }
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ir_kernel_single(), kSolveThreads, 0);
  per_sm = per_sm > 8 ? 8 : (per_sm < 1 ? 1 : per_sm);
  int bps = lg.bps_req > 0 ? (lg.bps_req < per_sm ? lg.bps_req : per_sm) : (per_sm < 4 ? per_sm : 4);
  int tz = lg.tz_req;
  if (tz <= 0) {
    tz = 1;
    for (int t = kMaxTz; t > 1; t >>= 1)
      if (tiles_of(a.g, t) >= 2 * sms) { tz = t; break; }
  }
  tz = tz < 2 ? 1 : (tz < 4 ? 2 : (tz < 8 ? 4 : 8));
  a.tz = tz;
  int blocks = bps * sms;
  if (blocks > lg.blocks) blocks = lg.blocks;
  const int tiles = tiles_of(a.g, tz);
  const int flat = int((a.g.count() + kSolveThreads - 1) / kSolveThreads);
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
  cudaError_t err = cudaLaunchKernelEx(&cfg, ir_kernel_single(), a, (const IrArgs*)nullptr, (const int*)nullptr, 0);
  if (launches) *launches += 1;
  return err;
}

}  // namespace cfd
