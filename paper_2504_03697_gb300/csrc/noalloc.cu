// Allocation-free variant of the standalone pressure solve.
//
// Some callers cannot allocate device memory at all: code running inside a
// host callback or an interrupt-like context, plug-ins whose host application
// owns the allocator and forbids outside allocations, or embedded runtimes
// that reserve all device memory up front.  cfd_poisson_solve_noalloc serves
// them: it runs the same persistent CG kernel as cfd_solve_pressure, but its
// scratch vectors live in one file-scope __device__ array of fixed size
// instead of a caller-provided workspace, and it calls no allocating routine
// (no cudaMalloc / cudaFree, no torch, no library that allocates).
//
// Limits and sharing rules (also stated in include/cfd.h):
//  * at most CFD_NOALLOC_MAX_CELLS cells; larger grids are rejected with
//    CFD_ERR_INVALID_ARG;
//  * every GPU that loads this library holds the array (about 11 MB) until
//    the process exits;
//  * all calls share the one array per device, so calls whose GPU work
//    overlaps (different streams, or different host threads on one device)
//    race; serialise them on one stream;
//  * the first call on a device looks up the array's device address (once
//    per device, with that device current); make that first call before any
//    stream capture.

#include <mutex>

#include "../../include/cfd.h"
#include "cfd_internal.h"

namespace cfd {
namespace {

constexpr size_t kNoallocCells = CFD_NOALLOC_MAX_CELLS;
constexpr int kNoallocMaxBlocks = 4096;
constexpr size_t kVecBytes = kNoallocCells * sizeof(double);
// b copy, r, d0, d1, q | partials | ctrl | stats
constexpr size_t kOffB = 0;
constexpr size_t kOffR = kOffB + kVecBytes;
constexpr size_t kOffD0 = kOffR + kVecBytes;
constexpr size_t kOffD1 = kOffD0 + kVecBytes;
constexpr size_t kOffQ = kOffD1 + kVecBytes;
constexpr size_t kOffPartials = kOffQ + kVecBytes;
constexpr size_t kOffCtrl = kOffPartials + partials_doubles(kNoallocMaxBlocks) * sizeof(double);
constexpr size_t kCtrlBytes = 1024;
static_assert(sizeof(SolveCtrl) <= kCtrlBytes, "control block does not fit");
constexpr size_t kOffStats = kOffCtrl + kCtrlBytes;
constexpr size_t kNoallocBytes = kOffStats + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
struct DeviceScratch {
  std::once_flag once;
  cudaError_t err = cudaSuccess;
  unsigned char* ptr = nullptr;  // device address of g_noalloc_scratch on that device
  int blocks = 0;                // co-resident blocks of the solve kernel
};
DeviceScratch g_dev[kMaxDevices];

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" int cfd_poisson_solve_noalloc(int32_t nx, int32_t ny, int32_t nz, const double* b_dev, double* x_dev,
                                         double rtol, int32_t max_iters, cfd_stream_t stream,
                                         cfd_solve_stats* stats) {
  if (nx < 1 || ny < 1 || nz < 1) return cfd_internal_error(CFD_ERR_INVALID_ARG, "noalloc: grid sizes must be >= 1");
  const size_t cells = size_t(nx) * size_t(ny) * size_t(nz);
  if (cells > kNoallocCells)
    return cfd_internal_error(CFD_ERR_INVALID_ARG,
                              "noalloc: %zu cells exceed the fixed scratch limit CFD_NOALLOC_MAX_CELLS = %zu",
                              cells, kNoallocCells);
  if (!b_dev || !x_dev) return cfd_internal_error(CFD_ERR_INVALID_ARG, "noalloc: b or x is NULL");
  if (!(rtol > 0) || rtol >= 1) return cfd_internal_error(CFD_ERR_INVALID_ARG, "noalloc: rtol must be in (0, 1)");
  if (max_iters < 0) return cfd_internal_error(CFD_ERR_INVALID_ARG, "noalloc: max_iters must be >= 0");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cfd_internal_error(CFD_ERR_CUDA, "noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return cfd_internal_error(CFD_ERR_INVALID_ARG, "noalloc: device ordinal %d too large", dev);
  DeviceScratch& ds = g_dev[dev];
  // once per device, with that device current: host code may not use the
  // array's name as an address, so look the device address up here
  std::call_once(ds.once, [&]() {
    void* p = nullptr;
    ds.err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    ds.ptr = static_cast<unsigned char*>(p);
    if (ds.err == cudaSuccess) ds.blocks = cg_max_coresident_blocks(0);
  });
  if (ds.err != cudaSuccess || !ds.ptr)
    return cfd_internal_error(CFD_ERR_CUDA, "noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(ds.err));
  if (ds.blocks < 1) return cfd_internal_error(CFD_ERR_CUDA, "noalloc: the solve kernel cannot be placed on device %d", dev);
  if (ds.blocks > kNoallocMaxBlocks) ds.blocks = kNoallocMaxBlocks;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* base = ds.ptr;
  double* b = reinterpret_cast<double*>(base + kOffB);
  SolveCtrl* ctrl = reinterpret_cast<SolveCtrl*>(base + kOffCtrl);
  DevSolveStats* dstats = reinterpret_cast<DevSolveStats*>(base + kOffStats);

  // the array keeps the previous call's contents: the copy of b overwrites
  // its part, the control block and statistics must start at zero
  e = cudaMemcpyAsync(b, b_dev, cells * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctrl, 0, kCtrlBytes + 256, s);
  if (e != cudaSuccess) return cfd_internal_error(CFD_ERR_CUDA, "noalloc: %s", cudaGetErrorString(e));

  CgArgs a{};
  a.g = GridDims{nx, ny, nz};
  a.kind = kOpPressure;
  a.precond = 0;
  a.c = 0.0;
  a.x = x_dev;
  a.b = b;
  a.r = reinterpret_cast<double*>(base + kOffR);
  a.d0 = reinterpret_cast<double*>(base + kOffD0);
  a.d1 = reinterpret_cast<double*>(base + kOffD1);
  a.q = reinterpret_cast<double*>(base + kOffQ);
  a.zero_x0 = 1;
  a.remove_mean = 1;
  a.gauge = 0;
  a.gauge_value = 0.0;
  a.rtol = rtol;
  int cap = max_iters;
  if (cap == 0) {
    int m = nx > ny ? nx : ny;
    m = m > nz ? m : nz;
    cap = 20 * m;
  }
  a.max_iters = cap;
  a.max_restarts = 8;
  a.timeout_ns = 2000000000ull;
  a.ctrl = ctrl;
  a.partials = reinterpret_cast<double*>(base + kOffPartials);
  a.stats = dstats;
  a.tz = solve_tile_depth(nz);
  LaunchGeom lg{};
  lg.blocks = ds.blocks;
  e = launch_cg(a, lg, s, nullptr);
  if (e != cudaSuccess) return cfd_internal_error(CFD_ERR_CUDA, "noalloc: launch: %s", cudaGetErrorString(e));
  if (!stats) return CFD_OK;

  DevSolveStats host{};
  SolveCtrl hctrl{};
  e = cudaMemcpyAsync(&host, dstats, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hctrl, ctrl, sizeof(hctrl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cfd_internal_error(CFD_ERR_CUDA, "noalloc: %s", cudaGetErrorString(e));
  *stats = cfd_solve_stats{};
  stats->iters = host.iters;
  stats->restarts = host.restarts;
  stats->status = hctrl.error != 0 ? hctrl.error : host.status;
  stats->rel_resid = host.rel_resid;
  stats->b_norm = host.b_norm;
  if (stats->status != CFD_OK) return cfd_internal_error(stats->status, "noalloc: solver status %d", stats->status);
  return CFD_OK;
}
