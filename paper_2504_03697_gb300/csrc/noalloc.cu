// Allocation-free variant of the standalone pressure solve.
//
// Some callers cannot allocate device memory at all: plug-ins whose host
// application owns the allocator and forbids outside allocations, or
// embedded runtimes that reserve all device memory up front.
// cfd_poisson_solve_noalloc serves them: it runs the persistent FP64 CG of
// cfd_solve_pressure in its two-reduction (textbook) form -- the array has
// no room for the three extra vectors of the single-reduction form, so
// rounding and iteration counts may differ slightly from cfd_solve_pressure's
// default form -- with its scratch vectors in one file-scope __device__
// array of fixed size instead of a caller-provided workspace, and it calls
// no allocating routine (no cudaMalloc / cudaFree, no torch, no library
// that allocates).  It does call the CUDA runtime (copies, a memset, a
// kernel launch), so it must not be called from inside a CUDA stream
// callback (cudaLaunchHostFunc), where CUDA calls are not allowed.
//
// Limits and sharing rules (also stated in include/cfd.h):
//  * at most CFD_NOALLOC_MAX_CELLS cells; larger grids are rejected with
//    CFD_ERR_INVALID_ARG;
//  * every GPU that loads this library holds the array (about 11 MB) until
//    the process exits;
//  * all calls share the one array per device, so calls whose GPU work
//    overlaps (different streams, or different host threads on one device)
//    race; serialise them on one stream;
//  * the first call on a device looks up the array's device address (with
//    that device current); make that first call before any stream capture.
//    A failed lookup is not cached: the next call on that device tries again.

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
  std::mutex mu;
  unsigned char* ptr = nullptr;  // device address of g_noalloc_scratch on that device (set once found)
  int blocks = 0;                // co-resident blocks of the solve kernel, capped at kNoallocMaxBlocks
};
DeviceScratch g_dev[kMaxDevices];

// The device address of the array and the launch width on the current
// device, looked up on the first successful call and kept; a failed lookup
// leaves nothing behind, so that a later call tries again.
cudaError_t device_scratch(DeviceScratch& ds, unsigned char** ptr, int* blocks) {
  std::lock_guard<std::mutex> lock(ds.mu);
  if (!ds.ptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    int nb = cg_max_coresident_blocks(0);
    if (nb < 1) return cudaErrorInvalidConfiguration;
    ds.blocks = nb > kNoallocMaxBlocks ? kNoallocMaxBlocks : nb;
    ds.ptr = static_cast<unsigned char*>(p);
  }
  *ptr = ds.ptr;
  *blocks = ds.blocks;
  return cudaSuccess;
}

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
  // host code may not use the array's name as an address: look the device
  // address up with this device current (kept after the first success)
  unsigned char* base = nullptr;
  int blocks = 0;
  e = device_scratch(g_dev[dev], &base, &blocks);
  if (e != cudaSuccess)
    return cfd_internal_error(CFD_ERR_CUDA, "noalloc: scratch lookup on device %d: %s", dev, cudaGetErrorString(e));

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
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
  // e0..e2 stay null: launch_cg then takes the two-reduction CG form, and it
  // picks the stencil tile depth itself
  LaunchGeom lg{};
  lg.blocks = blocks;
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
