// Assembled-matrix path of the pressure operator (Sec. 3.1: the paper
// assembles the Poisson matrix in CSR every step and multiplies with it;
// its optimised version keeps the sparsity pattern).  Here the CSR matrix
// is assembled once on the device and its SpMV set beside the matrix-free
// stencil, to measure what the matrix-free form saves.
//
// Layout in one caller-owned buffer (16-byte aligned pieces):
//   row_ptr  int32 [n + 1]
//   col      int32 [nnz]      (ascending within a row)
//   val      float64 [nnz]    (n_c on the diagonal, -1 per in-box neighbour)
// nnz = 7 n - 2 (nx ny + ny nz + nz nx) for an nx x ny x nz grid.

#include <cstdint>

#include "../../include/cfd.h"
#include "cfd_internal.h"

namespace cfd {
namespace {

constexpr int kCsrThreads = 256;

__device__ __forceinline__ size_t gtid() { return size_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride() { return size_t(gridDim.x) * blockDim.x; }

int64_t csr_nnz(int nx, int ny, int nz) {
  const int64_t n = int64_t(nx) * ny * nz;
  return 7 * n - 2 * (int64_t(nx) * ny + int64_t(ny) * nz + int64_t(nz) * nx);
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct CsrView {
  int32_t* row_ptr;
  int32_t* col;
  double* val;
};

CsrView csr_view(void* buf, int nx, int ny, int nz) {
  const size_t n = size_t(nx) * ny * nz;
  const size_t nnz = size_t(csr_nnz(nx, ny, nz));
  char* p = static_cast<char*>(buf);
  CsrView v;
  v.row_ptr = reinterpret_cast<int32_t*>(p);
  p += align16((n + 1) * 4);
  v.col = reinterpret_cast<int32_t*>(p);
  p += align16(nnz * 4);
  v.val = reinterpret_cast<double*>(p);
  return v;
}

__device__ __forceinline__ int row_len(int i, int j, int k, int nx, int ny, int nz) {
  return 1 + (i > 0) + (i < nx - 1) + (j > 0) + (j < ny - 1) + (k > 0) + (k < nz - 1);
}

// row_ptr[c] = sum of the row lengths of the cells before c = 7 c minus the
// neighbours those cells miss, counted per wall in closed form: cells with
// i = 0 (no x-1): ceil(c / nx); i = nx-1: floor(c / nx); with P = nx ny,
// c = f P + m: j = 0: f nx + min(m, nx); j = ny-1: f nx + max(0, m - (ny-1) nx);
// k = 0: min(c, P); k = nz-1: max(0, c - (nz-1) P).
__global__ void csr_rowptr_kernel(int nx, int ny, int nz, int32_t* row_ptr) {
  const long long n = (long long)nx * ny * nz;
  const long long P = (long long)nx * ny;
  for (size_t cc = gtid(); cc <= size_t(n); cc += gstride()) {
    const long long c = (long long)cc;
    long long miss = (c + nx - 1) / nx + c / nx;
    const long long f = c / P, m = c % P;
    miss += f * nx + (m < nx ? m : nx);
    const long long top = m - (long long)(ny - 1) * nx;
    miss += f * nx + (top > 0 ? top : 0);
    miss += c < P ? c : P;
    const long long last = c - (long long)(nz - 1) * P;
    miss += last > 0 ? last : 0;
    row_ptr[cc] = int32_t(7 * c - miss);
  }
}

__global__ void csr_fill_kernel(int nx, int ny, int nz, const int32_t* row_ptr, int32_t* col, double* val) {
  const size_t n = size_t(nx) * ny * nz;
  const size_t sy = size_t(nx), sz = size_t(nx) * ny;
  for (size_t c = gtid(); c < n; c += gstride()) {
    const int i = int(c % nx), j = int((c / nx) % ny), k = int(c / sz);
    int32_t q = row_ptr[c];
    const int nc = row_len(i, j, k, nx, ny, nz) - 1;
    auto put = [&](size_t cc, double v) {
      col[q] = int32_t(cc);
      val[q] = v;
      ++q;
    };
    if (k > 0) put(c - sz, -1.0);
    if (j > 0) put(c - sy, -1.0);
    if (i > 0) put(c - 1, -1.0);
    put(c, double(nc));
    if (i < nx - 1) put(c + 1, -1.0);
    if (j < ny - 1) put(c + sy, -1.0);
    if (k < nz - 1) put(c + sz, -1.0);
  }
}

// y = A x, one thread per row, entries in stored order
__global__ void __launch_bounds__(kCsrThreads) csr_spmv_kernel(size_t n, const int32_t* __restrict__ row_ptr,
                                                               const int32_t* __restrict__ col,
                                                               const double* __restrict__ val,
                                                               const double* __restrict__ x, double* __restrict__ y) {
  for (size_t r = gtid(); r < n; r += gstride()) {
    double s = 0.0;
    for (int32_t q = row_ptr[r]; q < row_ptr[r + 1]; ++q) s = fma(val[q], x[col[q]], s);
    y[r] = s;
  }
}

int csr_grid(size_t n) {
  size_t b = (n + kCsrThreads - 1) / kCsrThreads;
  return int(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace
}  // namespace cfd

using namespace cfd;

extern "C" {

int cfd_csr_bytes(int32_t nx, int32_t ny, int32_t nz, size_t* bytes, int64_t* nnz) {
  if (nx < 1 || ny < 1 || nz < 1 || !bytes || double(nx) * ny * nz * 7 > 2.0e9)
    return cfd_internal_error(CFD_ERR_INVALID_ARG, "csr: grid sizes >= 1 and 7 n below 2^31, bytes non-NULL");
  const size_t n = size_t(nx) * ny * nz;
  const size_t z = size_t(csr_nnz(nx, ny, nz));
  *bytes = align16((n + 1) * 4) + align16(z * 4) + z * 8;
  if (nnz) *nnz = int64_t(z);
  return CFD_OK;
}

int cfd_csr_assemble(int32_t nx, int32_t ny, int32_t nz, void* dev_buf, cfd_stream_t stream) {
  size_t bytes = 0;
  int rc = cfd_csr_bytes(nx, ny, nz, &bytes, nullptr);
  if (rc) return rc;
  if (!dev_buf || (reinterpret_cast<uintptr_t>(dev_buf) & 15))
    return cfd_internal_error(CFD_ERR_INVALID_ARG, "csr: buffer NULL or not 16-byte aligned");
  const CsrView v = csr_view(dev_buf, nx, ny, nz);
  const size_t n = size_t(nx) * ny * nz;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  csr_rowptr_kernel<<<csr_grid(n + 1), kCsrThreads, 0, s>>>(nx, ny, nz, v.row_ptr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    csr_fill_kernel<<<csr_grid(n), kCsrThreads, 0, s>>>(nx, ny, nz, v.row_ptr, v.col, v.val);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cfd_internal_error(CFD_ERR_CUDA, "csr assemble: %s", cudaGetErrorString(e));
  return CFD_OK;
}

int cfd_csr_spmv(int32_t nx, int32_t ny, int32_t nz, const void* dev_buf, const double* x_dev, double* y_dev,
                 cfd_stream_t stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !dev_buf || !x_dev || !y_dev)
    return cfd_internal_error(CFD_ERR_INVALID_ARG, "csr spmv: NULL argument or empty grid");
  const CsrView v = csr_view(const_cast<void*>(dev_buf), nx, ny, nz);
  const size_t n = size_t(nx) * ny * nz;
  csr_spmv_kernel<<<csr_grid(n), kCsrThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(n, v.row_ptr, v.col, v.val,
                                                                                            x_dev, y_dev);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cfd_internal_error(CFD_ERR_CUDA, "csr spmv: %s", cudaGetErrorString(e));
  return CFD_OK;
}

}  // extern "C"
