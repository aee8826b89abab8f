// Grid sweeps of the cavity time step (sm_103a): applyForces, semi-Lagrangian
// advection, diffusion right-hand side, divergence and pressure correction.
//
// Sec. 3.1 of arXiv 2504.03697: at the start of a step the forces g are added
// as a time-invariant offset, the velocity is advected semi-Lagrangianly, and
// the pressure correction computes the divergence, solves the Poisson
// equation and subtracts the gradient (Table 1: applyForces,
// solveAdvection, applyPressureCorrection).
//
// Readings fixed by this library (the paper prints no formulas):
//  * u faces (i, j, k) sit at (i h, (j+1/2) h, (k+1/2) h); v and w likewise.
//  * The lid is the y = ny h wall moving in +x at lid_u; other walls rest.
//  * Tangential samples outside the box are ghosts 2 W - (mirrored sample);
//    along several axes the mirror is applied for z first, then y, then x.
//  * Advection: velocity at the face (own component; other components as the
//    mean of the four surrounding faces, summed with the offset along the
//    face's own axis outermost), one explicit Euler backtrace, clamp into
//    the box, trilinear interpolation of the old field with floor lookup.
//  * Forcing: component c of every non-wall-normal face in the top cell
//    layer (j = ny - 1) gains dt g[c].
//  * Divergence right-hand side: b = -(rho h / dt) * (sum of outgoing face
//    differences); correction u_f -= dt / (rho h) (p_c - p_c').
//
// All sweeps are HBM/L2-bound elementwise passes: one thread per face or
// cell, x fastest across the warp so every load and store is coalesced.

#include "cfd_internal.h"

namespace cfd {

namespace {

constexpr int kSweepThreads = 256;

__device__ __forceinline__ size_t gtid() { return size_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ size_t gstride() { return size_t(gridDim.x) * blockDim.x; }

struct FaceDims {
  int mx, my, mz;
};

// (i, j, k) of linear index l in an mx x my x mz array (fewer than 2^32
// elements: 32-bit divisions)
__device__ __forceinline__ void decode3(size_t l, int mx, int my, int& i, int& j, int& k) {
  const unsigned u = unsigned(l), row = u / unsigned(mx);
  i = int(u - row * unsigned(mx));
  k = int(row / unsigned(my));
  j = int(row - unsigned(k) * unsigned(my));
}

__device__ __forceinline__ FaceDims face_dims(int comp, int nx, int ny, int nz) {
  return FaceDims{nx + (comp == 0), ny + (comp == 1), nz + (comp == 2)};
}

// Sample of face field f (component comp) at integer face index (i, j, k),
// which may lie one layer outside the box on tangential axes (ghost rule).
__device__ __forceinline__ double sample(const double* __restrict__ f, int comp, int i, int j, int k, int nx,
                                         int ny, int nz, double lid_u) {
  const FaceDims d = face_dims(comp, nx, ny, nz);
  // inside the array (the common case) the sample is the stored value
  if (i >= 0 && i < d.mx && j >= 0 && j < d.my && k >= 0 && k < d.mz) return f[idx3(i, j, k, d.mx, d.my)];
  double add = 0.0, sgn = 1.0;
  if (comp != 2) {
    if (k < 0) { k = 0; sgn = -sgn; }
    else if (k >= nz) { k = nz - 1; sgn = -sgn; }
  }
  if (comp != 1) {
    if (j < 0) { j = 0; sgn = -sgn; }
    else if (j >= ny) {
      j = ny - 1;
      if (comp == 0) add += sgn * (2.0 * lid_u);
      sgn = -sgn;
    }
  }
  if (comp != 0) {
    if (i < 0) { i = 0; sgn = -sgn; }
    else if (i >= nx) { i = nx - 1; sgn = -sgn; }
  }
  const double v = f[idx3(i, j, k, d.mx, d.my)];
  return add + sgn * v;
}

__device__ __forceinline__ double lerp(double a, double b, double t) { return a + t * (b - a); }

__device__ double interpolate(const double* __restrict__ f, int comp, double X, double Y, double Z, int nx,
                              int ny, int nz, double inv_h, double lid_u) {
  double g[3] = {X * inv_h, Y * inv_h, Z * inv_h};
  const int n[3] = {nx, ny, nz};
  int lo[3];
  double t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int lmin = 0;
    if (d != comp) {
      g[d] -= 0.5;
      lmin = -1;
    }
    int l = __double2int_rd(g[d]);
    l = l < lmin ? lmin : (l > n[d] - 1 ? n[d] - 1 : l);
    lo[d] = l;
    t[d] = g[d] - double(l);
  }
  const int i0 = lo[0], j0 = lo[1], k0 = lo[2];
  const double c00 = lerp(sample(f, comp, i0, j0, k0, nx, ny, nz, lid_u), sample(f, comp, i0 + 1, j0, k0, nx, ny, nz, lid_u), t[0]);
  const double c10 = lerp(sample(f, comp, i0, j0 + 1, k0, nx, ny, nz, lid_u), sample(f, comp, i0 + 1, j0 + 1, k0, nx, ny, nz, lid_u), t[0]);
  const double c01 = lerp(sample(f, comp, i0, j0, k0 + 1, nx, ny, nz, lid_u), sample(f, comp, i0 + 1, j0, k0 + 1, nx, ny, nz, lid_u), t[0]);
  const double c11 = lerp(sample(f, comp, i0, j0 + 1, k0 + 1, nx, ny, nz, lid_u), sample(f, comp, i0 + 1, j0 + 1, k0 + 1, nx, ny, nz, lid_u), t[0]);
  const double c0 = lerp(c00, c10, t[1]);
  const double c1 = lerp(c01, c11, t[1]);
  return lerp(c0, c1, t[2]);
}

// Mean of the four faces of component d around face (i, j, k) of component
// c: offsets oc in {-1, 0} along c's axis (outer), od in {0, +1} along d's.
__device__ __forceinline__ double face_avg(const double* __restrict__ f, int c, int d, int i, int j, int k, int nx,
                                           int ny, int nz) {
  const FaceDims fd = face_dims(d, nx, ny, nz);
  double s = 0.0;
#pragma unroll
  for (int oc = -1; oc <= 0; ++oc) {
#pragma unroll
    for (int od = 0; od <= 1; ++od) {
      int ii = i, jj = j, kk = k;
      if (c == 0) ii += oc; else if (c == 1) jj += oc; else kk += oc;
      if (d == 0) ii += od; else if (d == 1) jj += od; else kk += od;
      s = s + f[idx3(ii, jj, kk, fd.mx, fd.my)];
    }
  }
  return 0.25 * s;
}

// Each sweep is a body over the elements t0, t0 + stride, ... of one cavity:
// the whole grid in the single-cavity kernels, the cavity's block range in
// the batched ones (sweep_multi_kernel).
__device__ __forceinline__ void advect_body(const PhysArgs& a, size_t t0, size_t stride) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t n0 = size_t(nx + 1) * ny * nz;
  const size_t n1 = size_t(nx) * (ny + 1) * nz;
  const size_t n2 = size_t(nx) * ny * (nz + 1);
  const double ext[3] = {nx * a.h, ny * a.h, nz * a.h};
  const double* fields[3] = {a.u, a.v, a.w};
  double* outs[3] = {a.ua, a.va, a.wa};
  for (size_t e = t0; e < n0 + n1 + n2; e += stride) {
    int comp;
    size_t l;
    if (e < n0) { comp = 0; l = e; }
    else if (e < n0 + n1) { comp = 1; l = e - n0; }
    else { comp = 2; l = e - n0 - n1; }
    const FaceDims fd = face_dims(comp, nx, ny, nz);
    int i, j, k;
    decode3(l, fd.mx, fd.my, i, j, k);
    const int own = comp == 0 ? i : (comp == 1 ? j : k);
    const int own_n = comp == 0 ? nx : (comp == 1 ? ny : nz);
    if (own == 0 || own == own_n) {
      outs[comp][l] = 0.0;
      continue;
    }
    double pos[3] = {(i + 0.5) * a.h, (j + 0.5) * a.h, (k + 0.5) * a.h};
    pos[comp] = (comp == 0 ? i : (comp == 1 ? j : k)) * a.h;
    double vel[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d == comp) vel[d] = fields[comp][l];
      else vel[d] = face_avg(fields[d], comp, d, i, j, k, nx, ny, nz);
    }
    if (a.rk2) {
      // explicit midpoint: velocity sampled at x - dt/2 v(x), each component
      // from its own grid
      double mid[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double x = pos[d] - 0.5 * a.dt * vel[d];
        x = x < 0.0 ? 0.0 : (x > ext[d] ? ext[d] : x);
        mid[d] = x;
      }
#pragma unroll
      for (int d = 0; d < 3; ++d)
        vel[d] = interpolate(fields[d], d, mid[0], mid[1], mid[2], nx, ny, nz, a.inv_h, a.lid_u);
    }
    double back[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double x = pos[d] - a.dt * vel[d];
      x = x < 0.0 ? 0.0 : (x > ext[d] ? ext[d] : x);
      back[d] = x;
    }
    outs[comp][l] = interpolate(fields[comp], comp, back[0], back[1], back[2], nx, ny, nz, a.inv_h, a.lid_u);
  }
}

__global__ void __launch_bounds__(kSweepThreads) advect_kernel(PhysArgs a) { advect_body(a, gtid(), gstride()); }

__device__ __forceinline__ void forces_body(const PhysArgs& a, size_t t0, size_t stride) {
  // top cell layer j = ny - 1 of each component, non-wall-normal faces only
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t n0 = size_t(nx + 1) * nz, n1 = size_t(nx) * nz, n2 = size_t(nx) * (nz + 1);
  double* fs[3] = {a.u, a.v, a.w};
  for (size_t e = t0; e < n0 + n1 + n2; e += stride) {
    int comp;
    size_t l;
    if (e < n0) { comp = 0; l = e; }
    else if (e < n0 + n1) { comp = 1; l = e - n0; }
    else { comp = 2; l = e - n0 - n1; }
    const FaceDims fd = face_dims(comp, nx, ny, nz);
    const int i = int(l % fd.mx), k = int(l / fd.mx);
    const int j = ny - 1;
    if (comp == 0 && (i == 0 || i == nx)) continue;
    if (comp == 1 && j == 0) continue;  // ny == 1: the top layer is a wall face
    if (comp == 2 && (k == 0 || k == nz)) continue;
    const double inc = a.dt * a.g[comp];
    fs[comp][idx3(i, j, k, fd.mx, fd.my)] += inc;
  }
}

__global__ void __launch_bounds__(kSweepThreads) forces_kernel(PhysArgs a) { forces_body(a, gtid(), gstride()); }

// b = ua_c (+ c * 2 lid_u on u faces touching the lid); zero on wall rows.
// lid_term = c * (2 lid_u), c = nu dt / h^2.
__host__ __device__ __forceinline__ double diffusion_lid_term(const PhysArgs& a) {
  const double c = a.nu * a.dt / (a.h * a.h);
  return c * (2.0 * a.lid_u);
}

__device__ __forceinline__ void diffusion_rhs_body(const PhysArgs& a, int comp, double lid_term, size_t t0,
                                                   size_t stride) {
  const FaceDims fd = face_dims(comp, a.nx, a.ny, a.nz);
  const size_t n = size_t(fd.mx) * fd.my * fd.mz;
  const double* f = comp == 0 ? a.ua : (comp == 1 ? a.va : a.wa);
  for (size_t e = t0; e < n; e += stride) {
    int i, j, k;
    decode3(e, fd.mx, fd.my, i, j, k);
    const int own = comp == 0 ? i : (comp == 1 ? j : k);
    const int own_n = comp == 0 ? a.nx : (comp == 1 ? a.ny : a.nz);
    double v = 0.0;
    if (own != 0 && own != own_n) {
      v = f[e];
      if (comp == 0 && j == a.ny - 1) v = v + lid_term;
    }
    a.b[e] = v;
  }
}

__global__ void __launch_bounds__(kSweepThreads) diffusion_rhs_kernel(PhysArgs a, int comp, double lid_term) {
  diffusion_rhs_body(a, comp, lid_term, gtid(), gstride());
}

// scale = -(rho h / dt)
__host__ __device__ __forceinline__ double divergence_scale(const PhysArgs& a) { return -(a.rho * a.h / a.dt); }

__device__ __forceinline__ void divergence_body(const PhysArgs& a, double scale, size_t t0, size_t stride) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t n = size_t(nx) * ny * nz;
  for (size_t e = t0; e < n; e += stride) {
    int i, j, k;
    decode3(e, nx, ny, i, j, k);
    const double du = a.ua[idx3(i + 1, j, k, nx + 1, ny)] - a.ua[idx3(i, j, k, nx + 1, ny)];
    const double dv = a.va[idx3(i, j + 1, k, nx, ny + 1)] - a.va[idx3(i, j, k, nx, ny + 1)];
    const double dw = a.wa[idx3(i, j, k + 1, nx, ny)] - a.wa[idx3(i, j, k, nx, ny)];
    a.b[e] = scale * ((du + dv) + dw);
  }
}

__global__ void __launch_bounds__(kSweepThreads) divergence_kernel(PhysArgs a, double scale) {
  divergence_body(a, scale, gtid(), gstride());
}

// s = dt / (rho h)
__host__ __device__ __forceinline__ double correct_scale(const PhysArgs& a) { return a.dt / (a.rho * a.h); }

__device__ __forceinline__ void correct_body(const PhysArgs& a, double s, size_t t0, size_t stride) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t n0 = size_t(nx + 1) * ny * nz;
  const size_t n1 = size_t(nx) * (ny + 1) * nz;
  const size_t n2 = size_t(nx) * ny * (nz + 1);
  for (size_t e = t0; e < n0 + n1 + n2; e += stride) {
    int comp;
    size_t l;
    if (e < n0) { comp = 0; l = e; }
    else if (e < n0 + n1) { comp = 1; l = e - n0; }
    else { comp = 2; l = e - n0 - n1; }
    const FaceDims fd = face_dims(comp, nx, ny, nz);
    int i, j, k;
    decode3(l, fd.mx, fd.my, i, j, k);
    const double* in = comp == 0 ? a.ua : (comp == 1 ? a.va : a.wa);
    double* out = comp == 0 ? a.u : (comp == 1 ? a.v : a.w);
    const int own = comp == 0 ? i : (comp == 1 ? j : k);
    const int own_n = comp == 0 ? nx : (comp == 1 ? ny : nz);
    if (own == 0 || own == own_n) {
      out[l] = 0.0;
      continue;
    }
    const double pc = a.p[idx3(i, j, k, nx, ny)];
    const double pm = comp == 0 ? a.p[idx3(i - 1, j, k, nx, ny)]
                                : (comp == 1 ? a.p[idx3(i, j - 1, k, nx, ny)] : a.p[idx3(i, j, k - 1, nx, ny)]);
    out[l] = in[l] - s * (pc - pm);
  }
}

__global__ void __launch_bounds__(kSweepThreads) correct_kernel(PhysArgs a, double s) {
  correct_body(a, s, gtid(), gstride());
}

// Batched sweeps: one launch over many cavities, cavity k on the blocks
// [starts[k], starts[k+1]) (op: SweepOp; comp: the diffusion component).
template <int OP>
__global__ void __launch_bounds__(kSweepThreads) sweep_multi_kernel(const PhysArgs* __restrict__ tab,
                                                                    const int* __restrict__ starts, int nprob,
                                                                    int comp) {
  int lo = 0, hi = nprob - 1;
  const int blk = int(blockIdx.x);
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const PhysArgs& a = tab[lo];
  const size_t t0 = size_t(blk - starts[lo]) * blockDim.x + threadIdx.x;
  const size_t st = size_t(starts[lo + 1] - starts[lo]) * blockDim.x;
  if (OP == kSweepAdvect) advect_body(a, t0, st);
  else if (OP == kSweepForces) forces_body(a, t0, st);
  else if (OP == kSweepDiffusionRhs) diffusion_rhs_body(a, comp, diffusion_lid_term(a), t0, st);
  else if (OP == kSweepDivergence) divergence_body(a, divergence_scale(a), t0, st);
  else correct_body(a, correct_scale(a), t0, st);
}

__global__ void __launch_bounds__(kSweepThreads) zero_wall_faces_kernel(PhysArgs a) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  // u: i = 0, nx ; v: j = 0, ny ; w: k = 0, nz
  const size_t n0 = size_t(2) * ny * nz, n1 = size_t(2) * nx * nz, n2 = size_t(2) * nx * ny;
  for (size_t e = gtid(); e < n0 + n1 + n2; e += gstride()) {
    if (e < n0) {
      const int side = int(e % 2), rest = int(e / 2), j = rest % ny, k = rest / ny;
      a.u[idx3(side ? nx : 0, j, k, nx + 1, ny)] = 0.0;
    } else if (e < n0 + n1) {
      const size_t l = e - n0;
      const int side = int(l % 2), rest = int(l / 2), i = rest % nx, k = rest / nx;
      a.v[idx3(i, side ? ny : 0, k, nx, ny + 1)] = 0.0;
    } else {
      const size_t l = e - n0 - n1;
      const int side = int(l % 2), rest = int(l / 2), i = rest % nx, j = rest / nx;
      a.w[idx3(i, j, side ? nz : 0, nx, ny)] = 0.0;
    }
  }
}

__global__ void __launch_bounds__(kSweepThreads) fill_kernel(double* p, size_t n, double value) {
  for (size_t e = gtid(); e < n; e += gstride()) p[e] = value;
}


// ---------------------------------------------------------------------------
// Training pairs of the learned preconditioner: with b' = b - mean(b), the
// residual of an iterate x_k is r = b' - A x_k and its error against the
// converged solution x* is e = (x* - x_k) - mean(x* - x_k) (the Neumann
// system fixes x only up to a constant).  Means by fixed-order sums.
// ---------------------------------------------------------------------------
constexpr int kHarvestBlocks = 512;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();
  return t;  // valid in thread 0
}

// part[block] = sum of b, part[nb + block] = sum of x* - x_k over the block's cells
__global__ void __launch_bounds__(kSweepThreads) harvest_sums_kernel(const double* b, const double* xs,
                                                                     const double* xk, size_t n, double* part) {
  __shared__ double sh[kSweepThreads / 32];
  double sb = 0.0, se = 0.0;
  for (size_t e = gtid(); e < n; e += gstride()) {
    sb += b[e];
    se += xs[e] - xk[e];
  }
  sb = block_sum(sb, sh);
  se = block_sum(se, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sb;
    part[gridDim.x + blockIdx.x] = se;
  }
}

// one block: part[2 nb] = mean(b), part[2 nb + 1] = mean(x* - x_k), summing
// the block sums in block order
__global__ void __launch_bounds__(kSweepThreads) harvest_means_kernel(double* part, int nb, size_t n) {
  __shared__ double sh[kSweepThreads / 32];
  double sb = 0.0, se = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    sb += part[i];
    se += part[nb + i];
  }
  sb = block_sum(sb, sh);
  se = block_sum(se, sh);
  if (threadIdx.x == 0) {
    part[2 * nb] = sb / double(n);
    part[2 * nb + 1] = se / double(n);
  }
}

// r holds A x_k on entry: r = (b - mean b) - A x_k, e = (x* - x_k) - mean
__global__ void __launch_bounds__(kSweepThreads) harvest_pair_kernel(const double* b, const double* xs,
                                                                     const double* xk, size_t n,
                                                                     const double* means, double* r, double* e) {
  const double mb = means[0], me = means[1];
  for (size_t c = gtid(); c < n; c += gstride()) {
    r[c] = (b[c] - mb) - r[c];
    e[c] = (xs[c] - xk[c]) - me;
  }
}

int sweep_blocks(size_t n) {
  size_t b = (n + kSweepThreads - 1) / kSweepThreads;
  const size_t cap = 152 * 16;  // grid-stride beyond ~16 resident blocks per SM
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return int(b);
}

}  // namespace

cudaError_t launch_advect(const PhysArgs& a, cudaStream_t s, int64_t* launches) {
  const size_t n = size_t(a.nx + 1) * a.ny * a.nz + size_t(a.nx) * (a.ny + 1) * a.nz + size_t(a.nx) * a.ny * (a.nz + 1);
  advect_kernel<<<sweep_blocks(n), kSweepThreads, 0, s>>>(a);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_forces(const PhysArgs& a, cudaStream_t s, int64_t* launches) {
  const size_t n = size_t(a.nx + 1) * a.nz + size_t(a.nx) * a.nz + size_t(a.nx) * (a.nz + 1);
  forces_kernel<<<sweep_blocks(n), kSweepThreads, 0, s>>>(a);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_diffusion_rhs(const PhysArgs& a, int comp, cudaStream_t s, int64_t* launches) {
  const size_t n = size_t(a.nx + (comp == 0)) * (a.ny + (comp == 1)) * (a.nz + (comp == 2));
  diffusion_rhs_kernel<<<sweep_blocks(n), kSweepThreads, 0, s>>>(a, comp, diffusion_lid_term(a));
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_divergence(const PhysArgs& a, cudaStream_t s, int64_t* launches) {
  const size_t n = size_t(a.nx) * a.ny * a.nz;
  divergence_kernel<<<sweep_blocks(n), kSweepThreads, 0, s>>>(a, divergence_scale(a));
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_correct(const PhysArgs& a, cudaStream_t s, int64_t* launches) {
  const size_t n = size_t(a.nx + 1) * a.ny * a.nz + size_t(a.nx) * (a.ny + 1) * a.nz + size_t(a.nx) * a.ny * (a.nz + 1);
  correct_kernel<<<sweep_blocks(n), kSweepThreads, 0, s>>>(a, correct_scale(a));
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_zero_wall_faces(const PhysArgs& a, cudaStream_t s, int64_t* launches) {
  const size_t n = size_t(2) * (size_t(a.ny) * a.nz + size_t(a.nx) * a.nz + size_t(a.nx) * a.ny);
  zero_wall_faces_kernel<<<sweep_blocks(n), kSweepThreads, 0, s>>>(a);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

size_t sweep_elems(const PhysArgs& a, int op, int comp) {
  const size_t faces = size_t(a.nx + 1) * a.ny * a.nz + size_t(a.nx) * (a.ny + 1) * a.nz +
                       size_t(a.nx) * a.ny * (a.nz + 1);
  switch (op) {
    case kSweepAdvect:
    case kSweepCorrect:
      return faces;
    case kSweepForces:
      return size_t(a.nx + 1) * a.nz + size_t(a.nx) * a.nz + size_t(a.nx) * (a.nz + 1);
    case kSweepDiffusionRhs:
      return size_t(a.nx + (comp == 0)) * (a.ny + (comp == 1)) * (a.nz + (comp == 2));
    default:
      return size_t(a.nx) * a.ny * a.nz;
  }
}

int sweep_blocks_for(const PhysArgs& a, int op, int comp) { return sweep_blocks(sweep_elems(a, op, comp)); }

cudaError_t launch_sweep_multi(int op, const PhysArgs* d_tab, const int* d_starts, int nprob, int total_blocks,
                               int comp, cudaStream_t s, int64_t* launches) {
  if (nprob <= 0) return cudaSuccess;
  const dim3 g{unsigned(total_blocks)}, b{unsigned(kSweepThreads)};
  switch (op) {
    case kSweepAdvect: sweep_multi_kernel<kSweepAdvect><<<g, b, 0, s>>>(d_tab, d_starts, nprob, comp); break;
    case kSweepForces: sweep_multi_kernel<kSweepForces><<<g, b, 0, s>>>(d_tab, d_starts, nprob, comp); break;
    case kSweepDiffusionRhs:
      sweep_multi_kernel<kSweepDiffusionRhs><<<g, b, 0, s>>>(d_tab, d_starts, nprob, comp);
      break;
    case kSweepDivergence: sweep_multi_kernel<kSweepDivergence><<<g, b, 0, s>>>(d_tab, d_starts, nprob, comp); break;
    default: sweep_multi_kernel<kSweepCorrect><<<g, b, 0, s>>>(d_tab, d_starts, nprob, comp); break;
  }
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_fill(double* p, size_t n, double value, cudaStream_t s, int64_t* launches) {
  fill_kernel<<<sweep_blocks(n), kSweepThreads, 0, s>>>(p, n, value);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_harvest_pair(GridDims g, const double* b, const double* xs, const double* xk, double* r, double* e,
                                double* scratch, cudaStream_t s, int64_t* launches) {
  const size_t n = g.count();
  int nb = sweep_blocks(n);
  if (nb > kHarvestBlocks) nb = kHarvestBlocks;
  harvest_sums_kernel<<<nb, kSweepThreads, 0, s>>>(b, xs, xk, n, scratch);
  harvest_means_kernel<<<1, kSweepThreads, 0, s>>>(scratch, nb, n);
  if (launches) *launches += 2;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  err = launch_apply_poisson(g, xk, r, 0, s, launches);
  if (err != cudaSuccess) return err;
  harvest_pair_kernel<<<sweep_blocks(n), kSweepThreads, 0, s>>>(b, xs, xk, n, scratch + 2 * nb, r, e);
  if (launches) *launches += 1;
  return cudaGetLastError();
}

size_t harvest_scratch_doubles() { return size_t(2) * kHarvestBlocks + 2; }

}  // namespace cfd
