// Instantiations of the Jacobi-preconditioned FP64 CG kernel (one problem).

#include "solver_impl.cuh"
#include "solver_kernels.h"

namespace cfd {

CgKernel cg_kernel_jacobi(int rtz) {
  switch (rtz) {
    case 1: return cg_fp64_kernel<1, 1, false>;
    case 2: return cg_fp64_kernel<1, 2, false>;
    case 4: return cg_fp64_kernel<1, 4, false>;
    case 8: return cg_fp64_kernel<1, 8, false>;
    default: return cg_fp64_kernel<1, 0, false>;
  }
}

}  // namespace cfd
