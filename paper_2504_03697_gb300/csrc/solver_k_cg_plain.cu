// Instantiations of the FP64 CG kernel without preconditioner (one problem).

#include "solver_impl.cuh"
#include "solver_kernels.h"

namespace cfd {

CgKernel cg_kernel_plain(int rtz) {
  switch (rtz) {
    case 1: return cg_fp64_kernel<0, 1, false>;
    case 2: return cg_fp64_kernel<0, 2, false>;
    case 4: return cg_fp64_kernel<0, 4, false>;
    case 8: return cg_fp64_kernel<0, 8, false>;
    default: return cg_fp64_kernel<0, 0, false>;
  }
}

}  // namespace cfd
