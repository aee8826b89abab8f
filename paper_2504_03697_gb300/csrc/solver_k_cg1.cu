// Instantiations of the single-reduction FP64 CG kernel.

#include "solver_impl.cuh"
#include "solver_kernels.h"

namespace cfd {

Cg1Kernel cg1_kernel(int rtz) {
  switch (rtz) {
    case 1: return cg1_fp64_kernel<1>;
    case 2: return cg1_fp64_kernel<2>;
    case 4: return cg1_fp64_kernel<4>;
    case 8: return cg1_fp64_kernel<8>;
    default: return cg1_fp64_kernel<0>;
  }
}

}  // namespace cfd
