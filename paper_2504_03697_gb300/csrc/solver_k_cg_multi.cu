// Instantiations of the multi-problem FP64 CG kernel (batches).

#include "solver_impl.cuh"
#include "solver_kernels.h"

namespace cfd {

CgKernel cg_kernel_multi(int precond) { return precond ? cg_fp64_kernel<1, 0, true> : cg_fp64_kernel<0, 0, true>; }

}  // namespace cfd
