// Instantiations of the FP32-CG / FP64-refinement kernel (one problem, many problems).

#include "solver_impl.cuh"
#include "solver_kernels.h"

namespace cfd {

IrKernel ir_kernel_single() { return ir_kernel<false>; }

IrKernel ir_kernel_multi() { return ir_kernel<true>; }

}  // namespace cfd
