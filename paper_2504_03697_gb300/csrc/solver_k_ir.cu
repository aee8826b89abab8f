// Instantiation of the FP32-CG / FP64-refinement kernel (one problem; batches
// run the batched graph-form solve of ir_graph.cu).

#include "solver_impl.cuh"
#include "solver_kernels.h"

namespace cfd {

IrKernel ir_kernel_single() { return ir_kernel<false>; }

}  // namespace cfd
