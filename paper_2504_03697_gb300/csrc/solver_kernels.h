// Kernel pointers of the persistent solves.  Each kernel family is
// instantiated in its own translation unit (solver_k_*.cu) from the templates
// of solver_impl.cuh, so that the families compile in parallel; solver.cu
// launches them through these pointers.  Internal.
#pragma once

#include "cfd_internal.h"

namespace cfd {

using CgKernel = void (*)(const CgArgs, const CgArgs*, const int*, int);
using Cg1Kernel = void (*)(CgArgs);
using IrKernel = void (*)(const IrArgs, const IrArgs*, const int*, int);

// FP64 textbook CG, one problem; rtz 0: memory path, 1/2/4/8: register path
CgKernel cg_kernel_plain(int rtz);
// the same with the Jacobi preconditioner
CgKernel cg_kernel_jacobi(int rtz);
// multi-problem FP64 CG (memory path), precond 0 or 1
CgKernel cg_kernel_multi(int precond);
// single-reduction FP64 CG, one problem
Cg1Kernel cg1_kernel(int rtz);
// the same, tile-resident: one block of cgt_threads() per tile of depth
// kCgtTileDepth, all CG vectors of the tile in registers (solver_cgt.cu)
Cg1Kernel cgt_kernel();
int cgt_threads();
int cgt_tiles(GridDims g);
// FP32 CG with FP64 refinement: one problem / many problems
IrKernel ir_kernel_single();

}  // namespace cfd
