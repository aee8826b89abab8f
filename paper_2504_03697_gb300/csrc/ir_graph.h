// Graph-driven mixed-precision pressure solve (see ir_graph.cu).  Internal.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "cfd_internal.h"

namespace cfd {

struct IrGraph;  // an instantiated graph, cached per workspace and arguments

// Cells each FP32 vector of the mixed-precision solves needs for an nx x ny
// x nz cavity: the velocity matrices' rows are padded to a multiple of 4
// cells in the graph and batched forms.
size_t ir_fp32_vector_cells(int nx, int ny, int nz);
// Device bytes of the solver state and partial sums (16-byte aligned).
size_t ir_graph_state_bytes();
// The graph form needs mx % 4 == 0 (16-byte rows of the FP32 vectors).
bool ir_graph_eligible(const IrArgs& a);
// Enqueue one solve on s; builds (or rebuilds, when the arguments changed)
// the graph in *cache.  Same results contract as launch_ir: statistics in
// a.stats, x the solution.  a.ctrl, a.partials, a.tz and the TMA fields are
// not used.
cudaError_t launch_ir_graph(const IrArgs& a, void* state_buf, IrGraph** cache, cudaStream_t s);
void destroy_ir_graph(IrGraph* g);
// The learned initial guess alone, enqueued on s: a.x = alpha (z - mean z),
// z = U(s (a.b - mean)), alpha the energy line search (a.net, the pressure
// matrix, mx % 4 == 0).  Uses the state buffer's scalars and partial sums.
cudaError_t launch_learned_guess(const IrArgs& a, void* state_buf, cudaStream_t s, int64_t* launches);
// Batched form: nprob independent systems in one persistent cooperative
// launch, problem k on the blocks [d_starts[k], d_starts[k+1]).  Each
// problem's IrArgs supplies the vectors, the operator, ctrl (its
// synchronisation words, zeroed before every launch), stats and
// timeout_ns; its state buffer (ir_graph_state_bytes()) holds the partial
// sums.  ir_batch_table writes the device table (ir_batch_table_bytes) once
// (synchronises s); launch_ir_batch runs the solves (kind: the kOp* operator
// of every problem of the launch).  At most ir_batch_blocks_per_sm(kind)
// blocks per SM, and at most 1024 per problem.
// One problem's work in the batched launch: its (row, plane) work items per
// pass, and its largest extent (a proxy for the iteration count).  A solve
// on nb blocks takes about extent * ceil(items / nb) item passes.
void ir_batch_work(const IrArgs& ia, int* items, int* extent);
size_t ir_batch_table_bytes(int nprob);
cudaError_t ir_batch_table(const IrArgs* args, void* const* states, int nprob, void* d_table, cudaStream_t s);
int ir_batch_blocks_per_sm(int kind);
cudaError_t launch_ir_batch(const void* d_table, const int* d_starts, int nprob, int total_blocks, int kind,
                            cudaStream_t s, int64_t* launches);
// Kernels run so far by graph solves on this state buffer (synchronises s).
cudaError_t ir_graph_kernel_count(const void* state_buf, cudaStream_t s, long long* out);

}  // namespace cfd
