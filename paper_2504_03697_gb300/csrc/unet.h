// Internal interface of the tensor-core convolution and the U-Net
// preconditioner (public entry points are declared in include/cfd.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/cfd.h"

namespace cfd {

// Activation layout ("channel-octet planes"): a tensor of C channels on V
// voxels (x fastest) is stored as ceil(C / W) planes of [V][W] BF16, W =
// min(C, 8).  Eight channels of a voxel are one 16-byte vector, and within a
// plane consecutive voxels are consecutive 16-byte vectors, so a box of
// voxels of one plane is a set of contiguous x-runs (what a TMA copy moves
// efficiently) and a warp's stores of consecutive voxels coalesce.
__host__ __device__ inline size_t oct_index(size_t v, int c, int C, size_t V) {
  const int W = C < 8 ? C : 8;
  return (size_t(c / W) * V + v) * size_t(W) + size_t(c % W);
}

// One stride-1 3D convolution on a BF16 grid in octet planes (see unet.cu).
struct ConvArgs {
  int nx, ny, nz;                // grid of input and output
  const __nv_bfloat16* src0;     // c0 channels, octet planes (oct_index)
  int c0;
  const __nv_bfloat16* src1;     // c1 channels (concatenated after src0) or null
  int c1;
  int ks;                        // 3 or 1
  int packed;                    // 1: c0 == 1, ks == 3: K = 27 taps padded to 32
  const __nv_bfloat16* w;        // [ks^3][nout_pad][cin_pad] or packed [nout_pad][32]
  const __nv_bfloat16* w_cm;     // or null: the same 3x3x3 weights in shared-memory order,
                                 // [cin_pad/16][27] blocks of nout_pad x 16 K-major core
                                 // matrices (the tiled kernel then streams them with bulk copies)
  const float* bias;             // [cout] or null
  int cout;                      // output channels (<= nout_pad)
  __nv_bfloat16* dst0;           // channels [0, split), octet planes
  __nv_bfloat16* dst1;           // channels [split, cout), octet planes, or null
  int split;                     // == cout when dst1 is null
  float* dst_f32;                // if non-null: FP32 [V][cout] output instead of dst0/dst1
  int* err;                      // set to 1 on a device-side wait timeout
  int no_tile;                   // 1: never take the TMA-tiled kernel
  int stages;                    // with w_cm: 1 (default) or 2 shared-memory stages
};

// Hooks for solvers that run the U-Net inside their own CUDA graphs
// (ir_graph.cu): its BF16 input plane and FP32 output, its grid, and the
// forward pass enqueued on a given stream.  The forward pass is kernel
// launches only (no allocation, no synchronisation), so it can be captured.
struct UNetView {
  int nx, ny, nz;
  __nv_bfloat16* xin;  // network input, BF16 [V]
  float* z;            // head output, FP32 [V]
  int* err;            // device flag set by a timed-out tensor-core wait
  int conv_mode;       // CFD_UNET_CONV_* (changes the captured kernels)
};
bool unet_view(const cfd_unet* u, UNetView* v);
// Forward pass xin -> z on stream s; *kernels (nullable) receives the
// number of kernels it launched.  Returns CFD_OK or a CFD_ERR_* code.
int unet_forward_on(cfd_unet* u, cudaStream_t s, int* kernels);

// Weight gradient of a stride-1 3x3x3 convolution (input src0 with c0
// channels, then src1 with c1, octet planes; output gradient g with cout
// channels) on the tensor cores: FP32 partial sums partial[chunk][27][cout]
// [cin] and bias_partial[chunk][cout] for *chunks_out <= max_chunks chunks,
// to be summed over the chunks in order.  Returns cudaErrorNotSupported (and
// launches nothing) when the layer does not fit: channel counts not
// multiples of 8 or outside [16, 128], the smaller of cin and cout not 16,
// 32 or 64, or no tensor-map encoder.  err: set to 1 if a wait timed out.
cudaError_t launch_wgrad_tc(const __nv_bfloat16* src0, int c0, const __nv_bfloat16* src1, int c1,
                            const __nv_bfloat16* g, int cout, int nx, int ny, int nz, float* partial,
                            float* bias_partial, int max_chunks, int* chunks_out, int* err, cudaStream_t s);

// Launch the convolution: the TMA-tiled kernel for 3x3x3 layers whose
// sources have 16k channels (see conv3d_tile_eligible), else the gathering
// kernel.
cudaError_t launch_conv3d(const ConvArgs& a, int nout_pad, cudaStream_t s);
bool conv3d_tile_eligible(const ConvArgs& a);

}  // namespace cfd
