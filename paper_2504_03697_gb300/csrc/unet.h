// Internal interface of the tensor-core convolution and the U-Net
// preconditioner (public entry points are declared in include/cfd.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace cfd {

// One stride-1 3D convolution on a channels-last BF16 grid (see unet.cu).
struct ConvArgs {
  int nx, ny, nz;                // grid of input and output
  const __nv_bfloat16* src0;     // [V][c0]
  int c0;
  const __nv_bfloat16* src1;     // [V][c1] (channel-concatenated after src0) or null
  int c1;
  int ks;                        // 3 or 1
  int packed;                    // 1: c0 == 1, ks == 3: K = 27 taps padded to 32
  const __nv_bfloat16* w;        // [ks^3][nout_pad][cin_pad] or packed [nout_pad][32]
  const float* bias;             // [cout] or null
  int cout;                      // output channels (<= nout_pad)
  __nv_bfloat16* dst0;           // [V][split]: channels [0, split)
  __nv_bfloat16* dst1;           // [V][cout - split]: channels [split, cout), or null
  int split;                     // == cout when dst1 is null
  float* dst_f32;                // if non-null: FP32 [V][cout] output instead of dst0/dst1
  int* err;                      // set to 1 on a device-side wait timeout
  int no_tile;                   // 1: never take the TMA-tiled kernel
};

// Launch the convolution: the TMA-tiled kernel for 3x3x3 layers whose
// sources have 16k channels (see conv3d_tile_eligible), else the gathering
// kernel.
cudaError_t launch_conv3d(const ConvArgs& a, int nout_pad, cudaStream_t s);
bool conv3d_tile_eligible(const ConvArgs& a);

}  // namespace cfd
