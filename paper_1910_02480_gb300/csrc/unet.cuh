// unet.cuh -- the paper's own network form (Sec. 3.3, "Neural network"): a
// U-Net of two 3x3 convolutions per stage with batch normalisation and
// LeakyReLU, 2x2 max pooling, 2x bilinear upsampling, concatenated skips and
// a 1x1 head with ReLU, in FP32: its 3x3 layers on the tensor cores where
// the shape allows (the conv kernel family of conv_tc.cuh), else on the CUDA
// cores.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "trace.cuh"

namespace drc {

struct UnetShape {
  int cin, cout, base, levels;
};

// Packed parameter count (layer order of the C ABI's description).
size_t unet_param_count(const UnetShape &u);
// Workspace for N maps of H x W: folded weights and every activation.
size_t unet_workspace_bytes(const UnetShape &u, int N, int H, int W);
// The forward pass; the shapes are checked by the caller.
cudaError_t unet_forward(const UnetShape &u, const float *params, const float *in, float *out, int N, int H, int W,
                         void *workspace, cudaStream_t st, Tracer *tr);

// ---- the tensor-core form (NHWC activations; the 3x3 layers run as
// stride-1 implicit GEMMs on the tensor cores, driven by the host planner)

struct UnetLayer {
  int kind;  // 0: 3x3 convolution, 1: 3x3 transposed convolution, 2: 1x1 head
  int cin, cout, bn;
  size_t src;  // first float of the layer in the packed parameters
  size_t dst;  // first float of its folded weights (bias after them)
};
// The layers in execution order: per encoder level two convolutions, per
// decoder level two transposed convolutions, the head.
std::vector<UnetLayer> unet_layer_table(const UnetShape &u);

// Whether the shape takes the tensor-core form: channel counts that are
// whole K blocks (base a multiple of 32; the input padded to 8 channels, or
// a multiple of 32) and maps whose 128-row tiles are boxes of whole rows of
// whole maps at every level.
bool unet_tc_shape_ok(const UnetShape &u, int H, int W);
// Stored channels of the staged NHWC input.
int unet_tc_in_channels(const UnetShape &u);
// Bytes of one layer's packed weight tiles (tf32 hi or lo part).
size_t unet_tc_pack_bytes(int cin_stored, int cout);

struct UnetTcBufs {
  float *fold = nullptr;              // conv-form folded weights: per 3x3 layer [cout][cin][3][3], bias
  uint8_t *B = nullptr, *B_lo = nullptr;  // packed weight tiles, hi / lo
  float *in = nullptr;                // NHWC input, unet_tc_in_channels channels
  float *enc_a[8] = {}, *enc[8] = {}, *pool[8] = {}, *up[8] = {}, *dec_a[8] = {}, *dec[8] = {};  // NHWC
};
size_t unet_tc_carve(const UnetShape &u, int N, int H, int W, char *base, UnetTcBufs *b);

// Batch normalisation folded into every layer, the 3x3 layers in
// convolution form (transposed ones turned by 180 degrees, channel axes
// swapped), into b.fold; one launch per layer.
cudaError_t unet_fold_conv_form(const UnetShape &u, const float *params, float *fold, cudaStream_t st, Tracer *tr);
// NCHW [N][cin][H][W] -> NHWC [N][H][W][cs] (channels cin.. zero).
cudaError_t launch_unet_stage_nhwc(const float *in, int N, int cin, long long hw, int cs, float *out,
                                   cudaStream_t st, Tracer *tr);
// 2x2 max pooling, NHWC [N][H][W][C] -> [N][H/2][W/2][C] (C a multiple of 4).
cudaError_t launch_unet_pool_nhwc(const float *x, int N, int H, int W, int C, float *y, cudaStream_t st, Tracer *tr);
// 2x bilinear upsampling (half-pixel centres, clamped), NHWC [N][h][w][C] -> [N][2h][2w][C].
cudaError_t launch_unet_up_nhwc(const float *x, int N, int h, int w, int C, float *y, cudaStream_t st, Tracer *tr);
// The 1x1 head with ReLU: NHWC [N][HW][C] -> NCHW [N][cout][HW], weights [cout][C] then the bias.
cudaError_t launch_unet_head_nhwc(const float *d, int N, long long hw, int C, const float *wh, int cout, float *out,
                                  cudaStream_t st, Tracer *tr);

}  // namespace drc
