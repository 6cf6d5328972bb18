// unet.cuh -- the paper's own network form (Sec. 3.3, "Neural network"): a
// U-Net of two 3x3 convolutions per stage with batch normalisation and
// LeakyReLU, 2x2 max pooling, 2x bilinear upsampling, concatenated skips and
// a 1x1 head with ReLU, in FP32 on the CUDA cores.
#pragma once
#include <cstddef>
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

}  // namespace drc
