// head.cuh -- output layer of the autoencoder (3-channel transposed conv),
// fp32 FMA kernel with the fused decode and irradiance payload.
#pragma once
#include <cuda_runtime.h>

#include "pass.cuh"

namespace drc {

struct HeadArgs {
  const void *x;        // t_1, NHWC [N][Hh][Wh][C]: fp32, bf16, or e4m3 (value / in_scale[c])
  float *out;           // [N][3][2 Hh][2 Wh]
  float *payload;       // [N][3] accumulated E/pi, or nullptr
  const float *w;       // convT weights [C][3][3][3]
  const float *bias;    // [3]
  int N, Hh, Wh, C;
  int relu, decode;
  float inv_exposure;
  const PassSlot *slot; // nullable: out, payload, count (<= N) and decode flag from device memory
  const float *in_scale;  // e4m3 input: per-channel scales
  float band[256];      // payload weight of each output row
  int inline_w;         // wk holds the weights (C <= 64, C % 16 == 0)
  float wk[64 * 27];    // the weights again, read by the kernel as constant-bank operands
};

// prec: the activation precision of the context (0 fp32, 1 bf16, 2 e4m3).
cudaError_t launch_head(const HeadArgs &a, int prec, cudaStream_t st);

}  // namespace drc
