// indirect.cuh -- the indirect term of Eq. 3 by multiple importance sampling
// between the blended cached maps (as environment maps with perfect
// visibility) and a Lambertian BRDF (Sec. 3.2), composited with the
// emission and the direct term.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "trace.cuh"

namespace drc {

constexpr int kIndirectMaxRows = 256;  // map rows (polar bands) the launch parameters hold

struct IndirectArgs {
  int n, H, W;            // caches and their map size
  const float *maps;      // [n][3][H][W] linear radiance
  const float *cnrm;      // [n][3]
  long long P;
  int k, S;
  const int *nbr;         // [P][k] cache indices (-1: none)
  const float *nbr_w;     // [P][k] normalised weights (the map-choice probabilities)
  const float *gnrm;      // [P][3]
  const float *albedo;    // [P][3]
  const float4 *u;        // [P][S] uniforms in [0, 1)
  const float *emit;      // [P][3] or nullptr
  const float *direct;    // [P][3] or nullptr
  float *out;             // [P][3]
  // scratch: per map its luminance x solid-angle CDF over the texels (row
  // major, inclusive) and its frame (t, b, n; n.w = 0 for a zero normal)
  float *cdf;             // [n][H W]
  float4 *frame;          // [n][3]
  // per row a of the maps: cos(a pi / 2H) for a = 0..H, and the texel solid
  // angle of row a, (cos a - cos a+1)(2 pi / W), both from double on the host
  float rowcos[kIndirectMaxRows + 1];
  float omega[kIndirectMaxRows];
};

// Scratch bytes of the CDFs and frames for n maps of H x W.
size_t indirect_scratch_bytes(int n, int H, int W);
// Points a.cdf / a.frame into base (256-byte aligned).
void indirect_carve(IndirectArgs &a, void *base);
cudaError_t launch_indirect(const IndirectArgs &a, cudaStream_t st, Tracer *tr = nullptr);

}  // namespace drc
