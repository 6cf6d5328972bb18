// mapgen.cuh -- the input maps of the denoiser traced on the GPU from cache
// points in an analytic interior (Sec. 3.1-3.3): radiance without the first
// hit's own emission, distance and normal per texel.
#pragma once
#include <cuda_runtime.h>

#include "drc.h"
#include "trace.cuh"

namespace drc {

struct MapGenArgs {
  drc_scene scene;
  int n, H, W, D;
  const float *pos, *nrm;   // [n][3]
  const float2 *u;          // [n][H][W][D] uniform pairs
  float *maps;              // [n][7][H][W]
};

cudaError_t launch_gen_maps(const MapGenArgs &a, cudaStream_t st, Tracer *tr = nullptr);

}  // namespace drc
