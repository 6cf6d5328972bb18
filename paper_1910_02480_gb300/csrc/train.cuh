// train.cuh -- the training-loop pieces of Sec. 4 (Implementation): map
// augmentation by rotation and flipping, and the Adam optimiser step.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "trace.cuh"

namespace drc {

// out[n] = the symmetry codes[n] (low three bits; r + 4 f: column mirror if
// f, then r counter-clockwise quarter turns) of the square map in[n], every
// channel alike.  in, out: [N][C][S][S] fp32, not overlapping.
cudaError_t launch_augment(const float *in, float *out, int N, int C, int S, const int *codes, cudaStream_t st,
                           Tracer *tr);

// One Adam step on n parameters in place; c1 = 1 / (1 - b1^t), c2 = 1 /
// sqrt(1 - b2^t) (the bias corrections, from the host).
cudaError_t launch_adam(float *w, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st, Tracer *tr);

}  // namespace drc
