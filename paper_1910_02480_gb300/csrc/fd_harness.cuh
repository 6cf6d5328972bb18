// fd_harness.cuh -- a test harness, not a hot path: the network's L1 loss in
// FP64 on the GPU, for central finite differences of drc_backward's gradient.
#pragma once
#include <cuda_runtime.h>

namespace drc {

struct FdLayer {
  int transposed;   // 0: 3x3 stride-2 conv; 1: 3x3 stride-2 transposed conv (padding 1, output padding 1)
  int Cin, Cout;    // weight channels (conv W [Cout][Cin][3][3], transposed W [Cin][Cout][3][3])
  size_t w_off, b_off;
};

// layers: the S encoder convs, then the S decoder transposed convs (the last
// one the head).  Loss (written to *loss) = mean over N 3 H W of |out - target|.
// Allocates and frees its own device scratch; synchronises `st`.
cudaError_t fd_loss64(const FdLayer *layers, int S, const double *w, const float *in, const float *target, int N,
                      int Cin0, int H, int W, bool encode, float exposure, bool out_relu, double *loss,
                      cudaStream_t st);

}  // namespace drc
