// wgrad_tc.cuh -- launcher of the tensor-core weight-gradient kernel
// (wgrad_tc.cu): BF16 activations, fp32 accumulation, split K with atomics.
#pragma once
#include <cuda.h>  // CUtensorMap (type only)
#include <cuda_runtime.h>

namespace drc {

struct WgradTcArgs {
  CUtensorMap mapR;  // R as a 2-D bf16 tensor [pixels][Mr], box {64, 64}, 128-byte swizzle
  CUtensorMap mapQ;  // Q as [N][2Hb][2Wb][Qc] bf16, box {64, 2 Wb, 2 rows, maps}, element strides {1, 2, 2, 1}
  float *dW;         // [Mr][Qraw][3][3] fp32, accumulated into
  int *status;       // latches ERR_TIMEOUT when a bounded wait gives up
  unsigned long long timeout_ns;
  int N, Hb, Wb, Mr, Qraw;
  int BNq;               // q columns per tile: 64 or 128
  int m_tiles, n_tiles;  // ceil(Mr / 128), Qc / BNq
  int total_kb, kb_per_split, ksplit;  // filled in by launch_wgrad_tc
};

// Whether the kernel takes this shape: Qc a multiple of 64, Mr of 128, and
// every 64-pixel K block made of whole rows (Wb | 64) of whole maps.
bool wgrad_tc_supported(int Hb, int Wb, int Mr, int Qc);

// Rows of Q's box (the K block's coarse rows per map) and maps per box.
void wgrad_tc_box(int Hb, int Wb, int *rows, int *maps);

// dW[m][q][u][v] += sum_{n,i,j} R[n,i,j,m] Q[n,2i+u-1,2j+v-1,q]; the maps in
// `a` are encoded by the caller.  Nothing is launched for N = 0.
cudaError_t launch_wgrad_tc(const WgradTcArgs &a, int num_sms, cudaStream_t st);

}  // namespace drc
