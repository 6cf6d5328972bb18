// wgrad_tc.cuh -- launcher of the tensor-core weight-gradient kernel
// (wgrad_tc.cu): BF16 activations, fp32 accumulation, split K with atomics.
#pragma once
#include <cuda.h>  // CUtensorMap (type only)
#include <cuda_runtime.h>

namespace drc {

// Forms of the kernel: none (the shape needs the CUDA-core kernel), wide (Q
// channels a multiple of 64, one GEMM per tap) or narrow (8 Q channels, the
// nine taps stacked into one GEMM).
enum { WGRAD_TC_NONE = 0, WGRAD_TC_WIDE = 1, WGRAD_TC_NARROW = 2 };

struct WgradTcArgs {
  CUtensorMap mapR;  // R as a 2-D bf16 tensor [pixels][Mr], box {64, 64}, 128-byte swizzle
  CUtensorMap mapQ;  // Q as [N][2Hb][2Wb][Qc] bf16, box {64 (wide) / 8 (narrow), 2 Wb, 2 rows, maps},
                     // element strides {1, 2, 2, 1}; 128-byte swizzle (wide) / none (narrow)
  float *dW;         // [Mr][Qraw][3][3] fp32, accumulated into
  int *status;       // latches ERR_TIMEOUT when a bounded wait gives up
  unsigned long long timeout_ns;
  int N, Hb, Wb, Mr, Qraw;
  int BN;                // GEMM N per tile: Q channels (wide: 64 or 128) / R channels (narrow: 64 .. 256)
  int m_tiles, n_tiles;  // wide: Mr / 128, Qc / BN; narrow: 1, Mr / BN
  int total_kb, kb_per_split, ksplit;  // filled in by launch_wgrad_tc
};

// Which form takes this shape: every 64-pixel K block must be whole rows
// (Wb | 64) of whole maps; wide needs Qc % 64 == 0 and Mr % 128 == 0,
// narrow Qc == 8 and Mr % 64 == 0.
int wgrad_tc_form(int Hb, int Wb, int Mr, int Qc);

// Rows of Q's box (the K block's coarse rows per map) and maps per box.
void wgrad_tc_box(int Hb, int Wb, int *rows, int *maps);

// dW[m][q][u][v] += sum_{n,i,j} R[n,i,j,m] Q[n,2i+u-1,2j+v-1,q]; the maps in
// `a` are encoded by the caller for `form`.  Nothing is launched for N = 0.
cudaError_t launch_wgrad_tc(const WgradTcArgs &a, int form, int num_sms, cudaStream_t st);

}  // namespace drc
