// backward.cuh -- launchers of the backward-pass kernels that are not
// tensor-core convolutions (backward.cu).
#pragma once
#include <cuda_runtime.h>

namespace drc {

// L1 loss (added to *loss, nullable) and dL/dout as NHWC4 fp32 [N][H][W][4]
// (and, g8 nullable, as bf16 NHWC8) from out/target [N][3][H][W]; grad_out:
// target already is dL/dout.
cudaError_t launch_l1_grad(const float *out, const float *target, int N, int H, int W, bool grad_out, bool out_relu,
                           float *g4, void *g8, float *loss, cudaStream_t st);

// Head backward (data): gradient w.r.t. t_1 [N][Hh][Wh][C] from g4 and the
// head weights [C][3][3][3]; gt (nullable) unmasked, gz masked by mask > 0.
cudaError_t launch_head_bwd(const float *g4, const float *Whead, const void *mask, void *gt, void *gz, int N, int Hh,
                            int Wh, int C, bool bf16, int num_sms, cudaStream_t st);

// dW[m][q][3][3] = sum R[n,i,j,m] Q[n,2i+u-1,2j+v-1,q] (see backward.cu).
// part == nullptr: added to dW with fp32 atomics.  part given (the FP32
// path): compensated sums, split-K partials in part (wgrad_partial_elems
// float2), then a deterministic compensated reduction that OVERWRITES dW.
size_t wgrad_partial_elems(int N, int Hb, int Wb, int Mr, int Qc, int Qraw, int num_sms);
cudaError_t launch_wgrad(const void *R, bool r_bf16, const void *Q, bool q_bf16, int N, int Hb, int Wb, int Mr,
                         int Qc, int Qraw, float *dW, float2 *part, int num_sms, cudaStream_t st);

// Column sums of T [npix][C], c < Craw; C a multiple of 16 bytes' worth of
// elements (8 bf16 / 4 fp32).  part == nullptr: added to db with atomics;
// part given: compensated per-block pairs (colsum_partial_elems float2),
// then the compensated reduction, which OVERWRITES db.
size_t colsum_partial_elems(long long npix, int C, int Craw, bool bf16, int num_sms);
cudaError_t launch_colsum(const void *T, bool bf16, long long npix, int C, int Craw, float *db, float2 *part,
                          int num_sms, cudaStream_t st);

// NHWC16 input gradient -> [N][7][H][W], through the log encode if applied.
cudaError_t launch_dinput(const void *g16, bool bf16, const float *x_raw, long long hw, int N, bool encode,
                          float exposure, float *dinput, cudaStream_t st);

}  // namespace drc
