// conv_tc.cuh -- layer descriptions shared by the host planner and the
// tensor-core implicit-GEMM kernels of the autoencoder (Sec. 3.3).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace drc {

// How a GEMM row maps to pixels and how K maps to (tap, channel).
enum LayerKind {
  LK_CONV_NCHW7 = 0,  // first encoder layer: fp32 NCHW 7-channel input, K = c*9 + tap (63 -> pad)
  LK_CONV = 1,        // encoder conv3x3 s2 p1 on NHWC activations, K = tap*Cin + c
  LK_CONVT = 2,       // decoder convT3x3 s2, one GEMM per output parity phase
  LK_HEAD = 3         // output convT (3 channels): all four phases as 12 (->16) columns
};

enum Prec { PREC_TF32X3 = 0, PREC_BF16 = 1, PREC_FP8 = 2 };

constexpr int BM = 128;          // GEMM rows per tile (TMEM lanes)
constexpr int KROW_BYTES = 128;  // bytes of K per operand row per stage (one swizzle row)
constexpr int NUM_THREADS = 512; // 16 warps
constexpr int MMA_WARP = 0, BLOAD_WARP = 1, EPI_WARP0 = 4, PROD_WARP0 = 8;
constexpr int NUM_PROD_THREADS = 256;

struct PhaseDesc {
  int ntaps;         // taps feeding this phase
  int num_kb;        // K blocks (KROW_BYTES of K each)
  int oy, ox;        // output parity (LK_CONVT); 0 otherwise
  long long b_off;   // byte offset of this phase's packed B tiles
  signed char dy[9], dx[9];  // input pixel offset of each tap, from the row's base pixel
  signed char u[9], v[9];    // kernel tap (row, col) of each tap (weight packing)
};

struct ConvArgs {
  int kind;
  const void *x;     // input activations
  void *y;           // output activations (NHWC) or maps (NCHW, LK_HEAD)
  const void *skip;  // NHWC skip tensor shaped like y (LK_CONVT), or nullptr
  const uint8_t *B;  // packed B tiles (tf32 hi part for PREC_TF32X3)
  const uint8_t *B_lo;  // packed B tiles, tf32 lo part (PREC_TF32X3)
  const float *bias;    // [Cout] (LK_HEAD: [3])
  const float *bscale;  // FP8: per-output-column dequantisation scale, else nullptr
  float *payload;       // LK_HEAD: [N][3] accumulated E/pi, or nullptr
  int N, Hin, Win, Cin;  // input activation geometry (Cin = stored channels)
  int Hrow, Wrow;        // row grid per map
  int Hout, Wout, Cout;  // output geometry (Cout = stored channels; LK_HEAD: 3)
  int M;                 // N * Hrow * Wrow
  int BN, n_tiles, m_tiles, num_phases;
  int phase_order[4];    // heaviest phase first
  PhaseDesc ph[4];
  int relu;
  int encode;            // LK_CONV_NCHW7: log1p(s L) on channels 0..2
  int decode;            // LK_HEAD: write expm1(y)/s
  float exposure, inv_exposure;
  float act_scale_in;    // FP8: activations stored as value / scale
  float act_scale_out;
  float band[256];       // LK_HEAD: payload weight of each output row (1/pi factor folded)
  int *status;
  unsigned long long timeout_ns;
  int debug_stall;
};

// Host-side launch / pack entry points (conv_tc.cu).
cudaError_t launch_conv(const ConvArgs &a, int prec, int num_sms, cudaStream_t st);
__host__ __device__ int conv_stages(int prec, int BN);
size_t conv_smem_bytes(int prec, int BN);

struct PackArgs {
  int kind;
  const float *wraw;  // this layer's raw weights (start of W)
  int Cin, Cout;      // raw layer channels (LK_HEAD: Cout = 3)
  int BN, n_tiles, num_phases;
  PhaseDesc ph[4];
  uint8_t *B, *B_lo;  // packed outputs
  float *bscale;      // FP8: per-column scale out
  long long total_chunks;
};
cudaError_t launch_pack(const PackArgs &p, int prec, cudaStream_t st);

}  // namespace drc
