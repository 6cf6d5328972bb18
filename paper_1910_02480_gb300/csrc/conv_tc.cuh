// conv_tc.cuh -- layer descriptions shared by the host planner and the
// tensor-core implicit-GEMM kernels of the autoencoder (Sec. 3.3).
#pragma once
#include <cstdint>
#include <cuda.h>  // CUtensorMap (type only; encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

#include "pass.cuh"

namespace drc {

// How a GEMM row maps to pixels and how K maps to (tap, channel).
enum LayerKind {
  LK_CONV = 1,   // encoder conv3x3 s2 p1 on NHWC activations, K = tap*Cin + c
  LK_CONVT = 2,  // decoder convT3x3 s2, one GEMM per output parity phase
  LK_HEAD = 3,   // output convT (3 channels): not a tensor-core GEMM (head.cu)
  LK_CONV1 = 4   // conv3x3 s1 p1 ("same") on NHWC activations, K = tap*Cin + c; the input may be the
                 // channel concatenation of two tensors (x: channels [0, C1), x2: the rest)
};

enum Prec { PREC_TF32X3 = 0, PREC_BF16 = 1, PREC_FP8 = 2 };

constexpr int BM = 128;          // GEMM rows per tile (TMEM lanes)
constexpr int KROW_BYTES = 128;  // bytes of K per operand row per stage (one swizzle row)
constexpr int NUM_THREADS = 512; // 16 warps
constexpr int MMA_WARP = 0, BLOAD_WARP = 1, TMA_ISSUE_WARP = 2, EPI_WARP0 = 4, PROD_WARP0 = 8;
constexpr int NUM_PROD_THREADS = 256;

struct PhaseDesc {
  int ntaps;         // taps feeding this phase
  int num_kb;        // K blocks (KROW_BYTES of K each)
  int oy, ox;        // output parity (LK_CONVT); 0 otherwise
  long long b_off;   // byte offset of this phase's packed B tiles
  signed char dy[9], dx[9];  // input pixel offset of each tap, from the row's base pixel
  signed char u[9], v[9];    // kernel tap (row, col) of each tap (weight packing); -1: none (pair)
  // LK_CONVT phase pair (pair = 1): columns [Cout, 2 Cout) of the GEMM are a
  // second output parity (oy2, ox2) with kernel taps (u2, v2) over the same
  // input taps (the union of the two phases' taps; -1 where that phase has
  // no weight for the tap)
  int pair, oy2, ox2;
  signed char u2[9], v2[9];
};
// drc_describe_layer / autotune codes of a decoder layer run as phase pairs:
// A in tensor memory (the default path), or in shared memory (TMA + producer
// conversion; the tensor memory then holds two accumulator buffers)
constexpr int A_PATH_PAIRED = 8;
constexpr int A_PATH_PAIRED_SMEM = 9;

// How the A operand reaches shared memory.
enum ProdMode {
  PROD_CPASYNC = 0,      // per-thread 16-byte cp.async gathers (any shape)
  PROD_TMA_CONVERT = 1,  // one TMA box per K block into a raw slot, converted by the producer warps
  PROD_TMA_DIRECT = 2,   // one TMA box per K block straight into the A tile (bf16)
  PROD_TMA_TMEM = 3      // split-tf32: TMA box into a raw slot, hi/lo written to tensor memory,
                         // MMAs read A from tensor memory (B only in shared memory)
};

struct ConvArgs {
  CUtensorMap tmap;  // A operand view for the TMA modes (64-byte aligned)
  CUtensorMap ymap;  // y_tma: the output for TMA stores, 64-byte swizzle, one box = 16 channels of one
                     // epilogue warp's 32 rows -- LK_CONV: 2-D [M][Cout], box {16, 32}; LK_CONVT: 4-D
                     // [N][Hout][Wout][Cout] with element strides {1, 2, 2, 1}, box {16, 2 Wrow, 2 rw, mw}
  int y_tma;         // FP32 without training outputs: tiles stored by TMA from shared memory
  int y_rw, y_mw;    // LK_CONVT: phase rows and maps per 32-row box (Wrow * y_rw * y_mw = 32)
  int hi_raw;        // set by launch_conv: split-tf32 with A in shared memory over whole K-block boxes in the
                     // decoder forms -- the MMAs read A_hi from the raw slot, the producers write only A_lo
  int skip_tma;      // y_tma FP32 decoder whose skip is its output (in place): the epilogue reads the
                     // skip boxes through ymap by TMA, into the staging boxes the stores then read
  int prod_mode;
  int tap_boxes;     // TMA modes, FP32 with 8 stored input channels (32 bytes per tap): one box per tap,
                     // four per K block, placed tap-major in the raw slot (BM rows x 32 bytes each)
  int kind;
  const void *x;     // input activations, NHWC
  const void *x2;    // LK_CONV1: second input (NHWC, Cin - C1 channels) concatenated after x, or nullptr
  int C1;            // LK_CONV1 with x2: channels of x (a multiple of the K block's channels)
  CUtensorMap tmap2; // LK_CONV1 with x2: A operand view of x2 (TMA modes)
  void *y;           // output activations, NHWC
  const void *skip;  // NHWC skip tensor shaped like y (LK_CONVT), or nullptr
  const uint8_t *B;  // packed B tiles (tf32 hi part for PREC_TF32X3)
  const uint8_t *B_lo;  // packed B tiles, tf32 lo part (PREC_TF32X3)
  const float *bias;    // [Cout]
  const float *bscale;  // FP8: per-output-column dequantisation scale, else nullptr
  int N, Hin, Win, Cin;  // input activation geometry (Cin = stored channels)
  int cin_shift;         // log2(Cin) when Cin is a power of two, else -1
  int Hrow, Wrow;        // row grid per map
  int Hout, Wout, Cout;  // output geometry (Cout = stored channels)
  int M;                 // N * Hrow * Wrow
  const int *count;      // nullable: maps of this launch in device memory (0..N); M, m_tiles then
                         // describe the N-map maximum the launch was sized for
  int BN, n_tiles, m_tiles, num_phases;
  int phase_order[4];    // heaviest phase first
  PhaseDesc ph[4];
  int relu;
  float slope;             // with relu: 0 = ReLU, else LeakyReLU max(z, slope z) (0 < slope < 1)
  const float *out_qinv;   // nullable: store the output as e4m3, column c times out_qinv[c] (the inverse
                           // of the consuming layer's input scale); else in the kernel's activation type
  const float *skip_scale; // FP8 kernel: the e4m3 skip tensor's per-channel scales
  unsigned *amax;          // nullable: per output column max |output| before quantisation (calibration)
  // Training: y2 (nullable, NHWC like y) receives the value before the skip
  // add (y2_pre_skip = 1: the decoder's ReLU output) or before the mask
  // (y2_pre_skip = 0: an unmasked gradient); mask (nullable, NHWC like y)
  // zeroes the output where mask <= 0 (the ReLU derivative).
  void *y2;
  int y2_pre_skip;
  const void *mask;
  // FP32 accumulation in chunks (0: off; PROD_TMA_TMEM, BN <= KFOLD_MAX_BN):
  // the MMAs of every kfold K blocks of a tile go into a fresh
  // tensor-memory accumulator -- per K block the two small correction
  // products first, then the main one -- which the epilogue warps add into
  // an fp32 running sum in tensor memory (round to nearest) while the next
  // chunk accumulates in the other buffer.  The tensor core's own fp32
  // accumulation does not round to nearest, so its error grows with the
  // number of MMAs into one accumulator; deep K (thousands of terms) needs
  // this to stay at fp32 accuracy.
  int kfold;
  // U-Net form with the whole output row in one tile (n_tiles 1) and TMA
  // stores: the network's 1x1 head fused into the epilogue -- out[n][o][pixel]
  // = ReLU(head_w[o] . y + head_b[o]) for o < head_cout (<= KHEAD_MAX), head_w
  // [head_cout][Cout] then head_b; y itself is not stored (nullptr: off)
  const float *head_w;
  float *head_out;  // [N][head_cout][Hout * Wout]
  int head_cout;
  int *status;
  unsigned long long timeout_ns;
  int debug_stall;
  unsigned long long *prof;  // optional [PROF_SLOTS] wait-time counters (clock64 cycles), or nullptr
};

// Diagnostic counters of one conv launch (summed over CTAs; per-warp values
// are taken from lane 0 of each warp of the role).
enum ProfSlot {
  PROF_MMA_WAIT_FULL = 0, PROF_MMA_WAIT_TEMPTY, PROF_MMA_TOTAL, PROF_BLOAD_WAIT_EMPTY,
  PROF_PROD_WAIT_EMPTY, PROF_PROD_WAIT_COPY, PROF_PROD_TOTAL, PROF_EPI_WAIT_TFULL, PROF_EPI_TOTAL,
  PROF_CTAS, PROF_PROD_CONVERT, PROF_PROD_FENCE, PROF_PROD_ISSUE, PROF_EPI_LD, PROF_SLOTS = 16
};

struct SmemPlan {
  int stages, raw_depth, raw_slot_bytes;
  int epi_stage;  // the epilogue's staging buffer (EPI_STG_BYTES after the raw ring) fits
};
// Epilogue staging: 4 warps x 32 rows x (16 + 4 pad) floats.
constexpr int EPI_STG_FLOATS = 4 * 32 * 20;
constexpr int EPI_STG_BYTES = EPI_STG_FLOATS * 4;
// Epilogue staging for TMA stores: per warp a ring of boxes of 32 rows x 16
// columns (2 KB fp32), so a box is rewritten only once the store that read
// it EPI_TMA_BOXES chunks earlier is done, not the store just issued.
constexpr int EPI_TMA_BOXES = 4;
constexpr int EPI_TMA_BOX_BYTES = 2048;
constexpr int EPI_TMA_BYTES = 4 * EPI_TMA_BOXES * EPI_TMA_BOX_BYTES;
// Accumulation chunks (ConvArgs::kfold): the running sum and two chunk
// accumulators in tensor memory next to the A stages.
constexpr int KFOLD_MAX_BN = 128;
constexpr int KHEAD_MAX = 4;  // head outputs the fused epilogue keeps in registers
__host__ __device__ SmemPlan smem_plan(int prec, int BN, int mode, int ytma, int fold = 0);
size_t conv_smem_bytes(int prec, int BN, int mode, int ytma, int fold = 0);

// Host-side launch / pack entry points (conv_tc.cu).
cudaError_t launch_conv(const ConvArgs &a, int prec, int num_sms, cudaStream_t st);

struct PackArgs {
  int kind;
  const float *wraw;  // this layer's raw weights (start of W)
  int Cin, Cout;      // GEMM channels: Cin as stored in the activations
  int Cin_raw;        // channels of the raw weights (Cin_raw <= Cin; the rest pack as 0)
  int Cout_raw;       // LK_CONVT: output channels of the raw weights (<= Cout; the rest pack as 0)
  int BN, n_tiles, num_phases;
  PhaseDesc ph[4];
  uint8_t *B, *B_lo;  // packed outputs
  float *bscale;      // FP8: per-column scale out (this layer's columns)
  const float *in_scale;  // FP8: per-input-channel activation scale folded into W (nullable = 1)
  long long total_chunks;
};
cudaError_t launch_pack(const PackArgs &p, int prec, cudaStream_t st);

// First-layer input: fp32 NCHW [N][7][H][W] -> NHWC with 8 channels (the 8th
// zero), fp32 or bf16, with the optional log1p(s L) of channels 0..2.
// slot (nullable): take the input, the count (<= N) and the encode flag from
// device memory, and clear the slot's payload.
cudaError_t launch_nchw7_to_nhwc8(const float *in, void *out, long long pixels_per_map, int N,
                                  bool bf16, bool encode, float exposure, cudaStream_t st,
                                  const PassSlot *slot = nullptr);

}  // namespace drc
