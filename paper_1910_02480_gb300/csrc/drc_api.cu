// drc_api.cu -- the C ABI of include/drc.h: context, argument checks,
// weight packing, workspace, and the per-layer launch sequence of the
// autoencoder (Sec. 3.3) and of the interpolation (Sec. 3.2).
#include <cuda_runtime.h>

#include <cerrno>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "backward.cuh"
#include "conv_tc.cuh"
#include "drc.h"
#include "fd_harness.cuh"
#include "head.cuh"
#include "drc_status.cuh"
#include "indirect.cuh"
#include "mapgen.cuh"
#include "persist.cuh"
#include "interp.cuh"
#include "trace.cuh"
#include "train.cuh"
#include "unet.cuh"
#include "wgrad_tc.cuh"

using namespace drc;

static_assert(ERR_TIMEOUT == DRC_ERR_TIMEOUT, "device status code mismatch");

namespace {

struct Layer {
  int kind;
  int Cin, Cout;       // GEMM channels (Cin as stored in the input activations; LK_HEAD: Cout = 3)
  int Cin_raw;         // channels of the raw weights (7 for the first layer, whose input is padded to 8)
  int Cout_raw;        // LK_CONVT read of conv weights (data gradient): their input channels; 0 = Cout
  size_t w_off, b_off; // offsets (floats) into the packed raw weights
  int BN, n_tiles, num_phases;
  PhaseDesc ph[4];
  int phase_order[4];
  size_t pack_off, pack_bytes;  // in the packed operand buffer(s)
  int prec;                     // kernel precision of this layer (FP8 contexts run the first layer in BF16)
  size_t sc_off;                // FP8: offset of this layer's input-channel scales (Cin floats) in the scale arrays
  size_t bs_off;                // FP8: offset of this layer's output-column scales (Cout floats)
  char name[24];                // kernel label for the launch tracer
};

}  // namespace

struct drc_ctx {
  drc_config cfg;
  int device = 0;
  int num_sms = 0;
  int prec = PREC_TF32X3;
  size_t n_floats = 0;
  std::vector<Layer> layers;  // conv_1..conv_S, convT_S..convT_2, head
  // per layer: the FP32 decoder layer as two GEMMs of phase pairs (kind 0:
  // none), its own packed operands; used where drc_autotune picks a
  // phase-pair path (A_PATH_PAIRED, A_PATH_PAIRED_SMEM)
  std::vector<Layer> players;
  uint8_t *d_ppack = nullptr, *d_ppack_lo = nullptr;
  size_t ppack_total = 0;
  std::vector<int> modes;     // per layer: A-operand path chosen by drc_autotune (-1 = default)
  std::vector<Layer> dlayers; // data-gradient GEMMs of conv_1..conv_S, convT_S..convT_2 (training)
  uint8_t *d_dpack = nullptr, *d_dpack_lo = nullptr;
  size_t dpack_total = 0;
  unsigned long long dpack_version = 0;  // weights_version the data-gradient operands were packed from
  void *d_train = nullptr;
  size_t train_bytes = 0;
  float *d_zero = nullptr;              // zero bias of the data-gradient GEMMs
  float *d_wraw = nullptr;
  uint8_t *d_pack = nullptr, *d_pack_lo = nullptr;
  float *d_bscale = nullptr;   // FP8: per-layer output-column dequantisation scales
  float *d_inscale = nullptr;  // FP8: per-layer input-channel scales (activation = value / scale)
  float *d_qinv = nullptr;     // FP8: their inverses (quantisation by the producing layer)
  unsigned *d_amax = nullptr;  // FP8 calibration: per-layer output-column max |value| (float bits)
  bool calibrating = false;
  size_t n_scales = 0, n_bscales = 0;
  std::vector<float> h_inscale;
  std::vector<float> h_headw;  // the head's weights on the host (launch parameters of the head kernel)
  bool headw_stale = false;    // weights were set from device memory since h_headw was filled
  size_t pack_total = 0;
  void *d_act = nullptr;
  size_t act_bytes = 0;
  void *d_iscratch = nullptr;
  size_t iscratch_bytes = 0;
  void *d_indscratch = nullptr;  // drc_indirect: per-map CDFs and frames
  size_t indscratch_bytes = 0;
  int *d_status = nullptr;
  unsigned long long *d_prof = nullptr;  // wait-time counters (DRC_PROFILE_WAITS)
  bool weights_set = false;
  unsigned long long weights_version = 0;  // bumped by every drc_set_weights (plans repack on change)
  unsigned long long timeout_ns = 0;
  Tracer tracer;
  std::string err;
  // drc_frame_host: device staging, its copy stream and the events that
  // order uploads, compute and reuse across calls
  float *d_fmaps = nullptr, *d_fout = nullptr, *d_fpay = nullptr, *d_fgpos = nullptr, *d_fgnrm = nullptr,
        *d_frgb = nullptr;
  size_t fmaps_n = 0, fgbuf_p = 0;
  cudaStream_t fcopy = nullptr;
  cudaEvent_t fev_maps = nullptr, fev_gbuf = nullptr, fev_maps_free = nullptr, fev_gbuf_free = nullptr;
  // device memory the context owns (ctx_malloc / ctx_free), under an
  // optional limit (drc_set_memory_limit; 0 = none)
  std::unordered_map<void *, size_t> allocs;
  size_t mem_used = 0, mem_limit = 0;
  size_t refused = 0;  // bytes of the last request the limit refused (0: the last failure was CUDA's)
};

namespace {

drc_status fail(drc_ctx *c, drc_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
drc_status fail(drc_ctx *c, drc_status s, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

drc_status cuda_fail(drc_ctx *c, cudaError_t e, const char *what) {
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation && c && c->refused) {
    const size_t r = c->refused;
    c->refused = 0;
    return fail(c, DRC_ERR_OOM, "%s: %zu bytes requested with %zu in use exceed the context's memory limit of %zu bytes",
                what, r, c->mem_used, c->mem_limit);
  }
  if (e == cudaErrorMemoryAllocation) return fail(c, DRC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(c, DRC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Device memory owned by the context: counted, and refused (as
// cudaErrorMemoryAllocation, before cudaMalloc is called) where it would take
// the context past its limit.
cudaError_t ctx_malloc_raw(drc_ctx *c, void **p, size_t bytes) {
  *p = nullptr;
  if (c->mem_limit && c->mem_used + bytes > c->mem_limit) {
    c->refused = bytes;
    return cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  c->allocs[*p] = bytes;
  c->mem_used += bytes;
  return cudaSuccess;
}
template <class T>
cudaError_t ctx_malloc(drc_ctx *c, T **p, size_t bytes) {
  void *v = nullptr;
  const cudaError_t e = ctx_malloc_raw(c, &v, bytes);
  *p = static_cast<T *>(v);
  return e;
}
void ctx_free(drc_ctx *c, void *p) {
  if (!p) return;
  auto it = c->allocs.find(p);
  if (it != c->allocs.end()) {
    c->mem_used -= it->second;
    c->allocs.erase(it);
  }
  cudaFree(p);
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
    cudaGetLastError();
  }
  return fn;
}

// Choose how layer `a` feeds its A operand.  The TMA modes need the 128
// rows of every tile to be a box of the activation tensor (whole output rows
// of whole maps) and a K block to stay inside one tap; everything else uses
// the cp.async gather.
// force_mode >= 0 asks for that mode where the layer allows it (autotuner).
// FP32 convs whose epilogue only stores (no skip, no training outputs, no
// quantisation) write each tile's rows -- contiguous NHWC pixels -- by TMA:
// the output as a 2-D tensor [M][Cout] with 16-column x 32-row boxes.
void plan_store(int prec, ConvArgs &a) {
  a.y_tma = 0;
  a.skip_tma = 0;
  if (a.y2 || a.mask || a.amax || a.BN % 16 || a.Cout % 8) return;
  // e4m3 outputs (FP8 contexts: quantised for the consuming layer) of the
  // encoder convs, from the BF16 first layer or an FP8 layer: 16-byte rows,
  // no swizzle
  const bool e4m3 = a.out_qinv != nullptr;
  if (e4m3 ? (prec == PREC_TF32X3 || a.kind != LK_CONV || (prec == PREC_FP8) != (a.bscale != nullptr))
           : (prec == PREC_FP8 || a.bscale))
    return;
  // fp32: 64-byte box rows, 64-byte swizzle; bf16: 32-byte rows, 32-byte swizzle
  const int eb = e4m3 ? 1 : (prec == PREC_TF32X3 ? 4 : 2);
  const CUtensorMapDataType dt = e4m3 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                      : (prec == PREC_TF32X3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                             : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  const CUtensorMapSwizzle sw = e4m3 ? CU_TENSOR_MAP_SWIZZLE_NONE
                                     : (prec == PREC_TF32X3 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
  if (a.kind != LK_CONVT && a.skip) return;
  // BF16 decoder phases keep the per-row epilogue (its skip prefetch two
  // chunks ahead measured faster there: d2 0.21 against 0.24 ms)
  if (prec == PREC_BF16 && a.kind == LK_CONVT) return;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return;
  CUresult r;
  if (a.kind == LK_CONV || a.kind == LK_CONV1) {
    cuuint64_t dims[2] = {(cuuint64_t)a.Cout, (cuuint64_t)a.M};
    cuuint64_t strides[1] = {(cuuint64_t)a.Cout * eb};
    cuuint32_t box[2] = {16, 32}, estr[2] = {1, 1};
    r = enc(&a.ymap, dt, 2, a.y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else if (a.kind == LK_CONVT) {
    // a warp's 32 rows must be whole phase rows of whole maps
    const int Wr = a.Wrow, Hr = a.Hrow;
    if (Wr > 32 || 32 % Wr) return;
    const int rw = Hr < 32 / Wr ? Hr : 32 / Wr;
    if (rw < Hr ? Hr % rw != 0 : (32 / Wr) % Hr != 0) return;
    const int mw = 32 / (Wr * rw);
    a.y_rw = rw;
    a.y_mw = mw;
    cuuint64_t dims[4] = {(cuuint64_t)a.Cout, (cuuint64_t)a.Wout, (cuuint64_t)a.Hout, (cuuint64_t)a.N};
    cuuint64_t strides[3] = {(cuuint64_t)a.Cout * eb, (cuuint64_t)a.Cout * eb * a.Wout,
                             (cuuint64_t)a.Cout * eb * a.Wout * a.Hout};
    cuuint32_t box[4] = {16, (cuuint32_t)(2 * Wr), (cuuint32_t)(2 * rw), (cuuint32_t)mw}, estr[4] = {1, 2, 2, 1};
    r = enc(&a.ymap, dt, 4, a.y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    return;
  }
  if (r == CUDA_SUCCESS) {
    a.y_tma = 1;
    a.skip_tma = a.kind == LK_CONVT && prec == PREC_TF32X3 && a.skip && a.skip == a.y && !a.skip_scale;
  }
}

void plan_operand(int prec, ConvArgs &a, int force_mode = -1) {
  plan_store(prec, a);
  a.prod_mode = PROD_CPASYNC;
  a.tap_boxes = 0;
  const int bke = KROW_BYTES / (prec == PREC_TF32X3 ? 4 : (prec == PREC_BF16 ? 2 : 1));  // K elements per block
  const int Wr = a.Wrow, Hr = a.Hrow;
  // conv over 8 stored channels (the first layer): 32 bytes per tap in FP32
  // (four taps per K block) or 16 in BF16 (eight), each tap its own TMA box;
  // BF16 boxes land in the A tile directly (no-swizzle K-major layout).  FP8
  // conv over 64 channels: 64-byte taps, two per K block, 64-byte swizzle,
  // straight into the A tile.
  const bool conv = (a.kind == LK_CONV || a.kind == LK_CONV1) && !a.x2;
  const bool taps8 = conv && prec == PREC_FP8 && a.Cin == 64;  // the kernel's FP8 tap width
  const bool taps = (conv && a.Cin == 8 && (prec == PREC_TF32X3 || prec == PREC_BF16)) || taps8;
  if (Wr > BM || BM % Wr || (!taps && a.Cin % bke)) return;
  // a concatenated second input: every K block inside one of the two tensors
  const int C1 = a.x2 ? a.C1 : a.Cin;
  if (a.x2 && (a.kind != LK_CONV1 || C1 <= 0 || C1 >= a.Cin || C1 % bke)) return;
  const int rows_t = Hr < BM / Wr ? Hr : BM / Wr;
  if ((rows_t * Wr) % Wr || BM % (rows_t * Wr) || (rows_t < Hr && Hr % rows_t)) return;
  const int maps_t = BM / (rows_t * Wr);
  const bool s2 = a.kind == LK_CONV;
  if (s2 && 2 * Wr > 256) return;
  if (2 * rows_t > 256 || maps_t > 256) return;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return;
  const int eb = prec == PREC_TF32X3 ? 4 : (prec == PREC_BF16 ? 2 : 1);  // stored activation bytes
  const int box_c = taps ? a.Cin : KROW_BYTES / eb;                      // channels per box row (128 / 32 bytes)
  cuuint64_t dims[4] = {(cuuint64_t)C1, (cuuint64_t)a.Win, (cuuint64_t)a.Hin, (cuuint64_t)a.N};
  cuuint64_t strides[3] = {(cuuint64_t)C1 * eb, (cuuint64_t)C1 * eb * a.Win, (cuuint64_t)C1 * eb * a.Win * a.Hin};
  cuuint32_t box[4] = {(cuuint32_t)box_c, (cuuint32_t)(s2 ? 2 * Wr : Wr), (cuuint32_t)(s2 ? 2 * rows_t : rows_t),
                       (cuuint32_t)maps_t};
  cuuint32_t estr[4] = {1, (cuuint32_t)(s2 ? 2 : 1), (cuuint32_t)(s2 ? 2 : 1), 1};
  const CUtensorMapDataType dt = prec == PREC_TF32X3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                : (prec == PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8);
  CUresult r = enc(&a.tmap, dt,
                   4, const_cast<void *>(a.x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   taps8 ? CU_TENSOR_MAP_SWIZZLE_64B : (taps ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B),
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return;
  if (a.x2) {
    const int C2 = a.Cin - C1;
    dims[0] = (cuuint64_t)C2;
    strides[0] = (cuuint64_t)C2 * eb;
    strides[1] = strides[0] * a.Win;
    strides[2] = strides[1] * a.Hin;
    r = enc(&a.tmap2, dt, 4, const_cast<void *>(a.x2), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return;
  }
  if (force_mode == PROD_CPASYNC) return;
  a.tap_boxes = taps ? 1 : 0;
  if (prec == PREC_TF32X3 && force_mode == PROD_TMA_CONVERT) {
    a.prod_mode = PROD_TMA_CONVERT;
    return;
  }
  if (prec == PREC_BF16 || prec == PREC_FP8)
    a.prod_mode = PROD_TMA_DIRECT;
  else if (prec == PREC_TF32X3 && a.BN <= 128)
    a.prod_mode = PROD_TMA_TMEM;  // A operand in tensor memory
  else
    a.prod_mode = PROD_TMA_CONVERT;
}

int bke_of(int prec) { return KROW_BYTES / (prec == PREC_TF32X3 ? 4 : (prec == PREC_BF16 ? 2 : 1)); }
int elem_act(int prec) { return prec == PREC_TF32X3 ? 4 : 2; }
// Bytes per element of stored activation s (0 = the first layer's NHWC8
// input, s >= 1 = e_s): FP8 contexts keep the input in bf16 and store e4m3.
int elem_store(int prec, int s) { return prec == PREC_FP8 ? (s == 0 ? 2 : 1) : elem_act(prec); }

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

int pick_bn(int Cout) {
  if (Cout <= 256) return Cout;
  for (int bn = 256; bn >= 16; bn -= 16)
    if (Cout % bn == 0) return bn;
  return 16;
}

// Decoder phase (oy, ox): output pixel (2a+oy, 2b+ox) gathers input
// (a+di, b+dj) through kernel tap (u, v) with 2(a+di) + u - 1 = 2a + oy.
void convT_phase(PhaseDesc &pd, int oy, int ox, int Cin, int bke) {
  struct RT {
    int u, d;
  };
  RT rows[2], cols[2];
  int nr = 0, nc = 0;
  if (oy == 0) {
    rows[nr++] = {1, 0};
  } else {
    rows[nr++] = {0, 1};
    rows[nr++] = {2, 0};
  }
  if (ox == 0) {
    cols[nc++] = {1, 0};
  } else {
    cols[nc++] = {0, 1};
    cols[nc++] = {2, 0};
  }
  memset(&pd, 0, sizeof pd);
  pd.oy = oy;
  pd.ox = ox;
  pd.ntaps = nr * nc;
  for (int r = 0; r < nr; ++r)
    for (int c = 0; c < nc; ++c) {
      const int t = r * nc + c;
      pd.u[t] = (signed char)rows[r].u;
      pd.v[t] = (signed char)cols[c].u;
      pd.dy[t] = (signed char)rows[r].d;
      pd.dx[t] = (signed char)cols[c].d;
    }
  pd.num_kb = ceil_div((long long)pd.ntaps * Cin, bke);
}

// Offsets of every layer's packed B tiles ([phase][n_tile][k_block][BN rows
// x 128 B]) in one buffer; returns its size.
size_t layout_packs(std::vector<Layer> &Ls) {
  size_t pack = 0;
  for (Layer &L : Ls) {
    L.pack_off = pack;
    size_t bytes = 0;
    for (int p = 0; p < L.num_phases; ++p) {
      L.ph[p].b_off = (long long)(pack + bytes);
      bytes += (size_t)L.n_tiles * L.ph[p].num_kb * L.BN * KROW_BYTES;
    }
    L.pack_bytes = bytes;
    pack += (bytes + 255) & ~(size_t)255;
  }
  return pack;
}

void set_bn(Layer &L, int BN) {
  L.BN = BN;
  L.n_tiles = L.Cout / BN;
}

// Lay out every layer's GEMM(s) and the packed operand buffer.
void plan_layers(drc_ctx *c) {
  const drc_config &g = c->cfg;
  const int S = g.num_stages;
  std::vector<int> wd(S + 1);
  wd[0] = g.in_channels;
  for (int s = 1; s <= S; ++s) wd[s] = g.widths[s - 1];
  c->layers.clear();
  size_t off = 0, sc = 0, bs = 0;
  auto finish = [&](Layer &L) {
    // heaviest phase first
    for (int p = 0; p < 4; ++p) L.phase_order[p] = p < L.num_phases ? p : 0;
    for (int a = 0; a < L.num_phases; ++a)
      for (int b = a + 1; b < L.num_phases; ++b)
        if (L.ph[L.phase_order[b]].num_kb > L.ph[L.phase_order[a]].num_kb) {
          int t = L.phase_order[a];
          L.phase_order[a] = L.phase_order[b];
          L.phase_order[b] = t;
        }
    c->layers.push_back(L);
  };
  for (int s = 1; s <= S; ++s) {
    Layer L;
    memset(&L, 0, sizeof L);
    L.kind = LK_CONV;
    L.prec = (c->prec == PREC_FP8 && s == 1) ? PREC_BF16 : c->prec;
    snprintf(L.name, sizeof L.name, "conv e%d", s);
    L.Cin_raw = wd[s - 1];
    L.Cin = s == 1 ? 8 : wd[s - 1];  // the 7-channel input is staged as NHWC with 8 channels
    L.Cout = wd[s];
    L.w_off = off;
    off += 9ull * L.Cin_raw * L.Cout;
    L.b_off = off;
    off += L.Cout;
    set_bn(L, pick_bn(L.Cout));
    L.num_phases = 1;
    PhaseDesc &pd = L.ph[0];
    pd.ntaps = 9;
    for (int t = 0; t < 9; ++t) {
      pd.u[t] = pd.dy[t] = (signed char)(t / 3);
      pd.v[t] = pd.dx[t] = (signed char)(t % 3);
    }
    pd.num_kb = ceil_div(9ll * L.Cin, bke_of(L.prec));
    L.sc_off = sc;
    sc += L.Cin;
    L.bs_off = bs;
    bs += L.Cout;
    finish(L);
  }
  for (int s = S; s >= 1; --s) {
    Layer L;
    memset(&L, 0, sizeof L);
    L.Cin = L.Cin_raw = wd[s];
    L.Cout = s == 1 ? g.out_channels : wd[s - 1];
    L.prec = c->prec;
    L.sc_off = sc;
    sc += L.Cin;
    L.bs_off = bs;
    bs += L.Cout;
    L.w_off = off;
    off += 9ull * L.Cin * L.Cout;
    L.b_off = off;
    off += L.Cout;
    if (s == 1) {
      L.kind = LK_HEAD;  // fp32 FMA kernel (head.cu), no packed operands
      L.num_phases = 0;
      snprintf(L.name, sizeof L.name, "head");
    } else {
      L.kind = LK_CONVT;
      snprintf(L.name, sizeof L.name, "convT d%d", s);
      set_bn(L, pick_bn(L.Cout));
      L.num_phases = 4;
      for (int p = 0; p < 4; ++p) convT_phase(L.ph[p], p >> 1, p & 1, L.Cin, bke_of(L.prec));
    }
    finish(L);
  }
  c->pack_total = layout_packs(c->layers);
  // FP32 decoder layers whose two phases of one output row fit a 128-column
  // tile: phases (0,0)+(0,1) over their two input taps, (1,0)+(1,1) over four
  c->players.assign(c->layers.size(), Layer());
  for (size_t li = 0; li < c->layers.size(); ++li) {
    const Layer &L = c->layers[li];
    if (L.kind != LK_CONVT || L.prec != PREC_TF32X3 || 2 * L.Cout > 128 || L.Cout % 16) continue;
    Layer P = L;
    snprintf(P.name, sizeof P.name, "%s", L.name);
    set_bn(P, 2 * L.Cout);
    P.n_tiles = 1;
    P.num_phases = 2;
    for (int q = 0; q < 2; ++q) {
      const PhaseDesc &lo = L.ph[2 * q], &hi = L.ph[2 * q + 1];  // (q, 0) and (q, 1)
      PhaseDesc pd;
      memset(&pd, 0, sizeof pd);
      pd.pair = 1;
      pd.oy = lo.oy;
      pd.ox = lo.ox;
      pd.oy2 = hi.oy;
      pd.ox2 = hi.ox;
      for (int t = 0; t < hi.ntaps; ++t) {  // the second phase's taps hold the first's
        pd.dy[t] = hi.dy[t];
        pd.dx[t] = hi.dx[t];
        pd.u2[t] = hi.u[t];
        pd.v2[t] = hi.v[t];
        pd.u[t] = pd.v[t] = -1;
        for (int s = 0; s < lo.ntaps; ++s)
          if (lo.dy[s] == hi.dy[t] && lo.dx[s] == hi.dx[t]) {
            pd.u[t] = lo.u[s];
            pd.v[t] = lo.v[s];
          }
      }
      pd.ntaps = hi.ntaps;
      pd.num_kb = ceil_div((long long)pd.ntaps * L.Cin, bke_of(L.prec));
      P.ph[q] = pd;
    }
    P.phase_order[0] = 1;  // four taps first
    P.phase_order[1] = 0;
    c->players[li] = P;
  }
  c->ppack_total = layout_packs(c->players);
  c->n_scales = sc;
  c->n_bscales = bs;
}

drc_status check_config(const drc_config *g, drc_ctx *c) {
  if (!g) return fail(c, DRC_ERR_INVALID_ARG, "config is NULL");
  if (g->in_channels != 7) return fail(c, DRC_ERR_INVALID_ARG, "in_channels must be 7 (got %d)", g->in_channels);
  if (g->out_channels != 3) return fail(c, DRC_ERR_INVALID_ARG, "out_channels must be 3 (got %d)", g->out_channels);
  if (g->num_stages < 1 || g->num_stages > 6)
    return fail(c, DRC_ERR_INVALID_ARG, "num_stages must be 1..6 (got %d)", g->num_stages);
  for (int s = 0; s < g->num_stages; ++s)
    if (g->widths[s] < 16 || g->widths[s] > 1024 || g->widths[s] % 16)
      return fail(c, DRC_ERR_INVALID_ARG, "widths[%d] = %d: must be a multiple of 16 in 16..1024", s, g->widths[s]);
  if (g->precision < DRC_PREC_FP32 || g->precision > DRC_PREC_FP8_E4M3)
    return fail(c, DRC_ERR_INVALID_ARG, "unknown precision %d", (int)g->precision);
  if (!(g->exposure > 0.f) || !std::isfinite(g->exposure))
    return fail(c, DRC_ERR_INVALID_ARG, "exposure must be finite and > 0");
  if (g->wait_timeout_ms < 0) return fail(c, DRC_ERR_INVALID_ARG, "wait_timeout_ms must be >= 0");
  return DRC_OK;
}

size_t weight_count(const drc_config *g) {
  size_t n = 0;
  int prev = g->in_channels;
  for (int s = 0; s < g->num_stages; ++s) {
    n += 9ull * prev * g->widths[s] + g->widths[s];
    prev = g->widths[s];
  }
  for (int s = g->num_stages - 1; s >= 0; --s) {
    const int co = s == 0 ? g->out_channels : g->widths[s - 1];
    n += 9ull * g->widths[s] * co + co;
  }
  return n;
}

bool is_device_ptr(const void *p, int device) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice) return at.device == device;
  return at.type == cudaMemoryTypeManaged;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

drc_status check_dev(drc_ctx *c, const void *p, const char *name, bool nullable) {
  if (!p) return nullable ? DRC_OK : fail(c, DRC_ERR_INVALID_ARG, "%s is NULL", name);
  if (!aligned16(p)) return fail(c, DRC_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
  if (!is_device_ptr(p, c->device))
    return fail(c, DRC_ERR_INVALID_ARG, "%s is not device memory on device %d", name, c->device);
  return DRC_OK;
}

drc_status pack_layers(drc_ctx *c, const std::vector<Layer> &Ls, uint8_t *B, uint8_t *B_lo, cudaStream_t st) {
  for (const Layer &L : Ls) {
    if (L.kind == LK_HEAD) continue;
    PackArgs p;
    memset(&p, 0, sizeof p);
    p.kind = L.kind;
    p.wraw = c->d_wraw + L.w_off;
    p.Cin = L.Cin;
    p.Cin_raw = L.Cin_raw;
    p.Cout_raw = L.Cout_raw;
    p.Cout = L.Cout;
    p.BN = L.BN;
    p.n_tiles = L.n_tiles;
    p.num_phases = L.num_phases;
    for (int i = 0; i < 4; ++i) p.ph[i] = L.ph[i];
    p.B = B;
    p.B_lo = B_lo;
    if (L.prec == PREC_FP8) {
      p.bscale = c->d_bscale + L.bs_off;
      p.in_scale = c->d_inscale + L.sc_off;
    }
    p.total_chunks = (long long)(L.pack_bytes / 16);
    cudaError_t e;
    DRC_TRACED(&c->tracer, "weight pack", st, e = launch_pack(p, L.prec, st));
    if (L.prec == PREC_FP8) c->tracer.add_launches(1);  // the column-scale kernel before it
    if (e != cudaSuccess) return cuda_fail(c, e, "weight packing");
  }
  return DRC_OK;
}

drc_status pack_all(drc_ctx *c, cudaStream_t st) {
  drc_status s = pack_layers(c, c->layers, c->d_pack, c->d_pack_lo, st);
  if (s == DRC_OK && c->ppack_total) {
    std::vector<Layer> pl;
    for (const Layer &P : c->players)
      if (P.kind == LK_CONVT) pl.push_back(P);
    s = pack_layers(c, pl, c->d_ppack, c->d_ppack_lo, st);
  }
  return s;
}

size_t act_bytes_for(const drc_ctx *c, long long N, int H, int W) {
  // the first layer's NHWC input (8 channels), then e_1 .. e_S
  size_t b = (((size_t)N * H * W * 8 * elem_store(c->prec, 0)) + 255) & ~(size_t)255;
  for (int s = 1; s <= c->cfg.num_stages; ++s)
    b += (((size_t)N * (H >> s) * (W >> s) * c->cfg.widths[s - 1] * elem_store(c->prec, s)) + 255) &
         ~(size_t)255;
  return b;
}

drc_status ensure_act(drc_ctx *c, long long N, int H, int W) {
  const size_t need = act_bytes_for(c, N, H, W);
  if (need <= c->act_bytes) return DRC_OK;
  if (c->d_act) ctx_free(c, c->d_act);
  c->d_act = nullptr;
  c->act_bytes = 0;
  cudaError_t e = ctx_malloc(c, &c->d_act, need);
  if (e != cudaSuccess) return cuda_fail(c, e, "activation workspace");
  c->act_bytes = need;
  return DRC_OK;
}

void fill_common(const drc_ctx *c, const Layer &L, const uint8_t *B, const uint8_t *B_lo, ConvArgs &a) {
  memset(&a, 0, sizeof a);
  a.kind = L.kind;
  a.B = B;
  a.B_lo = B_lo;
  a.bias = c->d_wraw + L.b_off;
  a.BN = L.BN;
  a.n_tiles = L.n_tiles;
  a.num_phases = L.num_phases;
  for (int i = 0; i < 4; ++i) {
    a.ph[i] = L.ph[i];
    a.phase_order[i] = L.phase_order[i];
  }
  a.cin_shift = -1;
  for (int sh = 0; sh < 16; ++sh)
    if ((1 << sh) == L.Cin) a.cin_shift = sh;
  a.status = c->d_status;
  a.timeout_ns = c->timeout_ns;
}

// The head kernel takes weights of up to 64 input channels in its launch
// parameters (constant-bank operands).  Without a current host copy (weights
// set from device memory) it stages them from device memory instead.
void head_inline_weights(const drc_ctx *c, HeadArgs &h) {
  if (h.C <= 64 && h.C % 16 == 0 && c->h_headw.size() == (size_t)h.C * 27) {
    memcpy(h.wk, c->h_headw.data(), c->h_headw.size() * sizeof(float));
    h.inline_w = 1;
  }
}

// Inference calls bring the host copy of the head's weights up to date after
// weights were set from device memory: one synchronisation of `st` per
// weight update, not per call.  Never called inside a stream capture.
drc_status refresh_head_weights(drc_ctx *c, cudaStream_t st);

// Activation buffers and geometry of one launch sequence of the network over
// N maps of H x W (for a plan, N is the class's maximum and the real count is
// read from device memory).
struct Chain {
  int N = 0, H = 0, W = 0;
  uint8_t *in8 = nullptr;       // first layer's NHWC8 input
  std::vector<uint8_t *> act;   // act[s] = e_s, s = 1..S (decoder outputs overwrite in place)
  const int *count = nullptr;   // nullable: device map count (<= N)
  const PassSlot *slot = nullptr;
};

void carve_chain(const drc_ctx *c, void *base, int N, int H, int W, Chain &ch) {
  const int S = c->cfg.num_stages;
  ch.N = N;
  ch.H = H;
  ch.W = W;
  ch.in8 = static_cast<uint8_t *>(base);
  ch.act.assign(S + 1, nullptr);
  size_t off = (((size_t)N * H * W * 8 * elem_store(c->prec, 0)) + 255) & ~(size_t)255;
  for (int s2 = 1; s2 <= S; ++s2) {
    ch.act[s2] = static_cast<uint8_t *>(base) + off;
    off += (((size_t)N * (H >> s2) * (W >> s2) * c->cfg.widths[s2 - 1] * elem_store(c->prec, s2)) + 255) &
           ~(size_t)255;
  }
}

// ConvArgs of tensor-core layer li (encoder conv or decoder convT) of a chain.
// Ls: the chain's layer table (L = Ls[li] or a retiled copy of it).
// FP8 contexts: the output is quantised with the input scales of the layer
// that consumes it (layer li + 1 in the table's order e_1..e_S, d_S..d_2,
// head) and a decoder's skip e_{s-1} is dequantised with the input scales of
// e_s, the layer that consumed it.
void conv_args_for(const drc_ctx *c, const std::vector<Layer> &Ls, const Layer &L, size_t li, const Chain &ch,
                   const uint8_t *B, const uint8_t *B_lo, int force_mode, ConvArgs &a) {
  const int S = c->cfg.num_stages;
  const int H = ch.H, W = ch.W;
  fill_common(c, L, B, B_lo, a);
  a.N = ch.N;
  if (L.kind == LK_CONV) {
    const int s2 = (int)li + 1;  // encoder stage
    a.x = s2 == 1 ? static_cast<const void *>(ch.in8) : ch.act[s2 - 1];
    a.y = ch.act[s2];
    a.Hin = H >> (s2 - 1);
    a.Win = W >> (s2 - 1);
    a.Cin = L.Cin;
    a.Hrow = a.Hout = H >> s2;
    a.Wrow = a.Wout = W >> s2;
    a.Cout = L.Cout;
  } else {
    const int s2 = S - ((int)li - S);  // decoder stage S..2
    a.x = ch.act[s2];
    a.y = ch.act[s2 - 1];
    a.skip = ch.act[s2 - 1];
    a.Hin = a.Hrow = H >> s2;
    a.Win = a.Wrow = W >> s2;
    a.Cin = L.Cin;
    a.Hout = H >> (s2 - 1);
    a.Wout = W >> (s2 - 1);
    a.Cout = L.Cout;
  }
  a.relu = 1;
  a.M = (int)((long long)ch.N * a.Hrow * a.Wrow);
  a.m_tiles = ceil_div(a.M, BM);
  a.count = ch.count;
  if (c->prec == PREC_FP8) {
    if (L.prec == PREC_FP8) a.bscale = c->d_bscale + L.bs_off;
    a.out_qinv = c->d_qinv + Ls[li + 1].sc_off;
    if (L.kind == LK_CONVT) {
      const int s2 = S - ((int)li - S);
      a.skip_scale = c->d_inscale + Ls[s2 - 1].sc_off;
    }
    if (c->calibrating) a.amax = c->d_amax + L.bs_off;
  }
  plan_operand(L.prec, a, force_mode);
}

bool is_paired(int mode) { return mode == A_PATH_PAIRED || mode == A_PATH_PAIRED_SMEM; }

// ConvArgs of decoder layer li of the context's own table as its two GEMMs of
// phase pairs (mode A_PATH_PAIRED or A_PATH_PAIRED_SMEM); false where the
// layer has no paired form or its output tiles do not fit the TMA-store
// epilogue the pairs need.
bool paired_args(const drc_ctx *c, size_t li, const Chain &ch, int mode, ConvArgs &a) {
  if (li >= c->players.size() || c->players[li].kind != LK_CONVT || !is_paired(mode)) return false;
  const bool smem = mode == A_PATH_PAIRED_SMEM;
  conv_args_for(c, c->layers, c->players[li], li, ch, c->d_ppack, c->d_ppack_lo, smem ? PROD_TMA_CONVERT : -1, a);
  return a.y_tma && a.prod_mode == (smem ? PROD_TMA_CONVERT : PROD_TMA_TMEM);
}

// Enqueue the whole network over one chain: input staging, S encoder convs,
// S-1 decoder convTs, the head.  tr: launch tracer (nullptr while capturing a
// graph); prof: wait-time counters per layer, or nullptr.
drc_status run_chain(drc_ctx *c, const std::vector<Layer> &layers, const uint8_t *B, const uint8_t *B_lo,
                     const std::vector<int> *modes, const Chain &ch, const float *in, float *out, float *payload,
                     unsigned flags, cudaStream_t st, Tracer *tr, unsigned long long *prof) {
  cudaError_t e;
  DRC_TRACED(tr, "stage input", st,
             e = launch_nchw7_to_nhwc8(in, ch.in8, (long long)ch.H * ch.W, ch.N, c->prec != PREC_TF32X3,
                                       (flags & DRC_F_ENCODE_INPUT) != 0, c->cfg.exposure, st, ch.slot));
  if (e != cudaSuccess) return cuda_fail(c, e, "input staging");
  const int debug_stall = (flags & DRC_F_DEBUG_STALL) ? 1 : 0;
  for (size_t li = 0; li < layers.size(); ++li) {
    const Layer &L = layers[li];
    if (L.kind == LK_HEAD) {  // 3-channel transposed conv + decode + payload (head.cu)
      HeadArgs h;
      memset(&h, 0, sizeof h);
      h.x = ch.act[1];
      h.out = out;
      h.payload = payload;
      h.w = c->d_wraw + L.w_off;
      h.bias = c->d_wraw + L.b_off;
      h.N = ch.N;
      h.Hh = ch.H >> 1;
      h.Wh = ch.W >> 1;
      h.C = L.Cin;
      h.relu = c->cfg.out_relu ? 1 : 0;
      h.decode = (flags & DRC_F_DECODE_OUTPUT) ? 1 : 0;
      h.inv_exposure = 1.0f / c->cfg.exposure;
      h.slot = ch.slot;
      if (c->prec == PREC_FP8) h.in_scale = c->d_inscale + L.sc_off;
      head_inline_weights(c, h);
      if (payload || ch.slot) {
        const double pi = 3.14159265358979323846;
        for (int i = 0; i < ch.H; ++i) {
          const double t0 = i * pi / (2.0 * ch.H), t1 = (i + 1) * pi / (2.0 * ch.H);
          h.band[i] = (float)((std::sin(t1) * std::sin(t1) - std::sin(t0) * std::sin(t0)) / ch.W);
        }
      }
      DRC_TRACED(tr, L.name, st, e = launch_head(h, c->prec, st));
      if (e != cudaSuccess) return cuda_fail(c, e, "head launch");
      continue;
    }
    ConvArgs a;
    // phase-pair paths: the context's own layers only (plans keep their tiles)
    const bool paired = modes && &layers == &c->layers && paired_args(c, li, ch, (*modes)[li], a);
    if (!paired) conv_args_for(c, layers, L, li, ch, B, B_lo, modes ? (*modes)[li] : -1, a);
    a.debug_stall = debug_stall && li == 0;
    if (prof) a.prof = prof + li * PROF_SLOTS;
    DRC_TRACED(tr, L.name, st, e = launch_conv(a, L.prec, c->num_sms, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "layer launch");
  }
  return DRC_OK;
}

// ------------------------------------------------------------------ plans

constexpr int kMaxClasses = 8;

struct SlotUpdate {
  int n;
  unsigned flags;
  int max_maps[kMaxClasses];
  const float *in[kMaxClasses];
  float *out[kMaxClasses];
  float *payload[kMaxClasses];
};

// Write this pass's counts (from the caller's device array) and buffers into
// the plan's slots; a count outside 0..max_maps is clamped and latched as
// DRC_ERR_INVALID_ARG in the context status.
__global__ void set_slots_kernel(SlotUpdate u, const int *counts, PassSlot *slots, int *status) {
  const int k = threadIdx.x;
  if (k >= u.n) return;
  int cnt = counts[k];
  if (cnt < 0 || cnt > u.max_maps[k]) {
    atomicCAS(status, 0, (int)DRC_ERR_INVALID_ARG);
    cnt = cnt < 0 ? 0 : u.max_maps[k];
  }
  slots[k].count = cnt;
  slots[k].flags = u.flags;
  slots[k].in = u.in[k];
  slots[k].out = u.out[k];
  slots[k].payload = u.payload[k];
}

// Tile-width candidates of a layer: the default, and half of it while the
// half stays a multiple of 16.
std::vector<int> bn_candidates(const Layer &L) {
  std::vector<int> v{L.BN};
  if (L.BN % 32 == 0 && L.BN / 2 >= 32) v.push_back(L.BN / 2);
  return v;
}

drc_status refresh_head_weights(drc_ctx *c, cudaStream_t st) {
  if (!c->headw_stale) return DRC_OK;
  const Layer &Lh = c->layers.back();
  std::vector<float> h((size_t)Lh.Cin * 27);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess)
    e = cudaMemcpy(h.data(), c->d_wraw + Lh.w_off, h.size() * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "head weights");
  c->h_headw.swap(h);
  c->headw_stale = false;
  return DRC_OK;
}

}  // namespace

namespace {

// ---------------------------------------------------------------- training

// Data-gradient GEMMs: the gradient of a stride-2 conv w.r.t. its input is a
// transposed conv of the output gradient with the same weights (roles of
// input and output channels swapped), and that of a transposed conv is a
// stride-2 conv -- so encoder conv e_s becomes an LK_CONVT layer (Cin = c_s,
// Cout = c_{s-1}; the first layer's 7 input channels padded to 16) and
// decoder convT d_s an LK_CONV layer (Cin = c_{s-1}, Cout = c_s), both
// reading the forward layer's raw weights.
void plan_dgrad_layers(drc_ctx *c) {
  const int S = c->cfg.num_stages;
  const int bke = bke_of(c->prec);
  c->dlayers.clear();
  for (size_t li = 0; li + 1 < c->layers.size(); ++li) {
    const Layer &F = c->layers[li];
    Layer L;
    memset(&L, 0, sizeof L);
    L.prec = c->prec;
    L.w_off = F.w_off;
    L.b_off = F.b_off;
    if (F.kind == LK_CONV) {
      L.kind = LK_CONVT;
      L.Cin = L.Cin_raw = F.Cout;
      L.Cout_raw = F.Cin_raw;
      L.Cout = F.Cin_raw < 16 ? 16 : F.Cin_raw;
      set_bn(L, pick_bn(L.Cout));
      L.num_phases = 4;
      for (int p = 0; p < 4; ++p) convT_phase(L.ph[p], p >> 1, p & 1, L.Cin, bke);
      snprintf(L.name, sizeof L.name, "dgrad e%d", (int)li + 1);
    } else {
      L.kind = LK_CONV;
      L.Cin = L.Cin_raw = F.Cout;
      L.Cout = F.Cin;
      set_bn(L, pick_bn(L.Cout));
      L.num_phases = 1;
      PhaseDesc &pd = L.ph[0];
      pd.ntaps = 9;
      for (int t = 0; t < 9; ++t) {
        pd.u[t] = pd.dy[t] = (signed char)(t / 3);
        pd.v[t] = pd.dx[t] = (signed char)(t % 3);
      }
      pd.num_kb = ceil_div(9ll * L.Cin, bke);
      snprintf(L.name, sizeof L.name, "dgrad d%d", S - ((int)li - S));
    }
    for (int p = 0; p < 4; ++p) L.phase_order[p] = p < L.num_phases ? p : 0;
    for (int a = 0; a < L.num_phases; ++a)
      for (int b = a + 1; b < L.num_phases; ++b)
        if (L.ph[L.phase_order[b]].num_kb > L.ph[L.phase_order[a]].num_kb) {
          const int t = L.phase_order[a];
          L.phase_order[a] = L.phase_order[b];
          L.phase_order[b] = t;
        }
    c->dlayers.push_back(L);
  }
  c->dpack_total = layout_packs(c->dlayers);
}

drc_status ensure_dgrad_pack(drc_ctx *c, cudaStream_t st) {
  if (c->dlayers.empty()) {
    plan_dgrad_layers(c);
    cudaError_t e = ctx_malloc(c, &c->d_dpack, c->dpack_total);
    if (e == cudaSuccess && c->prec == PREC_TF32X3) e = ctx_malloc(c, &c->d_dpack_lo, c->dpack_total);
    if (e != cudaSuccess) {
      c->dlayers.clear();
      return cuda_fail(c, e, "data-gradient operands");
    }
    c->dpack_version = 0;
  }
  if (c->dpack_version == c->weights_version) return DRC_OK;
  drc_status s = pack_layers(c, c->dlayers, c->d_dpack, c->d_dpack_lo, st);
  if (s == DRC_OK) c->dpack_version = c->weights_version;
  return s;
}

// Training workspace: activation level q is (H >> q) x (W >> q) x c_q.
struct TrainBufs {
  uint8_t *in8 = nullptr;                 // level 0, 8 channels
  std::vector<uint8_t *> e, t, r;         // e[q] q=1..S; t[q] q=1..S-1; r[s] (output of d_s, level s-1) s=2..S
  std::vector<uint8_t *> Gt, gzd, gze;    // grad w.r.t. t_q (unmasked) and masked by r_{q+1}; encoder grad z_q
  float *out = nullptr, *g4 = nullptr;    // network output [N][3][H][W]; dL/dout NHWC4
  void *g8 = nullptr;                     // BF16 contexts: dL/dout as bf16 NHWC8 (the head's weight gradient)
  uint8_t *dx16 = nullptr;                // input gradient NHWC16
  float2 *part = nullptr;                 // FP32 path: compensated split partials of the weight gradients
};

// Largest compensated-partials buffer (float2 elements) any weight or bias
// gradient of drc_backward needs (FP32 path), with the shapes of its calls.
size_t train_partial_elems(const drc_ctx *c, int N, int H, int W) {
  const int S = c->cfg.num_stages, c1 = c->cfg.widths[0], ns = c->num_sms;
  size_t m = 0;
  auto take = [&](size_t v) { m = v > m ? v : m; };
  const Layer &Lh = c->layers.back();
  take(wgrad_partial_elems(N, H >> 1, W >> 1, c1, 4, 3, ns));
  take(colsum_partial_elems((long long)N * H * W, 4, 3, false, ns));
  (void)Lh;
  for (int s2 = 2; s2 <= S; ++s2) {
    const Layer &F = c->layers[(size_t)(2 * S - s2)];
    take(wgrad_partial_elems(N, H >> s2, W >> s2, F.Cin, F.Cout, F.Cout, ns));
    take(colsum_partial_elems((long long)N * (H >> (s2 - 1)) * (W >> (s2 - 1)), F.Cout, F.Cout, false, ns));
  }
  for (int s2 = S; s2 >= 1; --s2) {
    const Layer &F = c->layers[(size_t)(s2 - 1)];
    take(wgrad_partial_elems(N, H >> s2, W >> s2, F.Cout, F.Cin, F.Cin_raw, ns));
    take(colsum_partial_elems((long long)N * (H >> s2) * (W >> s2), F.Cout, F.Cout, false, ns));
  }
  return m;
}

size_t train_layout(const drc_ctx *c, int N, int H, int W, bool recompute, void *base, TrainBufs *tb) {
  const int S = c->cfg.num_stages;
  const size_t eb = elem_act(c->prec);
  size_t off = 0;
  auto take = [&](size_t bytes) -> uint8_t * {
    uint8_t *p = base ? static_cast<uint8_t *>(base) + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  auto level = [&](int q) { return (size_t)N * (H >> q) * (W >> q) * c->cfg.widths[q - 1] * eb; };
  TrainBufs b;
  b.e.assign(S + 1, nullptr);
  b.t.assign(S + 1, nullptr);
  b.r.assign(S + 1, nullptr);
  b.Gt.assign(S + 1, nullptr);
  b.gzd.assign(S + 1, nullptr);
  b.gze.assign(S + 1, nullptr);
  b.in8 = take((size_t)N * H * W * 8 * eb);
  for (int q = 1; q <= S; ++q) b.e[q] = take(level(q));
  for (int q = 1; q < S; ++q) b.t[q] = recompute ? b.e[q] : take(level(q));
  for (int s2 = 2; s2 <= S; ++s2) b.r[s2] = take(level(s2 - 1));
  for (int q = 1; q < S; ++q) {
    b.Gt[q] = take(level(q));
    b.gzd[q] = take(level(q));
  }
  for (int q = 1; q <= S; ++q) b.gze[q] = take(level(q));
  b.out = reinterpret_cast<float *>(take((size_t)N * 3 * H * W * sizeof(float)));
  b.g4 = reinterpret_cast<float *>(take((size_t)N * H * W * 4 * sizeof(float)));
  if (c->prec != PREC_TF32X3) b.g8 = take((size_t)N * H * W * 8 * 2);
  b.dx16 = take((size_t)N * H * W * 16 * eb);
  if (c->prec == PREC_TF32X3) b.part = reinterpret_cast<float2 *>(take(train_partial_elems(c, N, H, W) * sizeof(float2)));
  if (tb) *tb = b;
  return off;
}

// Weight gradient dW[m][q][3][3] += sum R[n,i,j,m] Q[n,2i+u-1,2j+v-1,q]: on
// the tensor cores where both operands are BF16 and the shape fits
// (wgrad_tc.cu), else the SIMT kernel (fp32 or compensated fp64 sums).
cudaError_t weight_grad(const drc_ctx *c, const void *R, bool r_bf16, const void *Q, bool q_bf16, int N, int Hb,
                        int Wb, int Mr, int Qc, int Qraw, float *dW, float2 *part, cudaStream_t st) {
  EncodeTiledFn enc = encode_tiled();
  const int form = r_bf16 && q_bf16 && !part && enc && N > 0 ? wgrad_tc_form(Hb, Wb, Mr, Qc) : WGRAD_TC_NONE;
  if (form != WGRAD_TC_NONE) {
    const bool narrow = form == WGRAD_TC_NARROW;
    WgradTcArgs a;
    memset(&a, 0, sizeof a);
    int rows, maps;
    wgrad_tc_box(Hb, Wb, &rows, &maps);
    const cuuint64_t K = (cuuint64_t)N * Hb * Wb;
    cuuint64_t rd[2] = {(cuuint64_t)Mr, K}, rs[1] = {(cuuint64_t)Mr * 2};
    cuuint32_t rb[2] = {64, 64}, re[2] = {1, 1};
    cuuint64_t qd[4] = {(cuuint64_t)Qc, (cuuint64_t)(2 * Wb), (cuuint64_t)(2 * Hb), (cuuint64_t)N};
    cuuint64_t qs[3] = {(cuuint64_t)Qc * 2, (cuuint64_t)Qc * 2 * 2 * Wb, (cuuint64_t)Qc * 2 * 2 * Wb * 2 * Hb};
    cuuint32_t qb[4] = {narrow ? 8u : 64u, (cuuint32_t)(2 * Wb), (cuuint32_t)(2 * rows), (cuuint32_t)maps};
    cuuint32_t qe[4] = {1, 2, 2, 1};
    const bool ok =
        enc(&a.mapR, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(R), rd, rs, rb, re,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
        enc(&a.mapQ, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(Q), qd, qs, qb, qe,
            CU_TENSOR_MAP_INTERLEAVE_NONE, narrow ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    if (ok) {
      a.dW = dW;
      a.status = c->d_status;
      a.timeout_ns = c->timeout_ns;
      a.N = N;
      a.Hb = Hb;
      a.Wb = Wb;
      a.Mr = Mr;
      a.Qraw = Qraw;
      if (narrow) {  // N of the GEMM = R channels, up to 256 per tile
        a.BN = Mr <= 256 ? Mr : (Mr % 256 == 0 ? 256 : (Mr % 128 == 0 ? 128 : 64));
        a.m_tiles = 1;
        a.n_tiles = Mr / a.BN;
      } else {
        a.BN = Qc % 128 == 0 ? 128 : 64;
        a.m_tiles = Mr / 128;
        a.n_tiles = Qc / a.BN;
      }
      return launch_wgrad_tc(a, form, c->num_sms, st);
    }
  }
  return launch_wgrad(R, r_bf16, Q, q_bf16, N, Hb, Wb, Mr, Qc, Qraw, dW, part, c->num_sms, st);
}

// ConvArgs of layer L on explicit buffers (input Hin x Win, N maps).
void train_conv_args(const drc_ctx *c, const Layer &L, const uint8_t *B, const uint8_t *B_lo, int N, int Hin,
                     int Win, const void *x, void *y, const void *skip, int relu, const float *bias, ConvArgs &a) {
  fill_common(c, L, B, B_lo, a);
  a.N = N;
  a.x = x;
  a.y = y;
  a.skip = skip;
  a.Hin = Hin;
  a.Win = Win;
  a.Cin = L.Cin;
  a.Cout = L.Cout;
  if (L.kind == LK_CONV) {
    a.Hrow = a.Hout = Hin / 2;
    a.Wrow = a.Wout = Win / 2;
  } else {
    a.Hrow = Hin;
    a.Wrow = Win;
    a.Hout = 2 * Hin;
    a.Wout = 2 * Win;
  }
  a.relu = relu;
  a.bias = bias;
  a.M = (int)((long long)N * a.Hrow * a.Wrow);
  a.m_tiles = ceil_div(a.M, BM);
}

// Forward pass keeping what the reverse pass needs: e_q, t_q, the decoder
// ReLU outputs r_s (before the skip add), the output.  encoder_only: run
// e_1..e_S again (activation checkpointing).
drc_status train_forward(drc_ctx *c, const TrainBufs &b, const float *in, int N, int H, int W, unsigned flags,
                         bool encoder_only, cudaStream_t st) {
  const int S = c->cfg.num_stages;
  const bool bf = c->prec != PREC_TF32X3;
  Tracer *tr = &c->tracer;
  cudaError_t e;
  if (!encoder_only) {
    DRC_TRACED(tr, "stage input", st,
               e = launch_nchw7_to_nhwc8(in, b.in8, (long long)H * W, N, bf, (flags & DRC_F_ENCODE_INPUT) != 0,
                                         c->cfg.exposure, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "input staging");
  }
  for (int s2 = 1; s2 <= S; ++s2) {
    const Layer &L = c->layers[s2 - 1];
    ConvArgs a;
    train_conv_args(c, L, c->d_pack, c->d_pack_lo, N, H >> (s2 - 1), W >> (s2 - 1),
                    s2 == 1 ? (const void *)b.in8 : b.e[s2 - 1], b.e[s2], nullptr, 1, c->d_wraw + L.b_off, a);
    plan_operand(L.prec, a, c->modes[s2 - 1]);
    DRC_TRACED(tr, L.name, st, e = launch_conv(a, L.prec, c->num_sms, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "encoder launch");
  }
  if (encoder_only) return DRC_OK;
  for (int s2 = S; s2 >= 2; --s2) {
    const size_t li = (size_t)(2 * S - s2);
    const Layer &L = c->layers[li];
    ConvArgs a;
    train_conv_args(c, L, c->d_pack, c->d_pack_lo, N, H >> s2, W >> s2, s2 == S ? b.e[S] : b.t[s2], b.t[s2 - 1],
                    b.e[s2 - 1], 1, c->d_wraw + L.b_off, a);
    a.y2 = b.r[s2];
    a.y2_pre_skip = 1;
    plan_operand(L.prec, a, c->modes[li]);
    DRC_TRACED(tr, L.name, st, e = launch_conv(a, L.prec, c->num_sms, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "decoder launch");
  }
  const Layer &Lh = c->layers.back();
  HeadArgs h;
  memset(&h, 0, sizeof h);
  h.x = S >= 2 ? b.t[1] : b.e[1];
  h.out = b.out;
  h.w = c->d_wraw + Lh.w_off;
  h.bias = c->d_wraw + Lh.b_off;
  h.N = N;
  h.Hh = H >> 1;
  h.Wh = W >> 1;
  h.C = Lh.Cin;
  h.relu = c->cfg.out_relu ? 1 : 0;
  h.inv_exposure = 1.0f / c->cfg.exposure;
  head_inline_weights(c, h);
  DRC_TRACED(tr, Lh.name, st, e = launch_head(h, c->prec, st));
  if (e != cudaSuccess) return cuda_fail(c, e, "head launch");
  return DRC_OK;
}

}  // namespace

struct drc_plan {
  drc_ctx *ctx = nullptr;
  unsigned flags = 0;
  std::vector<drc_size_class> cls;
  std::vector<std::vector<Layer>> layers;  // per class: the context's layers with the chosen tile widths
  std::vector<std::vector<int>> modes;     // per class and layer: A-operand path (-1 = default)
  std::vector<uint8_t *> pack, pack_lo;    // per class
  std::vector<Chain> chains;
  void *d_act = nullptr;
  PassSlot *d_slots = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long weights_version = 0;  // the context weights the packed operands hold
  unsigned long long graph_version = 0;    // ... and the graph's head parameters
  int kernels_per_launch = 0;
};

namespace {

void plan_free(drc_plan *p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (uint8_t *b : p->pack) ctx_free(p->ctx, b);
  for (uint8_t *b : p->pack_lo) ctx_free(p->ctx, b);
  ctx_free(p->ctx, p->d_act);
  ctx_free(p->ctx, p->d_slots);
  cudaGetLastError();
  delete p;
}

// Capture the launch sequence of every class into one graph (replacing any
// earlier one); the kernels read each pass's count and buffers from the
// plan's slots.  The head's weights travel in its launch parameters, so the
// graph is captured again whenever the context's weights change.
drc_status plan_capture(drc_plan *p, cudaStream_t cs) {
  drc_ctx *c = p->ctx;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
  p->kernels_per_launch = 0;
  // The size classes are independent chains: each class after the first is
  // captured on a stream of its own, forked from and joined back into the
  // capture stream, so that the graph runs them concurrently and one class's
  // layers fill the SMs the other's tail leaves idle.
  const size_t ncls = p->cls.size();
  std::vector<cudaStream_t> side(ncls > 1 ? ncls - 1 : 0, nullptr);
  std::vector<cudaEvent_t> done(side.size(), nullptr);
  cudaEvent_t fork = nullptr;
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; e == cudaSuccess && k < side.size(); ++k) {
    e = cudaStreamCreateWithFlags(&side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess && !side.empty()) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  auto release = [&]() {
    for (cudaStream_t x : side)
      if (x) cudaStreamDestroy(x);
    for (cudaEvent_t x : done)
      if (x) cudaEventDestroy(x);
    if (fork) cudaEventDestroy(fork);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "plan streams");
  }
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "begin capture");
  }
  drc_status cap = DRC_OK;
  if (fork) {
    cudaEventRecord(fork, cs);
    for (cudaStream_t x : side) cudaStreamWaitEvent(x, fork, 0);
  }
  for (size_t k = 0; cap == DRC_OK && k < ncls; ++k) {
    cudaStream_t sk = k == 0 ? cs : side[k - 1];
    cap = run_chain(c, p->layers[k], p->pack[k], p->pack_lo[k], &p->modes[k], p->chains[k], nullptr, nullptr,
                    nullptr, 0, sk, nullptr, nullptr);
    p->kernels_per_launch += 1 + (int)p->layers[k].size();
  }
  for (size_t k = 0; k < side.size(); ++k) {  // join (also after a failure: capture must end on one stream)
    cudaEventRecord(done[k], side[k]);
    cudaStreamWaitEvent(cs, done[k], 0);
  }
  e = cudaStreamEndCapture(cs, &p->graph);
  release();
  if (cap != DRC_OK) return cap;
  if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
  if ((e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
  p->graph_version = c->weights_version;
  return DRC_OK;
}

drc_status plan_pack(drc_plan *p, cudaStream_t st) {
  drc_ctx *c = p->ctx;
  for (size_t k = 0; k < p->cls.size(); ++k) {
    drc_status s = pack_layers(c, p->layers[k], p->pack[k], p->pack_lo[k], st);
    if (s != DRC_OK) return s;
  }
  p->weights_version = c->weights_version;
  return DRC_OK;
}

// Time one conv launch (min of 3 launches after one warm-up).
drc_status time_args(drc_ctx *c, ConvArgs &a, int prec, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                     float *best_ms) {
  a.count = nullptr;
  float best = 1e30f;
  for (int r = 0; r < 4; ++r) {
    cudaEventRecord(e0, st);
    cudaError_t e = launch_conv(a, prec, c->num_sms, st);
    cudaEventRecord(e1, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune launch");
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return cuda_fail(c, e, "autotune sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  *best_ms = best;
  return DRC_OK;
}

drc_status time_layer(drc_ctx *c, const std::vector<Layer> &Ls, const Layer &L, size_t li, const Chain &ch,
                      const uint8_t *B, const uint8_t *B_lo, int mode, cudaStream_t st, cudaEvent_t e0,
                      cudaEvent_t e1, float *best_ms) {
  ConvArgs a;
  conv_args_for(c, Ls, L, li, ch, B, B_lo, mode, a);
  return time_args(c, a, L.prec, st, e0, e1, best_ms);
}

// Pick each conv layer's tile width (and, split-tf32, the A-operand path) by
// timing the candidates on a chain's full-size buffers.  pairs: the chain is
// the context's own, whose decoder layers may also run as phase pairs.
drc_status autotune_layers(drc_ctx *c, std::vector<Layer> &Ls, std::vector<int> &modes, const Chain &ch,
                           cudaStream_t st, bool pairs = false) {
  size_t scratch = 0;
  for (const Layer &L : Ls) {
    if (L.kind == LK_HEAD) continue;
    std::vector<Layer> one{L};
    for (int bn : bn_candidates(L)) {
      set_bn(one[0], bn);
      const size_t b = layout_packs(one);
      if (b > scratch) scratch = b;
    }
  }
  uint8_t *B = nullptr, *B_lo = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = ctx_malloc(c, &B, scratch);
  if (e == cudaSuccess && c->prec == PREC_TF32X3) e = ctx_malloc(c, &B_lo, scratch);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  drc_status s = e == cudaSuccess ? DRC_OK : cuda_fail(c, e, "autotune scratch");
  for (size_t li = 0; s == DRC_OK && li < Ls.size(); ++li) {
    if (Ls[li].kind == LK_HEAD) continue;
    float best = 1e30f;
    int best_bn = Ls[li].BN, best_mode = -1;
    for (int bn : bn_candidates(Ls[li])) {
      std::vector<Layer> one{Ls[li]};
      set_bn(one[0], bn);
      layout_packs(one);
      if ((s = pack_layers(c, one, B, B_lo, st)) != DRC_OK) break;
      std::vector<int> mode_list{-1};
      if (c->prec == PREC_TF32X3 && bn <= 128) mode_list.push_back(PROD_TMA_CONVERT);
      if (c->prec == PREC_TF32X3 && Ls[li].kind == LK_CONV && Ls[li].Cin == 8) mode_list.push_back(PROD_CPASYNC);
      for (int mode : mode_list) {
        float ms = 0.f;
        if ((s = time_layer(c, Ls, one[0], li, ch, B, B_lo, mode, st, e0, e1, &ms)) != DRC_OK) break;
        if (ms < best) {
          best = ms;
          best_bn = bn;
          best_mode = mode;
        }
      }
      if (s != DRC_OK) break;
    }
    for (int pm : {A_PATH_PAIRED, A_PATH_PAIRED_SMEM}) {
      ConvArgs pa;
      if (s != DRC_OK || !pairs || !paired_args(c, li, ch, pm, pa)) continue;
      float ms = 0.f;
      s = time_args(c, pa, Ls[li].prec, st, e0, e1, &ms);
      if (s == DRC_OK && ms < best) {  // the unpaired tile width stays the fallback
        best = ms;
        best_mode = pm;
      }
    }
    set_bn(Ls[li], best_bn);
    modes[li] = best_mode;
  }
  cudaStreamSynchronize(st);
  ctx_free(c, B);
  ctx_free(c, B_lo);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  return s;
}

}  // namespace

extern "C" {

size_t drc_weight_count(const drc_config *cfg) { return cfg ? weight_count(cfg) : 0; }

drc_status drc_create(const drc_config *cfg, const float *weights_host, size_t n_floats, drc_ctx **out) {
  if (!out) return DRC_ERR_INVALID_ARG;
  *out = nullptr;
  drc_status s = check_config(cfg, nullptr);
  if (s != DRC_OK) return s;
  drc_ctx *c = new (std::nothrow) drc_ctx();
  if (!c) return DRC_ERR_OOM;
  c->cfg = *cfg;
  c->prec = cfg->precision == DRC_PREC_FP32 ? PREC_TF32X3 : (cfg->precision == DRC_PREC_BF16 ? PREC_BF16 : PREC_FP8);
  c->n_floats = weight_count(cfg);
  c->timeout_ns = (unsigned long long)(cfg->wait_timeout_ms > 0 ? cfg->wait_timeout_ms : 2000) * 1000000ull;
  if (weights_host && n_floats != c->n_floats) {
    delete c;
    return DRC_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  int major = 0, minor = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return DRC_ERR_CUDA;
  }
  if (major != 10 || minor != 3) {
    delete c;
    return DRC_ERR_UNSUPPORTED;  // built for sm_103a only
  }
  plan_layers(c);
  c->modes.assign(c->layers.size(), -1);
  e = ctx_malloc(c, &c->d_wraw, c->n_floats * sizeof(float));
  if (e == cudaSuccess) e = ctx_malloc(c, &c->d_pack, c->pack_total);
  if (e == cudaSuccess && c->prec == PREC_TF32X3) e = ctx_malloc(c, &c->d_pack_lo, c->pack_total);
  if (e == cudaSuccess && c->ppack_total) e = ctx_malloc(c, &c->d_ppack, c->ppack_total);
  if (e == cudaSuccess && c->ppack_total) e = ctx_malloc(c, &c->d_ppack_lo, c->ppack_total);
  if (e == cudaSuccess) e = ctx_malloc(c, &c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = ctx_malloc(c, &c->d_zero, 1024 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(c->d_zero, 0, 1024 * sizeof(float));
  if (e == cudaSuccess && c->prec == PREC_FP8) {
    // activation scales start at 1 (values up to the e4m3 maximum, 448)
    // until drc_calibrate measures the network's activations
    c->h_inscale.assign(c->n_scales, 1.0f);
    e = ctx_malloc(c, &c->d_inscale, c->n_scales * sizeof(float));
    if (e == cudaSuccess) e = ctx_malloc(c, &c->d_qinv, c->n_scales * sizeof(float));
    if (e == cudaSuccess) e = ctx_malloc(c, &c->d_bscale, c->n_bscales * sizeof(float));
    if (e == cudaSuccess) e = ctx_malloc(c, &c->d_amax, c->n_bscales * sizeof(unsigned));
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d_inscale, c->h_inscale.data(), c->n_scales * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->d_qinv, c->h_inscale.data(), c->n_scales * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    drc_destroy(c);
    return e == cudaErrorMemoryAllocation ? DRC_ERR_OOM : DRC_ERR_CUDA;
  }
  if (cfg->max_maps > 0 && cfg->max_hw > 0) {
    int side = (int)std::sqrt((double)cfg->max_hw);
    if (ensure_act(c, cfg->max_maps, side, side) != DRC_OK) {
      drc_destroy(c);
      return DRC_ERR_OOM;
    }
  }
  if (weights_host) {
    s = drc_set_weights(c, weights_host, 0, nullptr);
    if (s == DRC_OK && cudaDeviceSynchronize() != cudaSuccess) s = DRC_ERR_CUDA;
    if (s != DRC_OK) {
      drc_destroy(c);
      return s;
    }
  }
  *out = c;
  return DRC_OK;
}

drc_status drc_set_weights(drc_ctx *c, const float *weights, int weights_on_device, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  if (!weights) return fail(c, DRC_ERR_INVALID_ARG, "weights is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (weights_on_device) {
    if (!is_device_ptr(weights, c->device))
      return fail(c, DRC_ERR_INVALID_ARG, "weights_on_device set but weights is not device memory");
    e = cudaMemcpyAsync(c->d_wraw, weights, c->n_floats * sizeof(float), cudaMemcpyDeviceToDevice, st);
  } else {
    e = cudaMemcpy(c->d_wraw, weights, c->n_floats * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "weight upload");
  {
    const Layer &Lh = c->layers.back();
    if (weights_on_device) {
      // No read-back here (a training loop sets weights from the device every
      // step): until an inference call refreshes the host copy, the head
      // reads its weights from device memory.
      c->h_headw.clear();
      c->headw_stale = true;
    } else {
      c->h_headw.assign((size_t)Lh.Cin * 27, 0.f);
      memcpy(c->h_headw.data(), weights + Lh.w_off, c->h_headw.size() * sizeof(float));
      c->headw_stale = false;
    }
  }
  drc_status s = pack_all(c, st);
  if (s == DRC_OK) {
    c->weights_set = true;
    ++c->weights_version;
  }
  return s;
}

drc_status drc_destroy(drc_ctx *c) {
  if (!c) return DRC_ERR_INVALID_ARG;
  ctx_free(c, c->d_wraw);
  ctx_free(c, c->d_pack);
  ctx_free(c, c->d_pack_lo);
  ctx_free(c, c->d_ppack);
  ctx_free(c, c->d_ppack_lo);
  ctx_free(c, c->d_bscale);
  ctx_free(c, c->d_inscale);
  ctx_free(c, c->d_dpack);
  ctx_free(c, c->d_dpack_lo);
  ctx_free(c, c->d_train);
  ctx_free(c, c->d_zero);
  ctx_free(c, c->d_qinv);
  ctx_free(c, c->d_amax);
  ctx_free(c, c->d_act);
  ctx_free(c, c->d_iscratch);
  ctx_free(c, c->d_indscratch);
  ctx_free(c, c->d_status);
  ctx_free(c, c->d_prof);
  ctx_free(c, c->d_fmaps);
  ctx_free(c, c->d_fout);
  ctx_free(c, c->d_fpay);
  ctx_free(c, c->d_fgpos);
  ctx_free(c, c->d_fgnrm);
  ctx_free(c, c->d_frgb);
  for (cudaEvent_t e : {c->fev_maps, c->fev_gbuf, c->fev_maps_free, c->fev_gbuf_free})
    if (e) cudaEventDestroy(e);
  if (c->fcopy) cudaStreamDestroy(c->fcopy);
  cudaGetLastError();
  delete c;
  return DRC_OK;
}

drc_status drc_denoise(drc_ctx *c, const float *in, float *out, float *payload, int N, int H, int W,
                       unsigned flags, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  const int S = c->cfg.num_stages;
  const unsigned known = DRC_F_ENCODE_INPUT | DRC_F_DECODE_OUTPUT | DRC_F_DEBUG_STALL;
  if (flags & ~known) return fail(c, DRC_ERR_INVALID_ARG, "unknown flags 0x%x", flags & ~known);
  if (N < 0) return fail(c, DRC_ERR_INVALID_ARG, "N must be >= 0");
  if (H < (1 << S) || W < (1 << S) || H % (1 << S) || W % (1 << S))
    return fail(c, DRC_ERR_INVALID_ARG, "H, W (%d, %d) must be positive multiples of 2^S = %d", H, W, 1 << S);
  if (payload && H > 256) return fail(c, DRC_ERR_INVALID_ARG, "payload needs H <= 256");
  if ((long long)N * H * W * 7 >= (1ll << 31))
    return fail(c, DRC_ERR_INVALID_ARG, "N*7*H*W must stay below 2^31 elements per call");
  if (!c->weights_set) return fail(c, DRC_ERR_INVALID_ARG, "weights were never set");
  if (N == 0) return DRC_OK;
  drc_status s;
  if ((s = check_dev(c, in, "in", false)) != DRC_OK) return s;
  if ((s = check_dev(c, out, "out", false)) != DRC_OK) return s;
  if ((s = check_dev(c, payload, "payload", true)) != DRC_OK) return s;
  if ((s = ensure_act(c, N, H, W)) != DRC_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  Chain ch;
  carve_chain(c, c->d_act, N, H, W, ch);
  if (payload) {
    e = cudaMemsetAsync(payload, 0, (size_t)N * 3 * sizeof(float), st);
    if (e != cudaSuccess) return cuda_fail(c, e, "payload clear");
  }
  // Diagnostic: with DRC_PROFILE_WAITS set in the environment every conv
  // launch records how long each warp role waited, printed to stderr per
  // layer after the call (synchronising).  Off by default.
  const bool prof = std::getenv("DRC_PROFILE_WAITS") != nullptr;
  if (prof) {
    const size_t pb = c->layers.size() * PROF_SLOTS * sizeof(unsigned long long);
    if (!c->d_prof) {
      const cudaError_t pe = ctx_malloc(c, &c->d_prof, pb);
      if (pe != cudaSuccess) return cuda_fail(c, pe, "wait-time counters");
    }
    cudaMemsetAsync(c->d_prof, 0, pb, st);
  }
  if ((s = refresh_head_weights(c, st)) != DRC_OK) return s;
  s = run_chain(c, c->layers, c->d_pack, c->d_pack_lo, &c->modes, ch, in, out, payload, flags, st, &c->tracer,
                prof ? c->d_prof : nullptr);
  if (s != DRC_OK) return s;
  if (prof) {
    std::vector<unsigned long long> h(c->layers.size() * PROF_SLOTS);
    cudaStreamSynchronize(st);
    cudaMemcpy(h.data(), c->d_prof, h.size() * sizeof(h[0]), cudaMemcpyDeviceToHost);
    for (size_t li = 0; li < c->layers.size(); ++li) {
      const unsigned long long *v = h.data() + li * PROF_SLOTS;
      const double ctas = v[PROF_CTAS] ? (double)v[PROF_CTAS] : 1.0;
      if (!v[PROF_CTAS]) continue;
      fprintf(stderr,
              "[drc prof] layer %zu kind %d BN %d: per CTA kcycles: mma total %.1f wait_full %.1f wait_tempty %.1f | "
              "bload wait_empty %.1f | prod(8 warps) total %.1f wait_empty %.1f wait_copy %.1f issue %.1f convert %.1f "
              "fence %.1f | epi(4 warps) total %.1f wait_tfull %.1f acc_ld %.1f\n",
              li, c->layers[li].kind, c->layers[li].BN, v[PROF_MMA_TOTAL] / ctas / 1e3,
              v[PROF_MMA_WAIT_FULL] / ctas / 1e3, v[PROF_MMA_WAIT_TEMPTY] / ctas / 1e3,
              v[PROF_BLOAD_WAIT_EMPTY] / ctas / 1e3, v[PROF_PROD_TOTAL] / ctas / 8e3,
              v[PROF_PROD_WAIT_EMPTY] / ctas / 8e3, v[PROF_PROD_WAIT_COPY] / ctas / 8e3,
              v[PROF_PROD_ISSUE] / ctas / 8e3, v[PROF_PROD_CONVERT] / ctas / 8e3, v[PROF_PROD_FENCE] / ctas / 8e3,
              v[PROF_EPI_TOTAL] / ctas / 4e3, v[PROF_EPI_WAIT_TFULL] / ctas / 4e3, v[PROF_EPI_LD] / ctas / 4e3);
    }
  }
  return DRC_OK;
}

drc_status drc_interpolate(drc_ctx *c, const drc_caches *caches, const drc_gbuffer *gbuf,
                           const drc_interp_params *prm, float *out_rgb, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (!caches || !gbuf || !prm) return fail(c, DRC_ERR_INVALID_ARG, "NULL argument struct");
  if (caches->n < 1) return fail(c, DRC_ERR_INVALID_ARG, "caches->n must be >= 1");
  if (prm->k < 1 || prm->k > 32) return fail(c, DRC_ERR_INVALID_ARG, "k must be 1..32");
  if (prm->metric != DRC_METRIC_IMAGE && prm->metric != DRC_METRIC_WORLD)
    return fail(c, DRC_ERR_INVALID_ARG, "unknown metric");
  if (prm->wp_form != DRC_WP_INVERSE && prm->wp_form != DRC_WP_LINEAR)
    return fail(c, DRC_ERR_INVALID_ARG, "unknown wp_form");
  if (prm->mode != DRC_INTERP_IRRADIANCE && prm->mode != DRC_INTERP_LOOKUP)
    return fail(c, DRC_ERR_INVALID_ARG, "unknown mode");
  if (!(prm->r > 0.f) || !(prm->eps >= 0.f) || !(prm->delta_rel > 0.f))
    return fail(c, DRC_ERR_INVALID_ARG, "need r > 0, eps >= 0, delta_rel > 0");
  if (gbuf->width < 0 || gbuf->height < 0) return fail(c, DRC_ERR_INVALID_ARG, "negative G-buffer size");
  const long long P = (long long)gbuf->width * gbuf->height;
  if (P >= (1ll << 31) / 3) return fail(c, DRC_ERR_INVALID_ARG, "G-buffer too large");
  drc_status s;
  if (prm->metric == DRC_METRIC_WORLD) {
    if ((s = check_dev(c, caches->pos, "caches->pos", false)) != DRC_OK) return s;
  } else {
    if ((s = check_dev(c, caches->pix, "caches->pix", false)) != DRC_OK) return s;
  }
  if ((s = check_dev(c, caches->nrm, "caches->nrm", false)) != DRC_OK) return s;
  if (prm->mode == DRC_INTERP_IRRADIANCE) {
    if ((s = check_dev(c, caches->payload, "caches->payload", false)) != DRC_OK) return s;
  } else {
    if (caches->H < 1 || caches->W < 1) return fail(c, DRC_ERR_INVALID_ARG, "LOOKUP needs caches->H, W >= 1");
    if ((s = check_dev(c, caches->maps, "caches->maps", false)) != DRC_OK) return s;
  }
  if (P > 0) {
    if ((s = check_dev(c, out_rgb, "out_rgb", false)) != DRC_OK) return s;
    if ((s = check_dev(c, gbuf->nrm, "gbuf->nrm", false)) != DRC_OK) return s;
    if (prm->metric == DRC_METRIC_WORLD && (s = check_dev(c, gbuf->pos, "gbuf->pos", false)) != DRC_OK) return s;
    if (prm->mode == DRC_INTERP_LOOKUP && (s = check_dev(c, gbuf->dir, "gbuf->dir", false)) != DRC_OK) return s;
    if ((s = check_dev(c, prm->nbr_out, "nbr_out", true)) != DRC_OK) return s;
    if ((s = check_dev(c, prm->nbr_w, "nbr_w", true)) != DRC_OK) return s;
    if (prm->nbr_w && !prm->nbr_out) return fail(c, DRC_ERR_INVALID_ARG, "nbr_w needs nbr_out");
  }
  // grid scratch, plus the pixel ordering for the WORLD metric (the G-buffer's
  // first-hit positions are not coherent in image order)
  const bool order = prm->metric == DRC_METRIC_WORLD && P > 0;
  const size_t grid_bytes = (interp_scratch_bytes(caches->n, prm->k) + 255) & ~(size_t)255;
  const size_t need = grid_bytes + (order ? interp_order_bytes(P, caches->n) : 0);
  if (need > c->iscratch_bytes) {
    if (c->d_iscratch) ctx_free(c, c->d_iscratch);
    c->d_iscratch = nullptr;
    c->iscratch_bytes = 0;
    cudaError_t e = ctx_malloc(c, &c->d_iscratch, need);
    if (e != cudaSuccess) return cuda_fail(c, e, "interpolation scratch");
    c->iscratch_bytes = need;
  }
  InterpArgs a;
  memset(&a, 0, sizeof a);
  a.n = caches->n;
  a.mapH = caches->H;
  a.mapW = caches->W;
  a.maps = caches->maps;
  a.payload = caches->payload;
  a.cpos = caches->pos;
  a.cnrm = caches->nrm;
  a.cpix = caches->pix;
  a.width = gbuf->width;
  a.height = gbuf->height;
  a.gpos = gbuf->pos;
  a.gnrm = gbuf->nrm;
  a.gdir = gbuf->dir;
  a.k = prm->k;
  a.metric = prm->metric;
  a.wp_form = prm->wp_form;
  a.mode = prm->mode;
  a.r = prm->r;
  a.eps = prm->eps;
  a.delta_rel = prm->delta_rel;
  a.out = out_rgb;
  a.nbr_out = prm->nbr_out;
  a.nbr_w = prm->nbr_w;
  InterpScratch sc = interp_carve(c->d_iscratch, caches->n, prm->k);
  if (order) interp_attach_order(sc, static_cast<char *>(c->d_iscratch) + grid_bytes, P, caches->n);
  cudaError_t e = launch_interp(a, sc, static_cast<cudaStream_t>(stream), &c->tracer);
  if (e != cudaSuccess) return cuda_fail(c, e, "interpolation launch");
  return DRC_OK;
}

drc_status drc_indirect(drc_ctx *c, const drc_caches *caches, const drc_gbuffer *gbuf,
                        const drc_indirect_params *prm, float *out_rgb, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (!caches || !gbuf || !prm) return fail(c, DRC_ERR_INVALID_ARG, "NULL argument struct");
  if (caches->n < 1) return fail(c, DRC_ERR_INVALID_ARG, "caches->n must be >= 1");
  if (caches->H < 1 || caches->W < 1 || caches->H > kIndirectMaxRows)
    return fail(c, DRC_ERR_INVALID_ARG, "map size must be 1..%d rows, >= 1 column", kIndirectMaxRows);
  if ((long long)caches->n * caches->H * caches->W * 3 >= (1ll << 31))
    return fail(c, DRC_ERR_INVALID_ARG, "maps too large");
  if (prm->k < 1 || prm->k > 32) return fail(c, DRC_ERR_INVALID_ARG, "k must be 1..32");
  if (prm->S < 1 || prm->S > 4096) return fail(c, DRC_ERR_INVALID_ARG, "S must be 1..4096");
  if (gbuf->width < 0 || gbuf->height < 0) return fail(c, DRC_ERR_INVALID_ARG, "negative G-buffer size");
  const long long P = (long long)gbuf->width * gbuf->height;
  if (P * prm->S >= (1ll << 40)) return fail(c, DRC_ERR_INVALID_ARG, "too many samples");
  drc_status s;
  if ((s = check_dev(c, caches->maps, "caches->maps", false)) != DRC_OK) return s;
  if ((s = check_dev(c, caches->nrm, "caches->nrm", false)) != DRC_OK) return s;
  if (P > 0) {
    if ((s = check_dev(c, out_rgb, "out_rgb", false)) != DRC_OK) return s;
    if ((s = check_dev(c, gbuf->nrm, "gbuf->nrm", false)) != DRC_OK) return s;
    if ((s = check_dev(c, prm->nbr, "nbr", false)) != DRC_OK) return s;
    if ((s = check_dev(c, prm->nbr_w, "nbr_w", false)) != DRC_OK) return s;
    if ((s = check_dev(c, prm->u, "u", false)) != DRC_OK) return s;
    if ((s = check_dev(c, prm->albedo, "albedo", false)) != DRC_OK) return s;
    if ((s = check_dev(c, prm->emit, "emit", true)) != DRC_OK) return s;
    if ((s = check_dev(c, prm->direct, "direct", true)) != DRC_OK) return s;
  }
  IndirectArgs a;
  memset(&a, 0, sizeof a);
  a.n = caches->n;
  a.H = caches->H;
  a.W = caches->W;
  const size_t need = indirect_scratch_bytes(a.n, a.H, a.W);
  if (need > c->indscratch_bytes) {
    if (c->d_indscratch) ctx_free(c, c->d_indscratch);
    c->d_indscratch = nullptr;
    c->indscratch_bytes = 0;
    cudaError_t e = ctx_malloc(c, &c->d_indscratch, need);
    if (e != cudaSuccess) return cuda_fail(c, e, "indirect scratch");
    c->indscratch_bytes = need;
  }
  indirect_carve(a, c->d_indscratch);
  a.maps = caches->maps;
  a.cnrm = caches->nrm;
  a.P = P;
  a.k = prm->k;
  a.S = prm->S;
  a.nbr = prm->nbr;
  a.nbr_w = prm->nbr_w;
  a.gnrm = gbuf->nrm;
  a.albedo = prm->albedo;
  a.u = reinterpret_cast<const float4 *>(prm->u);
  a.emit = prm->emit;
  a.direct = prm->direct;
  a.out = out_rgb;
  // row geometry in double: cos of the band edges, and the texel solid angle
  // written as 2 sin(mid) sin(half-width) (2 pi / W), free of the cancellation
  // of a difference of cosines near the pole
  const double pi = 3.14159265358979323846;
  for (int r = 0; r <= a.H; ++r) a.rowcos[r] = (float)std::cos(r * 0.5 * pi / a.H);
  for (int r = 0; r < a.H; ++r) {
    const double t0 = r * 0.5 * pi / a.H, t1 = (r + 1) * 0.5 * pi / a.H;
    a.omega[r] = (float)(2.0 * std::sin(0.5 * (t0 + t1)) * std::sin(0.5 * (t1 - t0)) * (2.0 * pi / a.W));
  }
  cudaError_t e = launch_indirect(a, static_cast<cudaStream_t>(stream), &c->tracer);
  if (e != cudaSuccess) return cuda_fail(c, e, "indirect launch");
  return DRC_OK;
}

drc_status drc_gen_maps(drc_ctx *c, const drc_scene *scene, int n, const float *pos, const float *nrm, int H,
                        int W, int D, const float *u, float *maps, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (!scene) return fail(c, DRC_ERR_INVALID_ARG, "scene is NULL");
  if (scene->nsph < 0 || scene->nsph > DRC_MAX_SPHERES)
    return fail(c, DRC_ERR_INVALID_ARG, "nsph must be 0..%d", DRC_MAX_SPHERES);
  if (n < 0 || H < 1 || W < 1 || H > 4096 || W > 4096 || D < 0 || D > 64)
    return fail(c, DRC_ERR_INVALID_ARG, "need n >= 0, H and W in 1..4096, D in 0..64");
  if ((long long)n * 7 * H * W >= (1ll << 40)) return fail(c, DRC_ERR_INVALID_ARG, "maps too large");
  if (n == 0) return DRC_OK;
  drc_status s;
  if ((s = check_dev(c, pos, "pos", false)) != DRC_OK) return s;
  if ((s = check_dev(c, nrm, "nrm", false)) != DRC_OK) return s;
  if ((s = check_dev(c, maps, "maps", false)) != DRC_OK) return s;
  if (D > 0 && (s = check_dev(c, u, "u", false)) != DRC_OK) return s;
  MapGenArgs a;
  memset(&a, 0, sizeof a);
  a.scene = *scene;
  a.n = n;
  a.H = H;
  a.W = W;
  a.D = D;
  a.pos = pos;
  a.nrm = nrm;
  a.u = reinterpret_cast<const float2 *>(u);
  a.maps = maps;
  cudaError_t e = launch_gen_maps(a, static_cast<cudaStream_t>(stream), &c->tracer);
  if (e != cudaSuccess) return cuda_fail(c, e, "map generation launch");
  return DRC_OK;
}

drc_status drc_fd_loss64(drc_ctx *c, const double *w64, const float *in, const float *target, int N, int H, int W,
                         unsigned flags, double *loss64, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  const int S = c->cfg.num_stages;
  if (flags & ~DRC_F_ENCODE_INPUT) return fail(c, DRC_ERR_INVALID_ARG, "flags: DRC_F_ENCODE_INPUT or 0");
  if (N < 1) return fail(c, DRC_ERR_INVALID_ARG, "N must be >= 1");
  if (H < (1 << S) || W < (1 << S) || H % (1 << S) || W % (1 << S))
    return fail(c, DRC_ERR_INVALID_ARG, "H, W (%d, %d) must be positive multiples of 2^S = %d", H, W, 1 << S);
  if ((long long)N * H * W * 16 >= (1ll << 31)) return fail(c, DRC_ERR_INVALID_ARG, "too large");
  drc_status s;
  if ((s = check_dev(c, w64, "weights64", false)) != DRC_OK) return s;
  if ((s = check_dev(c, in, "in", false)) != DRC_OK) return s;
  if ((s = check_dev(c, target, "target", false)) != DRC_OK) return s;
  if ((s = check_dev(c, loss64, "loss64", false)) != DRC_OK) return s;
  std::vector<FdLayer> L(c->layers.size());
  for (size_t i = 0; i < c->layers.size(); ++i) {
    const Layer &l = c->layers[i];
    L[i].transposed = l.kind == LK_CONV ? 0 : 1;
    L[i].Cin = l.kind == LK_CONV ? l.Cin_raw : l.Cin;
    L[i].Cout = l.Cout;
    L[i].w_off = l.w_off;
    L[i].b_off = l.b_off;
  }
  cudaError_t e = fd_loss64(L.data(), S, w64, in, target, N, c->cfg.in_channels, H, W,
                            (flags & DRC_F_ENCODE_INPUT) != 0, c->cfg.exposure, c->cfg.out_relu != 0, loss64,
                            static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DRC_OK : cuda_fail(c, e, "fd loss");
}

drc_status drc_pass_points(int width, int height, int spacing0, int pass, int *pix, int max_points, int *count) {
  if (!count || width < 1 || height < 1 || pass < 0 || spacing0 < 1 || (spacing0 & (spacing0 - 1)) || max_points < 0)
    return DRC_ERR_INVALID_ARG;
  *count = 0;
  if (pass > 30 || (spacing0 >> pass) < 1) return DRC_OK;  // the grid cannot get finer than every pixel
  const int st = spacing0 >> pass, prev = pass > 0 ? st * 2 : 0;
  long long n = 0;
  bool fits = true;
  for (int y = 0; y < height; y += st)
    for (int x = 0; x < width; x += st) {
      if (prev && x % prev == 0 && y % prev == 0) continue;  // an earlier pass's point
      if (n < max_points && pix) {
        pix[2 * n] = x;
        pix[2 * n + 1] = y;
      } else {
        fits = false;
      }
      ++n;
    }
  if (n > 0x7fffffff) return DRC_ERR_INVALID_ARG;
  *count = (int)n;
  return fits ? DRC_OK : DRC_ERR_INVALID_ARG;
}

drc_status drc_backward(drc_ctx *c, const float *in, const float *target, int N, int H, int W, unsigned flags,
                        float *dweights, float *dinput, float *loss, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (c->prec == PREC_FP8) return fail(c, DRC_ERR_UNSUPPORTED, "backward runs in FP32 or BF16 contexts");
  const int S = c->cfg.num_stages;
  const unsigned known = DRC_F_ENCODE_INPUT | DRC_BWD_L1_TARGET | DRC_BWD_GRAD_OUT | DRC_BWD_RECOMPUTE_ENCODER;
  if (flags & ~known) return fail(c, DRC_ERR_INVALID_ARG, "unknown flags 0x%x", flags & ~known);
  const bool grad_out = (flags & DRC_BWD_GRAD_OUT) != 0;
  if (grad_out == ((flags & DRC_BWD_L1_TARGET) != 0))
    return fail(c, DRC_ERR_INVALID_ARG, "give exactly one of DRC_BWD_L1_TARGET and DRC_BWD_GRAD_OUT");
  if (N < 1) return fail(c, DRC_ERR_INVALID_ARG, "N must be >= 1");
  if (H < (1 << S) || W < (1 << S) || H % (1 << S) || W % (1 << S))
    return fail(c, DRC_ERR_INVALID_ARG, "H, W (%d, %d) must be positive multiples of 2^S = %d", H, W, 1 << S);
  if ((long long)N * H * W * 16 >= (1ll << 31))
    return fail(c, DRC_ERR_INVALID_ARG, "N*16*H*W must stay below 2^31 elements per call");
  if (!c->weights_set) return fail(c, DRC_ERR_INVALID_ARG, "weights were never set");
  drc_status s;
  if ((s = check_dev(c, in, "in", false)) != DRC_OK) return s;
  if ((s = check_dev(c, target, "target", false)) != DRC_OK) return s;
  if ((s = check_dev(c, dweights, "dweights", false)) != DRC_OK) return s;
  if ((s = check_dev(c, dinput, "dinput", true)) != DRC_OK) return s;
  if ((s = check_dev(c, loss, "loss", true)) != DRC_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((s = ensure_dgrad_pack(c, st)) != DRC_OK) return s;
  const bool recompute = (flags & DRC_BWD_RECOMPUTE_ENCODER) != 0;
  const size_t need = train_layout(c, N, H, W, recompute, nullptr, nullptr);
  cudaError_t e;
  if (need > c->train_bytes) {
    ctx_free(c, c->d_train);
    c->d_train = nullptr;
    c->train_bytes = 0;
    if ((e = ctx_malloc(c, &c->d_train, need)) != cudaSuccess) return cuda_fail(c, e, "training workspace");
    c->train_bytes = need;
  }
  TrainBufs b;
  train_layout(c, N, H, W, recompute, c->d_train, &b);
  const bool bf = c->prec != PREC_TF32X3;
  Tracer *tr = &c->tracer;
  if ((e = cudaMemsetAsync(dweights, 0, c->n_floats * sizeof(float), st)) != cudaSuccess)
    return cuda_fail(c, e, "dweights clear");
  // FP32: compensated partials, reduced (deterministically) into dweights
  float2 *const part = b.part;
  auto opart = [&](size_t) -> float2 * { return part; };
  if (loss && (e = cudaMemsetAsync(loss, 0, sizeof(float), st)) != cudaSuccess) return cuda_fail(c, e, "loss clear");

  if ((s = train_forward(c, b, in, N, H, W, flags, false, st)) != DRC_OK) return s;
  DRC_TRACED(tr, "loss", st, e = launch_l1_grad(b.out, target, N, H, W, grad_out, c->cfg.out_relu != 0, b.g4, b.g8, loss, st));
  if (e != cudaSuccess) return cuda_fail(c, e, "loss");

  // output head: t_1 -> out; the gradient w.r.t. t_1 is masked by the ReLU of
  // d_2 (or of e_1 when there is no decoder stage)
  const Layer &Lh = c->layers.back();
  const int c1 = c->cfg.widths[0];
  DRC_TRACED(tr, "head bwd", st,
             e = launch_head_bwd(b.g4, c->d_wraw + Lh.w_off, S >= 2 ? (const void *)b.r[2] : b.e[1],
                                 S >= 2 ? (void *)b.Gt[1] : nullptr, S >= 2 ? b.gzd[1] : b.gze[1], N, H >> 1, W >> 1,
                                 c1, bf, c->num_sms, st));
  if (e != cudaSuccess) return cuda_fail(c, e, "head backward");
  DRC_TRACED(tr, "wgrad head", st,
             e = weight_grad(c, S >= 2 ? b.t[1] : b.e[1], bf, bf ? b.g8 : (const void *)b.g4, bf, N, H >> 1, W >> 1,
                             c1, bf ? 8 : 4, 3,
                              dweights + Lh.w_off, opart(Lh.w_off), st));
  if (e == cudaSuccess)
    DRC_TRACED(tr, "bgrad head", st,
               e = launch_colsum(b.g4, false, (long long)N * H * W, 4, 3, dweights + Lh.b_off, opart(Lh.b_off),
                                 c->num_sms, st));
  if (e != cudaSuccess) return cuda_fail(c, e, "head weight gradient");

  // decoder, from the output inwards: t_{s-1} = r_s + e_{s-1},
  // r_s = ReLU(convT_s(t_s) + b)
  for (int s2 = 2; s2 <= S; ++s2) {
    const size_t li = (size_t)(2 * S - s2);
    const Layer &F = c->layers[li], &D = c->dlayers[li];
    const void *tin = s2 == S ? b.e[S] : b.t[s2];
    const long long npix = (long long)N * (H >> (s2 - 1)) * (W >> (s2 - 1));
    const std::string wname = std::string("wgrad ") + F.name, bname = std::string("bgrad ") + F.name;
    DRC_TRACED(tr, wname.c_str(), st,
               e = weight_grad(c, tin, bf, b.gzd[s2 - 1], bf, N, H >> s2, W >> s2, F.Cin, F.Cout, F.Cout,
                                dweights + F.w_off, opart(F.w_off), st));
    if (e == cudaSuccess)
      DRC_TRACED(tr, bname.c_str(), st,
                 e = launch_colsum(b.gzd[s2 - 1], bf, npix, F.Cout, F.Cout, dweights + F.b_off, opart(F.b_off),
                                   c->num_sms, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "decoder weight gradient");
    ConvArgs a;
    train_conv_args(c, D, c->d_dpack, c->d_dpack_lo, N, H >> (s2 - 1), W >> (s2 - 1), b.gzd[s2 - 1],
                    s2 < S ? b.gzd[s2] : b.gze[S], nullptr, 0, c->d_zero, a);
    if (s2 < S) {
      a.y2 = b.Gt[s2];
      a.y2_pre_skip = 0;
      a.mask = b.r[s2 + 1];
    } else {
      a.mask = b.e[S];
    }
    plan_operand(D.prec, a, -1);
    DRC_TRACED(tr, D.name, st, e = launch_conv(a, D.prec, c->num_sms, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "decoder data gradient");
  }
  if (recompute && (s = train_forward(c, b, in, N, H, W, flags, true, st)) != DRC_OK) return s;

  // encoder, from the bottleneck outwards: e_s = ReLU(conv_s(e_{s-1}) + b);
  // the gradient w.r.t. e_{s-1} adds the skip branch's Gt_{s-1}
  for (int s2 = S; s2 >= 1; --s2) {
    const size_t li = (size_t)(s2 - 1);
    const Layer &F = c->layers[li], &D = c->dlayers[li];
    const long long npix = (long long)N * (H >> s2) * (W >> s2);
    const void *xin = s2 == 1 ? (const void *)b.in8 : b.e[s2 - 1];
    const std::string wname = std::string("wgrad ") + F.name, bname = std::string("bgrad ") + F.name;
    DRC_TRACED(tr, wname.c_str(), st,
               e = weight_grad(c, b.gze[s2], bf, xin, bf, N, H >> s2, W >> s2, F.Cout, F.Cin, F.Cin_raw,
                                dweights + F.w_off, opart(F.w_off), st));
    if (e == cudaSuccess)
      DRC_TRACED(tr, bname.c_str(), st,
                 e = launch_colsum(b.gze[s2], bf, npix, F.Cout, F.Cout, dweights + F.b_off, opart(F.b_off),
                                   c->num_sms, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "encoder weight gradient");
    if (s2 == 1 && !dinput) break;
    ConvArgs a;
    train_conv_args(c, D, c->d_dpack, c->d_dpack_lo, N, H >> s2, W >> s2, b.gze[s2], s2 > 1 ? b.gze[s2 - 1] : b.dx16,
                    s2 > 1 ? (const void *)b.Gt[s2 - 1] : nullptr, 0, c->d_zero, a);
    if (s2 > 1) a.mask = b.e[s2 - 1];
    plan_operand(D.prec, a, -1);
    DRC_TRACED(tr, D.name, st, e = launch_conv(a, D.prec, c->num_sms, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "encoder data gradient");
  }
  if (dinput) {
    DRC_TRACED(tr, "input grad", st,
               e = launch_dinput(b.dx16, bf, in, (long long)H * W, N, (flags & DRC_F_ENCODE_INPUT) != 0,
                                 c->cfg.exposure, dinput, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "input gradient");
  }
  return DRC_OK;
}

drc_status drc_weight_grad(drc_ctx *c, const void *R, const void *Q, drc_precision dtype, int N, int Hb, int Wb,
                           int Mr, int Qc, int Qraw, float *dW, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (dtype != DRC_PREC_FP32 && dtype != DRC_PREC_BF16)
    return fail(c, DRC_ERR_INVALID_ARG, "operands are FP32 or BF16");
  if (N < 0 || Hb < 1 || Wb < 1 || Mr < 1 || Qc < 1 || Qraw < 1 || Qraw > Qc)
    return fail(c, DRC_ERR_INVALID_ARG, "bad shape N=%d Hb=%d Wb=%d Mr=%d Qc=%d Qraw=%d", N, Hb, Wb, Mr, Qc, Qraw);
  if ((long long)N * 4 * Hb * Wb * (Qc > Mr ? Qc : Mr) >= (1ll << 31))
    return fail(c, DRC_ERR_INVALID_ARG, "operands must stay below 2^31 elements");
  drc_status s;
  if ((s = check_dev(c, dW, "dW", false)) != DRC_OK) return s;
  if (N == 0) return DRC_OK;
  if ((s = check_dev(c, R, "R", false)) != DRC_OK) return s;
  if ((s = check_dev(c, Q, "Q", false)) != DRC_OK) return s;
  const bool bf = dtype == DRC_PREC_BF16;
  cudaError_t e = weight_grad(c, R, bf, Q, bf, N, Hb, Wb, Mr, Qc, Qraw, dW, nullptr, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DRC_OK : cuda_fail(c, e, "weight gradient");
}

drc_status drc_augment(drc_ctx *c, const float *in, float *out, int N, int C, int H, int W, const int *codes,
                       void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (N < 0 || C < 1 || H < 1 || W < 1) return fail(c, DRC_ERR_INVALID_ARG, "bad shape N=%d C=%d H=%d W=%d", N, C, H, W);
  if (H != W) return fail(c, DRC_ERR_INVALID_ARG, "the rotations need square maps (H=%d, W=%d)", H, W);
  const long long count = (long long)N * C * H * W;
  if (count >= (1ll << 31)) return fail(c, DRC_ERR_INVALID_ARG, "maps must stay below 2^31 elements");
  if (N == 0) return DRC_OK;
  drc_status s;
  if ((s = check_dev(c, in, "in", false)) != DRC_OK) return s;
  if ((s = check_dev(c, out, "out", false)) != DRC_OK) return s;
  if ((s = check_dev(c, codes, "codes", false)) != DRC_OK) return s;
  if (in < out + count && out < in + count) return fail(c, DRC_ERR_INVALID_ARG, "in and out overlap");
  const cudaError_t e = launch_augment(in, out, N, C, H, codes, static_cast<cudaStream_t>(stream), &c->tracer);
  return e == cudaSuccess ? DRC_OK : cuda_fail(c, e, "augment");
}

drc_status drc_adam_step(drc_ctx *c, float *w, const float *grad, float *m, float *v, size_t n, int t, float lr,
                         float beta1, float beta2, float eps, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (t < 1) return fail(c, DRC_ERR_INVALID_ARG, "t counts steps from 1");
  if (!(lr > 0.f) || !(lr < INFINITY) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps >= 0.f && eps < INFINITY))
    return fail(c, DRC_ERR_INVALID_ARG, "need lr > 0, 0 <= beta1, beta2 < 1, eps >= 0");
  if (n == 0) return DRC_OK;
  drc_status s;
  if ((s = check_dev(c, w, "w", false)) != DRC_OK) return s;
  if ((s = check_dev(c, grad, "grad", false)) != DRC_OK) return s;
  if ((s = check_dev(c, m, "m", false)) != DRC_OK) return s;
  if ((s = check_dev(c, v, "v", false)) != DRC_OK) return s;
  // bias corrections in double on the host, applied as factors
  const double c1 = 1.0 / (1.0 - std::pow((double)beta1, (double)t));
  const double c2 = 1.0 / std::sqrt(1.0 - std::pow((double)beta2, (double)t));
  const cudaError_t e = launch_adam(w, grad, m, v, n, lr, beta1, beta2, eps, (float)c1, (float)c2,
                                    static_cast<cudaStream_t>(stream), &c->tracer);
  return e == cudaSuccess ? DRC_OK : cuda_fail(c, e, "adam step");
}

static bool unet_shape_ok(int in_ch, int out_ch, int base, int levels) {
  return in_ch >= 1 && in_ch <= 64 && out_ch >= 1 && out_ch <= 64 && levels >= 1 && levels <= 6 && base >= 1 &&
         ((long long)base << levels) <= 4096;
}

namespace {

// The paper-form U-Net with its 3x3 layers on the tensor cores: each is a
// stride-1 implicit GEMM of conv_tc_kernel (LK_CONV1) over NHWC fp32
// activations in the split-tf32 product, with batch normalisation folded
// into the weights and bias, LeakyReLU in the epilogue, and a decoder's
// concatenated input read from its two tensors (upsampled deeper features,
// then the level's encoder output) by two tensor maps -- no copy.  Pooling,
// upsampling, the input staging and the 1x1 head are NHWC kernels of their
// own (unet.cu).  Weights are folded and packed on every call (the caller
// owns the parameters).
drc_status unet_forward_tc(drc_ctx *c, const UnetShape &u, const float *params, const float *in, float *out, int N,
                           int H, int W, void *workspace, cudaStream_t st) {
  Tracer *tr = &c->tracer;
  UnetTcBufs b;
  unet_tc_carve(u, N, H, W, static_cast<char *>(workspace), &b);
  const std::vector<UnetLayer> T = unet_layer_table(u);
  const int cs = unet_tc_in_channels(u);
  // the 3x3 layers as GEMM layers, their packed tiles laid out like the
  // autoencoder's
  // Accumulation in chunks of one K block (32 input channels of a tap) on
  // every layer: the tensor core's own fp32 accumulation loses about an ulp
  // of the running sum per MMA, so one accumulator over this network's
  // reductions (up to 216 K blocks, 6912 terms) measured 1.6e-3 max floored
  // relative error at the paper-size output (normwise 4.8e-5); added into an
  // fp32 running sum every K block, at the level of a plain float32
  // evaluation.  The running sum and two chunk accumulators share tensor
  // memory with the A stages, which caps the tiles at 128 columns.
  constexpr int kFoldKb = 1, kFoldAbove = kFoldKb;
  std::vector<Layer> Ls;
  std::vector<int> kfold;
  for (size_t i = 0; i < T.size(); ++i) {
    const UnetLayer &d = T[i];
    if (d.kind == 2) continue;
    Layer L;
    memset(&L, 0, sizeof L);
    L.kind = LK_CONV1;
    L.prec = PREC_TF32X3;
    L.Cin_raw = d.cin;
    L.Cin = i == 0 ? cs : d.cin;
    L.Cout = d.cout;
    L.num_phases = 1;
    PhaseDesc &pd = L.ph[0];
    pd.ntaps = 9;
    for (int t = 0; t < 9; ++t) {
      pd.u[t] = pd.dy[t] = (signed char)(t / 3);
      pd.v[t] = pd.dx[t] = (signed char)(t % 3);
    }
    pd.num_kb = ceil_div(9ll * L.Cin, bke_of(PREC_TF32X3));
    const bool fold = pd.num_kb > kFoldAbove;
    kfold.push_back(fold ? kFoldKb : 0);
    set_bn(L, fold && L.Cout > KFOLD_MAX_BN ? KFOLD_MAX_BN : pick_bn(L.Cout));
    snprintf(L.name, sizeof L.name, "unet conv %d", (int)i);
    Ls.push_back(L);
  }
  layout_packs(Ls);
  cudaError_t e = unet_fold_conv_form(u, params, b.fold, st, tr);
  if (e != cudaSuccess) return cuda_fail(c, e, "unet fold");
  for (size_t i = 0; i < Ls.size(); ++i) {
    const Layer &L = Ls[i];
    PackArgs p;
    memset(&p, 0, sizeof p);
    p.kind = L.kind;
    p.wraw = b.fold + T[i].dst;
    p.Cin = L.Cin;
    p.Cin_raw = L.Cin_raw;
    p.Cout = L.Cout;
    p.BN = L.BN;
    p.n_tiles = L.n_tiles;
    p.num_phases = 1;
    p.ph[0] = L.ph[0];
    p.B = b.B;
    p.B_lo = b.B_lo;
    p.total_chunks = (long long)(L.pack_bytes / 16);
    DRC_TRACED(tr, "weight pack", st, e = launch_pack(p, PREC_TF32X3, st));
    if (e != cudaSuccess) return cuda_fail(c, e, "unet weight packing");
  }
  if ((e = launch_unet_stage_nhwc(in, N, u.cin, (long long)H * W, cs, b.in, st, tr)) != cudaSuccess)
    return cuda_fail(c, e, "unet input staging");
  size_t li = 0;
  bool head_fused = false;
  // one 3x3 layer: x (and x2 after its C1 channels) at h x w -> y; the last
  // one takes the 1x1 head into its epilogue where its tile holds whole rows
  auto conv = [&](const float *x, const float *x2, int C1, int h, int w, float *y) -> drc_status {
    const Layer &L = Ls[li];
    ConvArgs a;
    fill_common(c, L, b.B, b.B_lo, a);
    a.N = N;
    a.x = x;
    a.x2 = x2;
    a.C1 = x2 ? C1 : 0;
    a.y = y;
    a.Hin = a.Hrow = a.Hout = h;
    a.Win = a.Wrow = a.Wout = w;
    a.Cin = L.Cin;
    a.Cout = L.Cout;
    a.relu = 1;
    a.slope = 0.01f;  // LeakyReLU
    a.bias = b.fold + T[li].dst + 9 * (size_t)T[li].cin * T[li].cout;
    a.M = (int)((long long)N * h * w);
    a.m_tiles = ceil_div(a.M, BM);
    a.kfold = kfold[li];
    plan_operand(PREC_TF32X3, a);
    if (a.prod_mode != PROD_TMA_TMEM)
      return fail(c, DRC_ERR_CUDA, "unet layer %zu: no tensor map for the A operand", li);
    if (li + 1 == Ls.size() && a.y_tma && a.n_tiles == 1 && u.cout <= KHEAD_MAX) {
      a.head_w = b.fold + T.back().dst;  // [cout][base], then the bias
      a.head_out = out;
      a.head_cout = u.cout;
      head_fused = true;
    }
    cudaError_t le;
    DRC_TRACED(tr, L.name, st, le = launch_conv(a, PREC_TF32X3, c->num_sms, st));
    if (le != cudaSuccess) return cuda_fail(c, le, "unet layer launch");
    ++li;
    return DRC_OK;
  };
  drc_status s;
  int ci = cs;
  const float *x = b.in;
  for (int l = 0; l <= u.levels; ++l) {
    const int h = H >> l, w = W >> l, ch = u.base << l;
    if (l > 0) {
      if ((e = launch_unet_pool_nhwc(b.enc[l - 1], N, h * 2, w * 2, ci, b.pool[l], st, tr)) != cudaSuccess)
        return cuda_fail(c, e, "unet pool");
      x = b.pool[l];
    }
    if ((s = conv(x, nullptr, 0, h, w, b.enc_a[l])) != DRC_OK) return s;
    if ((s = conv(b.enc_a[l], nullptr, 0, h, w, b.enc[l])) != DRC_OK) return s;
    ci = ch;
  }
  const float *d = b.enc[u.levels];
  for (int l = u.levels - 1; l >= 0; --l) {
    const int h = H >> l, w = W >> l, ch = u.base << l;
    if ((e = launch_unet_up_nhwc(d, N, h / 2, w / 2, 2 * ch, b.up[l], st, tr)) != cudaSuccess)
      return cuda_fail(c, e, "unet upsampling");
    if ((s = conv(b.up[l], b.enc[l], 2 * ch, h, w, b.dec_a[l])) != DRC_OK) return s;
    if ((s = conv(b.dec_a[l], nullptr, 0, h, w, b.dec[l])) != DRC_OK) return s;
    d = b.dec[l];
  }
  const UnetLayer &hd = T.back();
  if (!head_fused &&
      (e = launch_unet_head_nhwc(d, N, (long long)H * W, u.base, b.fold + hd.dst, u.cout, out, st, tr)) != cudaSuccess)
    return cuda_fail(c, e, "unet head");
  return DRC_OK;
}

}  // namespace

int drc_unet_tensor_cores(int in_ch, int out_ch, int base, int levels, int H, int W) {
  if (!unet_shape_ok(in_ch, out_ch, base, levels) || H < 1 || W < 1 || H % (1 << levels) || W % (1 << levels))
    return 0;
  return unet_tc_shape_ok(UnetShape{in_ch, out_ch, base, levels}, H, W) ? 1 : 0;
}

size_t drc_unet_param_count(int in_ch, int out_ch, int base, int levels) {
  if (!unet_shape_ok(in_ch, out_ch, base, levels)) return 0;
  return unet_param_count(UnetShape{in_ch, out_ch, base, levels});
}

size_t drc_unet_workspace_bytes(int in_ch, int out_ch, int base, int levels, int N, int H, int W) {
  if (!unet_shape_ok(in_ch, out_ch, base, levels) || N < 0 || H < 1 || W < 1 || H % (1 << levels) ||
      W % (1 << levels))
    return 0;
  const UnetShape u{in_ch, out_ch, base, levels};
  const size_t simt = unet_workspace_bytes(u, N, H, W);
  if (!unet_tc_shape_ok(u, H, W)) return simt;
  const size_t tc = unet_tc_carve(u, N, H, W, nullptr, nullptr);
  return tc > simt ? tc : simt;
}

drc_status drc_unet_forward(drc_ctx *c, int in_ch, int out_ch, int base, int levels, const float *params,
                            const float *in, float *out, int N, int H, int W, void *workspace, size_t workspace_bytes,
                            void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (!unet_shape_ok(in_ch, out_ch, base, levels))
    return fail(c, DRC_ERR_INVALID_ARG, "bad network in_ch=%d out_ch=%d base=%d levels=%d", in_ch, out_ch, base, levels);
  if (N < 0 || H < 1 || W < 1 || H % (1 << levels) || W % (1 << levels))
    return fail(c, DRC_ERR_INVALID_ARG, "maps must be multiples of 2^levels (N=%d H=%d W=%d)", N, H, W);
  const long long widest = 3LL * base > in_ch ? 3LL * base : in_ch;
  if ((long long)N * H * W * widest >= (1ll << 31))
    return fail(c, DRC_ERR_INVALID_ARG, "activations must stay below 2^31 elements");
  const UnetShape u{in_ch, out_ch, base, levels};
  const size_t need = unet_workspace_bytes(u, N, H, W);
  if (workspace_bytes < need)
    return fail(c, DRC_ERR_INVALID_ARG, "workspace of %zu bytes, %zu needed (drc_unet_workspace_bytes)",
                workspace_bytes, need);
  if (N == 0) return DRC_OK;
  drc_status s;
  if ((s = check_dev(c, params, "params", false)) != DRC_OK) return s;
  if ((s = check_dev(c, in, "in", false)) != DRC_OK) return s;
  if ((s = check_dev(c, out, "out", false)) != DRC_OK) return s;
  if ((s = check_dev(c, workspace, "workspace", false)) != DRC_OK) return s;
  if (unet_tc_shape_ok(u, H, W))
    return unet_forward_tc(c, u, params, in, out, N, H, W, workspace, static_cast<cudaStream_t>(stream));
  const cudaError_t e = unet_forward(u, params, in, out, N, H, W, workspace, static_cast<cudaStream_t>(stream),
                                     &c->tracer);
  return e == cudaSuccess ? DRC_OK : cuda_fail(c, e, "unet forward");
}

drc_status drc_frame_host(drc_ctx *c, const float *maps_host, int N, int H, int W, unsigned flags,
                          const drc_caches *caches, const drc_gbuffer *gbuf_host, const drc_interp_params *prm,
                          float *rgb_host, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (!caches || !gbuf_host || !prm) return fail(c, DRC_ERR_INVALID_ARG, "NULL argument struct");
  if (N < 1) return fail(c, DRC_ERR_INVALID_ARG, "N must be >= 1");
  if (caches->n != N) return fail(c, DRC_ERR_INVALID_ARG, "caches->n (%d) must equal N (%d)", caches->n, N);
  if (prm->mode != DRC_INTERP_IRRADIANCE) return fail(c, DRC_ERR_INVALID_ARG, "the frame call blends payloads");
  if (flags & ~(unsigned)DRC_F_ENCODE_INPUT) return fail(c, DRC_ERR_INVALID_ARG, "flags: DRC_F_ENCODE_INPUT only");
  if (gbuf_host->width < 0 || gbuf_host->height < 0) return fail(c, DRC_ERR_INVALID_ARG, "negative G-buffer size");
  const long long P = (long long)gbuf_host->width * gbuf_host->height;
  if (!maps_host || (P > 0 && (!gbuf_host->nrm || !rgb_host || (prm->metric == DRC_METRIC_WORLD && !gbuf_host->pos))))
    return fail(c, DRC_ERR_INVALID_ARG, "NULL host buffer");
  if ((long long)N * H * W * 7 >= (1ll << 31) || P >= (1ll << 31) / 3)
    return fail(c, DRC_ERR_INVALID_ARG, "frame too large");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  // staging, copy stream and events (first use / growth)
  const size_t map_floats = (size_t)7 * H * W;
  if ((size_t)N * map_floats > c->fmaps_n) {
    ctx_free(c, c->d_fmaps);
    ctx_free(c, c->d_fout);
    ctx_free(c, c->d_fpay);
    c->d_fmaps = c->d_fout = c->d_fpay = nullptr;
    c->fmaps_n = 0;
    if ((e = ctx_malloc(c, &c->d_fmaps, (size_t)N * map_floats * 4)) != cudaSuccess ||
        (e = ctx_malloc(c, &c->d_fout, (size_t)N * 3 * H * W * 4)) != cudaSuccess ||
        (e = ctx_malloc(c, &c->d_fpay, (size_t)N * 3 * 4)) != cudaSuccess)
      return cuda_fail(c, e, "frame staging");
    c->fmaps_n = (size_t)N * map_floats;
  }
  if ((size_t)P > c->fgbuf_p) {
    ctx_free(c, c->d_fgpos);
    ctx_free(c, c->d_fgnrm);
    ctx_free(c, c->d_frgb);
    c->d_fgpos = c->d_fgnrm = c->d_frgb = nullptr;
    c->fgbuf_p = 0;
    if ((e = ctx_malloc(c, &c->d_fgpos, (size_t)P * 12)) != cudaSuccess ||
        (e = ctx_malloc(c, &c->d_fgnrm, (size_t)P * 12)) != cudaSuccess ||
        (e = ctx_malloc(c, &c->d_frgb, (size_t)P * 12)) != cudaSuccess)
      return cuda_fail(c, e, "frame staging");
    c->fgbuf_p = (size_t)P;
  }
  if (!c->fcopy) {
    if ((e = cudaStreamCreateWithFlags(&c->fcopy, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(c, e, "copy stream");
    for (cudaEvent_t *ev : {&c->fev_maps, &c->fev_gbuf, &c->fev_maps_free, &c->fev_gbuf_free})
      if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(c, e, "event");
    // nothing to wait for before the first call
    cudaEventRecord(c->fev_maps_free, st);
    cudaEventRecord(c->fev_gbuf_free, st);
  }
  // uploads: the maps (waiting only until the previous call's denoise has
  // read the staging, so they land under its interpolation), then the
  // G-buffer (after the previous call's interpolation, so it lands under this
  // call's denoise).  One denoise launch sequence over all N maps: splitting
  // it into chunks that start as they land measured slower (1024-map chunks
  // 2.65 against 2.35 ms per 4096-map frame), and in a frame loop the maps
  // are already there.
  cudaStreamWaitEvent(c->fcopy, c->fev_maps_free, 0);
  if ((e = cudaMemcpyAsync(c->d_fmaps, maps_host, (size_t)N * map_floats * 4, cudaMemcpyHostToDevice, c->fcopy)) !=
      cudaSuccess)
    return cuda_fail(c, e, "map upload");
  cudaEventRecord(c->fev_maps, c->fcopy);
  if (P > 0) {
    cudaStreamWaitEvent(c->fcopy, c->fev_gbuf_free, 0);
    if (prm->metric == DRC_METRIC_WORLD &&
        (e = cudaMemcpyAsync(c->d_fgpos, gbuf_host->pos, (size_t)P * 12, cudaMemcpyHostToDevice, c->fcopy)) !=
            cudaSuccess)
      return cuda_fail(c, e, "G-buffer upload");
    if ((e = cudaMemcpyAsync(c->d_fgnrm, gbuf_host->nrm, (size_t)P * 12, cudaMemcpyHostToDevice, c->fcopy)) !=
        cudaSuccess)
      return cuda_fail(c, e, "G-buffer upload");
    cudaEventRecord(c->fev_gbuf, c->fcopy);
  }
  // compute on the caller's stream
  drc_status s;
  cudaStreamWaitEvent(st, c->fev_maps, 0);
  if ((s = drc_denoise(c, c->d_fmaps, c->d_fout, c->d_fpay, N, H, W, flags, stream)) != DRC_OK) return s;
  cudaEventRecord(c->fev_maps_free, st);
  if (P > 0) {
    cudaStreamWaitEvent(st, c->fev_gbuf, 0);
    drc_caches cc = *caches;
    cc.payload = c->d_fpay;
    drc_gbuffer gd = *gbuf_host;
    gd.pos = c->d_fgpos;
    gd.nrm = c->d_fgnrm;
    gd.dir = nullptr;
    if ((s = drc_interpolate(c, &cc, &gd, prm, c->d_frgb, stream)) != DRC_OK) return s;
    cudaEventRecord(c->fev_gbuf_free, st);
    if ((e = cudaMemcpyAsync(rgb_host, c->d_frgb, (size_t)P * 12, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_fail(c, e, "image download");
  }
  return DRC_OK;
}

drc_status drc_get_status(drc_ctx *c, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  int v = 0;
  e = cudaMemcpy(&v, c->d_status, sizeof v, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "status read");
  if (v != 0) {
    cudaMemset(c->d_status, 0, sizeof(int));
    return fail(c, (drc_status)v, "device-side error %d latched (%s)", v,
                v == DRC_ERR_TIMEOUT ? "a bounded wait ran out" : "a plan pass count was out of range");
  }
  return DRC_OK;
}

const char *drc_last_error(drc_ctx *c) { return c ? c->err.c_str() : "NULL context"; }

drc_status drc_set_memory_limit(drc_ctx *c, size_t bytes) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  c->mem_limit = bytes;
  return DRC_OK;
}

size_t drc_memory_in_use(const drc_ctx *c) { return c ? c->mem_used : 0; }

drc_status drc_get_weights(drc_ctx *c, float *out, int out_on_device, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (!out) return fail(c, DRC_ERR_INVALID_ARG, "out is NULL");
  if (!c->weights_set) return fail(c, DRC_ERR_INVALID_ARG, "weights were never set");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (out_on_device) {
    if (!is_device_ptr(out, c->device))
      return fail(c, DRC_ERR_INVALID_ARG, "out_on_device set but out is not device memory");
    e = cudaMemcpyAsync(out, c->d_wraw, c->n_floats * sizeof(float), cudaMemcpyDeviceToDevice, st);
  } else {
    e = cudaMemcpyAsync(out, c->d_wraw, c->n_floats * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  return e == cudaSuccess ? DRC_OK : cuda_fail(c, e, "weight read-back");
}



namespace {

// Make per-layer tile widths and A paths current: lay the packed operands
// out again (a larger buffer where the new widths pad more) and repack.
drc_status apply_tiles(drc_ctx *c, std::vector<Layer> &Ls, const std::vector<int> &modes, cudaStream_t st) {
  drc_status s = DRC_OK;
  cudaError_t e;
  {
    const size_t need = layout_packs(Ls);
    if (need > c->pack_total) {  // a narrower tile can pad the packed image differently
      uint8_t *B = nullptr, *B_lo = nullptr;
      e = ctx_malloc(c, &B, need);
      if (e == cudaSuccess && c->prec == PREC_TF32X3) e = ctx_malloc(c, &B_lo, need);
      if (e != cudaSuccess) {
        ctx_free(c, B);
        s = cuda_fail(c, e, "autotune operands");
      } else {
        cudaStreamSynchronize(st);
        ctx_free(c, c->d_pack);
        ctx_free(c, c->d_pack_lo);
        c->d_pack = B;
        c->d_pack_lo = B_lo;
        c->pack_total = need;
      }
    }
  }
  if (s == DRC_OK) {
    c->layers = Ls;
    c->modes = modes;
    s = pack_all(c, st);
  }
  return s;
}

}  // namespace

drc_status drc_autotune(drc_ctx *c, int N, int H, int W) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  const int S = c->cfg.num_stages;
  if (N < 1 || H < (1 << S) || W < (1 << S) || H % (1 << S) || W % (1 << S) ||
      (long long)N * H * W * 7 >= (1ll << 31))
    return fail(c, DRC_ERR_INVALID_ARG, "autotune shape N=%d H=%d W=%d is not a valid denoise batch", N, H, W);
  if (!c->weights_set) return fail(c, DRC_ERR_INVALID_ARG, "weights were never set");
  // the timing launches write the context's workspace and the repack its
  // packed operands: calls still in flight on any stream finish first
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "device synchronize");
  drc_status s = ensure_act(c, N, H, W);
  if (s != DRC_OK) return s;
  cudaStream_t st = nullptr;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune stream");
  Chain ch;
  carve_chain(c, c->d_act, N, H, W, ch);
  std::vector<Layer> Ls = c->layers;
  std::vector<int> modes = c->modes;
  s = autotune_layers(c, Ls, modes, ch, st, true);
  if (s == DRC_OK) s = apply_tiles(c, Ls, modes, st);
  if (s == DRC_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) s = cuda_fail(c, e, "autotune");
  cudaStreamDestroy(st);
  return s;
}

drc_status drc_calibrate(drc_ctx *c, const float *in, int N, int H, int W, unsigned flags, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (c->prec != PREC_FP8) return fail(c, DRC_ERR_UNSUPPORTED, "calibration applies to FP8 contexts only");
  const int S = c->cfg.num_stages;
  if (flags & ~(DRC_F_ENCODE_INPUT | DRC_F_DECODE_OUTPUT))
    return fail(c, DRC_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
  if (N < 1 || H < (1 << S) || W < (1 << S) || H % (1 << S) || W % (1 << S) ||
      (long long)N * H * W * 7 >= (1ll << 31))
    return fail(c, DRC_ERR_INVALID_ARG, "calibration batch N=%d H=%d W=%d is not a valid denoise batch", N, H, W);
  if (!c->weights_set) return fail(c, DRC_ERR_INVALID_ARG, "weights were never set");
  drc_status s;
  if ((s = check_dev(c, in, "in", false)) != DRC_OK) return s;
  if ((s = ensure_act(c, N, H, W)) != DRC_OK) return s;
  float *out = nullptr;
  cudaError_t e = ctx_malloc(c, &out, (size_t)N * 3 * H * W * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(c, e, "calibration output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Chain ch;
  carve_chain(c, c->d_act, N, H, W, ch);
  std::vector<unsigned> amax(c->n_bscales);
  // Two passes: the first runs with the current scales, the second with the
  // scales the first measured, so every layer sees well-quantised inputs.
  for (int pass = 0; pass < 2 && s == DRC_OK; ++pass) {
    if ((e = cudaMemsetAsync(c->d_amax, 0, c->n_bscales * sizeof(unsigned), st)) != cudaSuccess) {
      s = cuda_fail(c, e, "calibration clear");
      break;
    }
    c->calibrating = true;
    s = run_chain(c, c->layers, c->d_pack, c->d_pack_lo, &c->modes, ch, in, out, nullptr, flags, st, &c->tracer,
                  nullptr);
    c->calibrating = false;
    if (s != DRC_OK) break;
    if ((e = cudaMemcpyAsync(amax.data(), c->d_amax, amax.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      s = cuda_fail(c, e, "calibration read");
      break;
    }
    // layer li + 1 consumes layer li's output: its input scale for channel
    // ch is that channel's measured maximum over 448 (the e4m3 maximum), with
    // one binade of headroom for batches brighter than this one
    std::vector<float> qinv(c->n_scales);
    for (size_t li = 0; li + 1 < c->layers.size(); ++li) {
      const Layer &P = c->layers[li], &Q = c->layers[li + 1];
      for (int ch2 = 0; ch2 < Q.Cin; ++ch2) {
        float m;
        memcpy(&m, &amax[P.bs_off + ch2], sizeof m);
        c->h_inscale[Q.sc_off + ch2] = m > 0.f && std::isfinite(m) ? 2.0f * m / 448.0f : 1.0f;
      }
    }
    for (size_t i = 0; i < c->n_scales; ++i) qinv[i] = 1.0f / c->h_inscale[i];
    e = cudaMemcpy(c->d_inscale, c->h_inscale.data(), c->n_scales * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_qinv, qinv.data(), c->n_scales * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      s = cuda_fail(c, e, "calibration upload");
      break;
    }
    s = pack_all(c, st);  // fold the new input scales into the e4m3 weights
    ++c->weights_version;
  }
  cudaStreamSynchronize(st);
  ctx_free(c, out);
  cudaGetLastError();
  return s;
}

drc_status drc_describe_layer(drc_ctx *c, int layer, int *bn, int *a_path) {
  if (!c || layer < 0 || layer >= (int)c->layers.size()) return DRC_ERR_INVALID_ARG;
  const Layer &L = c->layers[layer];
  if (bn) *bn = L.kind == LK_HEAD ? 0 : L.BN;
  if (a_path) *a_path = c->modes[layer];
  return DRC_OK;
}

drc_status drc_plan_create(drc_ctx *c, const drc_size_class *classes, int n_classes, unsigned flags,
                           drc_plan **out) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (!out) return fail(c, DRC_ERR_INVALID_ARG, "plan output pointer is NULL");
  *out = nullptr;
  if (!classes || n_classes < 1 || n_classes > kMaxClasses)
    return fail(c, DRC_ERR_INVALID_ARG, "need 1..%d size classes", kMaxClasses);
  if (flags & ~DRC_PLAN_AUTOTUNE) return fail(c, DRC_ERR_INVALID_ARG, "unknown plan flags 0x%x", flags);
  if (!c->weights_set) return fail(c, DRC_ERR_INVALID_ARG, "weights were never set");
  const int S = c->cfg.num_stages;
  for (int k = 0; k < n_classes; ++k) {
    const drc_size_class &q = classes[k];
    if (q.H < (1 << S) || q.W < (1 << S) || q.H % (1 << S) || q.W % (1 << S) || q.H > 256)
      return fail(c, DRC_ERR_INVALID_ARG, "class %d: H, W must be multiples of 2^S = %d, H <= 256", k, 1 << S);
    if (q.max_maps < 1 || (long long)q.max_maps * q.H * q.W * 7 >= (1ll << 31))
      return fail(c, DRC_ERR_INVALID_ARG, "class %d: max_maps must be >= 1 and max_maps*7*H*W < 2^31", k);
  }
  // the plan packs from the context's weights on its own stream: updates in
  // flight on any stream land first
  if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "device synchronize");
  drc_plan *p = new (std::nothrow) drc_plan();
  if (!p) return fail(c, DRC_ERR_OOM, "plan");
  p->ctx = c;
  p->flags = flags;
  p->cls.assign(classes, classes + n_classes);
  size_t act_total = 0;
  std::vector<size_t> act_off(n_classes);
  for (int k = 0; k < n_classes; ++k) {
    act_off[k] = act_total;
    act_total += (act_bytes_for(c, classes[k].max_maps, classes[k].H, classes[k].W) + 255) & ~(size_t)255;
  }
  cudaError_t e = ctx_malloc(c, &p->d_act, act_total);
  if (e == cudaSuccess) e = cudaMemset(p->d_act, 0, act_total);
  if (e == cudaSuccess) e = ctx_malloc(c, &p->d_slots, n_classes * sizeof(PassSlot));
  if (e == cudaSuccess) e = cudaMemset(p->d_slots, 0, n_classes * sizeof(PassSlot));
  if (e != cudaSuccess) {
    drc_status s = cuda_fail(c, e, "plan buffers");
    plan_free(p);
    return s;
  }
  p->chains.resize(n_classes);
  p->layers.assign(n_classes, c->layers);
  p->modes.assign(n_classes, c->modes);
  for (auto &m : p->modes)  // plans keep the four-GEMM decoders (their own tiles and packing)
    for (int &x : m)
      if (is_paired(x)) x = -1;
  p->pack.assign(n_classes, nullptr);
  p->pack_lo.assign(n_classes, nullptr);
  cudaStream_t cs = nullptr;
  drc_status s = DRC_OK;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) s = cuda_fail(c, e, "plan stream");
  for (int k = 0; s == DRC_OK && k < n_classes; ++k) {
    carve_chain(c, static_cast<char *>(p->d_act) + act_off[k], classes[k].max_maps, classes[k].H, classes[k].W,
                p->chains[k]);
    if (flags & DRC_PLAN_AUTOTUNE) s = autotune_layers(c, p->layers[k], p->modes[k], p->chains[k], cs);
    if (s != DRC_OK) break;
    const size_t bytes = layout_packs(p->layers[k]);
    e = ctx_malloc(c, &p->pack[k], bytes);
    if (e == cudaSuccess && c->prec == PREC_TF32X3) e = ctx_malloc(c, &p->pack_lo[k], bytes);
    if (e != cudaSuccess) s = cuda_fail(c, e, "plan operands");
  }
  if (s == DRC_OK) s = plan_pack(p, cs);
  if (s == DRC_OK && (e = cudaStreamSynchronize(cs)) != cudaSuccess) s = cuda_fail(c, e, "plan packing");
  for (int k = 0; k < n_classes; ++k) {
    p->chains[k].count = &p->d_slots[k].count;
    p->chains[k].slot = &p->d_slots[k];
  }
  if (s == DRC_OK) s = refresh_head_weights(c, cs);
  if (s == DRC_OK) s = plan_capture(p, cs);
  if (cs) cudaStreamDestroy(cs);
  if (s != DRC_OK) {
    plan_free(p);
    return s;
  }
  *out = p;
  return DRC_OK;
}

drc_status drc_plan_launch(drc_plan *p, const int *counts, const float *const *in, float *const *out,
                           float *const *payload, unsigned flags, void *stream) {
  if (!p) return DRC_ERR_INVALID_ARG;
  drc_ctx *c = p->ctx;
  c->err.clear();
  const unsigned known = DRC_F_ENCODE_INPUT | DRC_F_DECODE_OUTPUT;
  if (flags & ~known) return fail(c, DRC_ERR_INVALID_ARG, "unknown flags 0x%x", flags & ~known);
  if (!in || !out) return fail(c, DRC_ERR_INVALID_ARG, "in and out arrays are required");
  drc_status s;
  if ((s = check_dev(c, counts, "counts", false)) != DRC_OK) return s;
  SlotUpdate u;
  memset(&u, 0, sizeof u);
  u.n = (int)p->cls.size();
  u.flags = flags;
  for (int k = 0; k < u.n; ++k) {
    if ((s = check_dev(c, in[k], "in[k]", false)) != DRC_OK) return s;
    if ((s = check_dev(c, out[k], "out[k]", false)) != DRC_OK) return s;
    if (payload && (s = check_dev(c, payload[k], "payload[k]", true)) != DRC_OK) return s;
    u.max_maps[k] = p->cls[k].max_maps;
    u.in[k] = in[k];
    u.out[k] = out[k];
    u.payload[k] = payload ? payload[k] : nullptr;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p->weights_version != c->weights_version && (s = plan_pack(p, st)) != DRC_OK) return s;
  if (p->graph_version != c->weights_version) {
    if ((s = refresh_head_weights(c, st)) != DRC_OK) return s;
    cudaStream_t cs = nullptr;
    cudaError_t ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "plan stream");
    s = plan_capture(p, cs);
    cudaStreamDestroy(cs);
    if (s != DRC_OK) return s;
  }
  cudaError_t e;
  DRC_TRACED(&c->tracer, "plan slots", st,
             (set_slots_kernel<<<1, 32, 0, st>>>(u, counts, p->d_slots, c->d_status), e = cudaGetLastError()));
  if (e != cudaSuccess) return cuda_fail(c, e, "plan slots");
  DRC_TRACED(&c->tracer, "plan graph", st, e = cudaGraphLaunch(p->exec, st));
  if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
  c->tracer.add_launches(p->kernels_per_launch - 1);  // the graph's kernels (one counted above)
  return DRC_OK;
}

drc_status drc_plan_describe(drc_plan *p, int k, int layer, int *bn, int *a_path) {
  if (!p || k < 0 || k >= (int)p->cls.size() || layer < 0 || layer >= (int)p->layers[k].size())
    return DRC_ERR_INVALID_ARG;
  const Layer &L = p->layers[k][layer];
  if (bn) *bn = L.kind == LK_HEAD ? 0 : L.BN;
  if (a_path) *a_path = p->modes[k][layer];
  return DRC_OK;
}

drc_status drc_plan_destroy(drc_plan *p) {
  if (!p) return DRC_ERR_INVALID_ARG;
  plan_free(p);
  return DRC_OK;
}

drc_status drc_launch_count(drc_ctx *c, unsigned long long *count) {
  if (!c || !count) return DRC_ERR_INVALID_ARG;
  *count = c->tracer.launches();
  return DRC_OK;
}

drc_status drc_set_timing(drc_ctx *c, int enable) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->tracer.set_timing(enable != 0);
  return DRC_OK;
}

drc_status drc_read_timing(drc_ctx *c, drc_kernel_time *out, int capacity, int *n_out) {
  if (!c || !n_out || capacity < 0 || (capacity > 0 && !out)) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  std::vector<Tracer::Total> t = c->tracer.drain();
  int n = 0;
  for (const auto &x : t) {
    if (n >= capacity) break;
    memset(&out[n], 0, sizeof out[n]);
    snprintf(out[n].name, sizeof out[n].name, "%s", x.name.c_str());
    out[n].launches = x.launches;
    out[n].total_ms = x.ms;
    ++n;
  }
  *n_out = n;
  if ((int)t.size() > capacity) return fail(c, DRC_ERR_INVALID_ARG, "capacity %d < %zu kernels", capacity, t.size());
  return DRC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- checkpoint
namespace {

const char *prec_name(int prec) { return prec == PREC_TF32X3 ? "fp32" : (prec == PREC_BF16 ? "bf16" : "fp8"); }

// The architecture part of a header: what a checkpoint or a tile choice is
// tied to (precision is not part of it: the weights are fp32 masters).
std::string arch_json(const drc_config &g) {
  std::string w;
  for (int i = 0; i < g.num_stages; ++i) w += (i ? "," : "") + std::to_string(g.widths[i]);
  char buf[256];
  snprintf(buf, sizeof buf, "\"in_channels\": %d, \"out_channels\": %d, \"widths\": [%s], \"out_relu\": %d, "
                            "\"exposure\": %.9g",
           g.in_channels, g.out_channels, w.c_str(), g.out_relu ? 1 : 0, (double)g.exposure);
  return buf;
}

// Whether header h describes the same network as g; *why says how it differs.
bool arch_matches(const FlatJson &h, const drc_config &g, std::string *why) {
  double ic = -1, oc = -1, orl = -1, ex = -1;
  std::vector<double> w;
  if (!h.num("in_channels", &ic) || !h.num("out_channels", &oc) || !h.num("out_relu", &orl) ||
      !h.num("exposure", &ex) || !h.nums("widths", &w)) {
    *why = "header lacks the network description";
    return false;
  }
  bool same = (int)ic == g.in_channels && (int)oc == g.out_channels && (int)w.size() == g.num_stages &&
              ((int)orl != 0) == (g.out_relu != 0) && (float)ex == g.exposure;
  for (size_t i = 0; same && i < w.size(); ++i) same = (int)w[i] == g.widths[i];
  if (!same) *why = "it was written for another network (channels, widths, out_relu or exposure differ)";
  return same;
}

}  // namespace

drc_status drc_save_checkpoint(drc_ctx *c, const char *path, const float *adam_m, const float *adam_v,
                               int adam_step, void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (!path || !*path) return fail(c, DRC_ERR_INVALID_ARG, "path is empty");
  if (!c->weights_set) return fail(c, DRC_ERR_INVALID_ARG, "weights were never set");
  if ((adam_m == nullptr) != (adam_v == nullptr))
    return fail(c, DRC_ERR_INVALID_ARG, "adam_m and adam_v must both be given or both be NULL");
  if (adam_step < 0) return fail(c, DRC_ERR_INVALID_ARG, "adam_step must be >= 0");
  drc_status s;
  if (adam_m && ((s = check_dev(c, adam_m, "adam_m", false)) != DRC_OK || (s = check_dev(c, adam_v, "adam_v", false)) != DRC_OK))
    return s;
  const size_t n = c->n_floats;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<float> w(n), m(adam_m ? n : 0), v(adam_v ? n : 0);
  cudaError_t e = cudaMemcpyAsync(w.data(), c->d_wraw, n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && adam_m) e = cudaMemcpyAsync(m.data(), adam_m, n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && adam_v) e = cudaMemcpyAsync(v.data(), adam_v, n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint read-back");
  uint64_t h = fnv1a64(w.data(), n * 4);
  if (adam_m) h = fnv1a64(v.data(), n * 4, fnv1a64(m.data(), n * 4, h));
  char head[160];
  snprintf(head, sizeof head, "\"n_floats\": %zu, \"adam\": %d, \"adam_step\": %d, \"payload_bytes\": %zu, "
                              "\"fnv1a64\": \"%016llx\"}",
           n, adam_m ? 1 : 0, adam_step, n * 4 * (adam_m ? 3 : 1), (unsigned long long)h);
  const std::string header = "{\"format\": \"drc-checkpoint\", \"version\": 1, " + arch_json(c->cfg) + ", " + head;
  std::vector<std::pair<const void *, size_t>> blobs{{w.data(), n * 4}};
  if (adam_m) {
    blobs.push_back({m.data(), n * 4});
    blobs.push_back({v.data(), n * 4});
  }
  if (!write_file_atomic(path, header, blobs))
    return fail(c, DRC_ERR_INVALID_ARG, "cannot write %s: %s", path, strerror(errno));
  return DRC_OK;
}

drc_status drc_load_checkpoint(drc_ctx *c, const char *path, float *adam_m, float *adam_v, int *adam_step,
                               void *stream) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (!path || !*path) return fail(c, DRC_ERR_INVALID_ARG, "path is empty");
  if ((adam_m == nullptr) != (adam_v == nullptr))
    return fail(c, DRC_ERR_INVALID_ARG, "adam_m and adam_v must both be given or both be NULL");
  drc_status s;
  if (adam_m && ((s = check_dev(c, adam_m, "adam_m", false)) != DRC_OK || (s = check_dev(c, adam_v, "adam_v", false)) != DRC_OK))
    return s;
  std::string data;
  if (!read_file(path, &data)) return fail(c, DRC_ERR_INVALID_ARG, "cannot read %s: %s", path, strerror(errno));
  const size_t nl = data.find('\n');
  FlatJson h;
  std::string fmt;
  double ver = 0, nf = 0, has_adam = 0, step = 0, pbytes = 0;
  std::string sum, why;
  if (nl == std::string::npos || !parse_flat_json(data.substr(0, nl), &h) || !h.str("format", &fmt) ||
      fmt != "drc-checkpoint" || !h.num("version", &ver) || !h.num("n_floats", &nf) || !h.num("adam", &has_adam) ||
      !h.num("adam_step", &step) || !h.num("payload_bytes", &pbytes) || !h.str("fnv1a64", &sum))
    return fail(c, DRC_ERR_INVALID_ARG, "%s is not a checkpoint of this library", path);
  if ((int)ver != 1) return fail(c, DRC_ERR_UNSUPPORTED, "%s: checkpoint version %d", path, (int)ver);
  if (!arch_matches(h, c->cfg, &why)) return fail(c, DRC_ERR_INVALID_ARG, "%s: %s", path, why.c_str());
  const size_t n = c->n_floats;
  const size_t want = n * 4 * (has_adam != 0 ? 3 : 1);
  if ((size_t)nf != n || (size_t)pbytes != want || data.size() - nl - 1 != want)
    return fail(c, DRC_ERR_INVALID_ARG, "%s: payload of %zu bytes, %zu expected", path, data.size() - nl - 1, want);
  const char *pay = data.data() + nl + 1;
  char hex[17];
  snprintf(hex, sizeof hex, "%016llx", (unsigned long long)fnv1a64(pay, want));
  if (sum != hex) return fail(c, DRC_ERR_INVALID_ARG, "%s: checksum mismatch (the file is damaged)", path);
  if (adam_m && has_adam == 0) return fail(c, DRC_ERR_INVALID_ARG, "%s holds no optimizer state", path);
  std::vector<float> w(n);
  memcpy(w.data(), pay, n * 4);
  if ((s = drc_set_weights(c, w.data(), 0, stream)) != DRC_OK) return s;
  if (adam_m) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(adam_m, pay + n * 4, n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(adam_v, pay + 2 * n * 4, n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host copy is freed on return
    if (e != cudaSuccess) return cuda_fail(c, e, "optimizer state upload");
  }
  if (adam_step) *adam_step = (int)step;
  return DRC_OK;
}

// ----------------------------------------------------------- autotune cache
drc_status drc_autotune_cached(drc_ctx *c, int N, int H, int W, const char *path, int *from_cache) {
  if (!c) return DRC_ERR_INVALID_ARG;
  c->err.clear();
  if (from_cache) *from_cache = 0;
  if (!path || !*path) return fail(c, DRC_ERR_INVALID_ARG, "path is empty");
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "device properties");
  const int cc = prop.major * 10 + prop.minor;
  // the entries of this device, network, precision and batch shape
  std::string data;
  if (read_file(path, &data)) {
    std::vector<Layer> best;
    std::vector<int> best_modes;
    size_t pos = 0;
    while (pos < data.size()) {
      size_t end = data.find('\n', pos);
      if (end == std::string::npos) end = data.size();
      const std::string line = data.substr(pos, end - pos);
      pos = end + 1;
      FlatJson j;
      std::string fmt, dev, prec, why;
      double sms = 0, jcc = 0;
      std::vector<double> shape, tn, ap;
      if (!parse_flat_json(line, &j) || !j.str("format", &fmt) || fmt != "drc-autotune" || !j.str("device", &dev) ||
          !j.num("sms", &sms) || !j.num("cc", &jcc) || !j.str("precision", &prec) || !j.nums("shape", &shape) ||
          !j.nums("tile_n", &tn) || !j.nums("a_path", &ap))
        continue;  // not an entry (or damaged): skipped
      if (dev != prop.name || (int)sms != c->num_sms || (int)jcc != cc || prec != prec_name(c->prec) ||
          shape.size() != 3 || (int)shape[0] != N || (int)shape[1] != H || (int)shape[2] != W ||
          !arch_matches(j, c->cfg, &why) || tn.size() != c->layers.size() || ap.size() != c->layers.size())
        continue;
      // the choices must be ones drc_autotune can make for these layers
      std::vector<Layer> Ls = c->layers;
      std::vector<int> modes(Ls.size(), -1);
      bool ok = true;
      for (size_t li = 0; ok && li < Ls.size(); ++li) {
        if (Ls[li].kind == LK_HEAD) continue;
        const int bn = (int)tn[li], mode = (int)ap[li];
        bool bn_ok = false;
        for (int cand : bn_candidates(Ls[li])) bn_ok = bn_ok || cand == bn;
        const bool mode_ok = mode == -1 || (c->prec == PREC_TF32X3 && mode == PROD_TMA_CONVERT && bn <= 128) ||
                             (c->prec == PREC_TF32X3 && mode == PROD_CPASYNC && Ls[li].kind == LK_CONV && Ls[li].Cin == 8) ||
                             (is_paired(mode) && li < c->players.size() && c->players[li].kind == LK_CONVT);
        ok = bn_ok && mode_ok;
        if (ok) {
          set_bn(Ls[li], bn);
          modes[li] = mode;
        }
      }
      if (ok) {  // the last valid entry wins
        best = Ls;
        best_modes = modes;
      }
    }
    if (!best.empty()) {
      // the repack rewrites operands that calls in flight may be reading
      if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(c, e, "device synchronize");
      drc_status s = ensure_act(c, N, H, W);
      if (s != DRC_OK) return s;
      if (!c->weights_set) return fail(c, DRC_ERR_INVALID_ARG, "weights were never set");
      cudaStream_t st = nullptr;
      if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(c, e, "autotune stream");
      s = apply_tiles(c, best, best_modes, st);
      if (s == DRC_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) s = cuda_fail(c, e, "autotune cache");
      cudaStreamDestroy(st);
      if (s == DRC_OK && from_cache) *from_cache = 1;
      return s;
    }
  }
  drc_status s = drc_autotune(c, N, H, W);
  if (s != DRC_OK) return s;
  std::string tn, ap;
  for (size_t li = 0; li < c->layers.size(); ++li) {
    tn += (li ? "," : "") + std::to_string(c->layers[li].kind == LK_HEAD ? 0 : c->layers[li].BN);
    ap += (li ? "," : "") + std::to_string(c->modes[li]);
  }
  char buf[256];
  snprintf(buf, sizeof buf, "\"sms\": %d, \"cc\": %d, \"precision\": \"%s\", \"shape\": [%d,%d,%d], ", c->num_sms, cc,
           prec_name(c->prec), N, H, W);
  const std::string line = "{\"format\": \"drc-autotune\", \"version\": 1, \"device\": " + json_quote(prop.name) +
                           ", " + buf + arch_json(c->cfg) + ", \"tile_n\": [" + tn + "], \"a_path\": [" + ap + "]}";
  if (!append_line(path, line)) return fail(c, DRC_ERR_INVALID_ARG, "cannot append to %s: %s", path, strerror(errno));
  return DRC_OK;
}
