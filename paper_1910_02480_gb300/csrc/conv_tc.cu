// conv_tc.cu -- implicit-GEMM convolution / transposed convolution on the
// sm_103a tensor cores (tcgen05), the layers of the autoencoder of Sec. 3.3.
//
// One persistent CTA per SM walks a static list of (phase, M tile, N tile)
// output tiles.  A tile is D[128 x BN] = A[128 x K] * B[BN x K]^T with
//   rows of A  = output pixels (encoder) or input-resolution pixels of one
//                output parity phase (decoder), gathered on the fly
//                (implicit im2col, zero padding) by eight producer warps;
//   rows of B  = output channels; pre-packed weight tiles in the exact
//                shared-memory image (128-byte swizzle), fetched by one thread
//                with cp.async.bulk;
//   D          = fp32 accumulator in tensor memory, double buffered (when it
//                fits) so the epilogue of tile i overlaps the MMAs of tile i+1.
// Warp roles (16 warps): 0 = MMA issuer + TMEM owner, 1 = B loader,
// 4..7 = epilogue (TMEM lane quarters 0..3), 8..15 = A producers.
// FP32 parity uses the split-tf32 product: x = hi + lo with hi, lo tf32, and
// D += A_hi B_hi, C += A_hi B_lo + A_lo B_hi in two accumulators, summed in
// the epilogue (the dropped lo*lo term is below 2^-21 relative).  BF16 / FP8
// use one product per K step.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "conv_tc.cuh"
#include "drc_status.cuh"
#include "ptx.cuh"

namespace drc {

template <int PREC>
struct PrecTraits;
template <>
struct PrecTraits<PREC_TF32X3> {
  static constexpr int ELEM = 4;  // bytes per stored operand element
  static constexpr int KIND = KIND_TF32;
  static constexpr int SPLIT = 2;  // hi + lo copies of each operand tile
  using act_t = float;             // activation storage
};
template <>
struct PrecTraits<PREC_BF16> {
  static constexpr int ELEM = 2;
  static constexpr int KIND = KIND_F16;
  static constexpr int SPLIT = 1;
  using act_t = __nv_bfloat16;
};
template <>
struct PrecTraits<PREC_FP8> {
  static constexpr int ELEM = 1;
  static constexpr int KIND = KIND_F8;
  static constexpr int SPLIT = 1;
  using act_t = uint8_t;  // e4m3 activations, quantised per channel by the producing layer
};

constexpr int SMEM_BUDGET = 227 * 1024;
constexpr int SMEM_CTRL = 1024;  // barriers + TMEM slot, padded to the 1024-byte swizzle atom

__host__ __device__ inline int stage_bytes(int prec, int BN, int mode) {
  const int split = prec == PREC_TF32X3 ? 2 : 1;
  if (mode == PROD_TMA_TMEM) return split * BN * KROW_BYTES;  // A lives in tensor memory
  return split * (BM * KROW_BYTES + BN * KROW_BYTES);
}

// PROD_TMA_TMEM tensor-memory map: accumulators in columns [0, 256), A
// stages of 64 columns (tf32 hi 32 | lo 32) from column 256.  With
// accumulation chunks (ConvArgs::kfold) the accumulators are the running
// sum R [0, BN) and two chunk buffers [BN, 3 BN); above 256 columns of
// those (BN 128) the A stages shrink to two, from column 384.
constexpr int TS_STAGES = 4;
constexpr int RAW_MAX = 6;  // raw TMA slots at most (the control block's barrier arrays); 8 measured no faster
constexpr int TS_A_COL0 = 256;
__host__ __device__ inline int ts_a_col0(int BN, int fold) { return fold && 3 * BN > TS_A_COL0 ? 384 : TS_A_COL0; }
__host__ __device__ inline int ts_stages(int BN, int fold) { return (512 - ts_a_col0(BN, fold)) / 64; }

// Raw bytes of one operand row per K block, in the stored activation type
// (fp32 for the split-tf32 path, bf16 / e4m3 otherwise): one swizzle row.
__host__ __device__ inline int raw_row_bytes(int) { return 128; }

// Shared memory: MMA stages (A and B tiles) plus, except when the TMA writes
// the A tile itself, a ring of R raw slots; R = 3 keeps two K blocks of
// copies in flight beyond the one being converted, shrunk to 2 when 2 MMA
// stages would not fit otherwise.
static __host__ __device__ SmemPlan smem_plan_avail(int prec, int BN, int mode, int avail, int fold);

// With the epilogue's staging buffer where the pipeline keeps at least two
// stages (and two raw slots where it uses a raw ring); otherwise without.
// fold: accumulation chunks (fewer tensor-memory A stages at BN 128).
__host__ __device__ SmemPlan smem_plan(int prec, int BN, int mode, int ytma, int fold) {
  const int avail = SMEM_BUDGET - SMEM_CTRL - 1024;
  // the FP32 path, and BF16 stores by TMA: with 16-byte bf16 / e4m3 row
  // chunks the staged per-lane epilogue measured slower than the per-row one
  SmemPlan p = smem_plan_avail(prec, BN, mode, avail - (ytma ? EPI_TMA_BYTES : EPI_STG_BYTES), fold);
  if ((prec == PREC_TF32X3 || ytma) && p.stages >= 2 && (mode == PROD_TMA_DIRECT || p.raw_depth >= 2)) {
    p.epi_stage = 1;
    return p;
  }
  p = smem_plan_avail(prec, BN, mode, avail, fold);
  p.epi_stage = 0;
  return p;
}

static __host__ __device__ SmemPlan smem_plan_avail(int prec, int BN, int mode, int avail, int fold) {
  const int sb = stage_bytes(prec, BN, mode);
  const int rb = BM * raw_row_bytes(prec);
  if (mode == PROD_TMA_TMEM) {
    // B stages match the tensor-memory A stages; the rest of shared memory
    // holds raw TMA boxes in flight (up to RAW_MAX)
    SmemPlan p;
    p.stages = ts_stages(BN, fold);
    int R = (avail - p.stages * sb) / rb;
    p.raw_depth = R > RAW_MAX ? RAW_MAX : R;
    p.raw_slot_bytes = rb;
    return p;
  }
  if (mode == PROD_TMA_DIRECT) {
    SmemPlan p;
    p.stages = avail / sb > 8 ? 8 : avail / sb;
    p.raw_depth = 0;
    p.raw_slot_bytes = rb;
    return p;
  }
  int R = 3;
  while (R > 2 && avail - R * rb < 2 * sb) --R;
  int st = (avail - R * rb) / sb;
  if (st > 8) st = 8;
  // what the stages leave over: more raw boxes in flight
  if (mode == PROD_TMA_CONVERT) {
    R += (avail - R * rb - st * sb) / rb;
    if (R > RAW_MAX) R = RAW_MAX;
  }
  SmemPlan p;
  p.stages = st;
  p.raw_depth = R;
  p.raw_slot_bytes = rb;
  return p;
}
size_t conv_smem_bytes(int prec, int BN, int mode, int ytma, int fold) {
  const SmemPlan p = smem_plan(prec, BN, mode, ytma, fold);
  return (size_t)SMEM_CTRL + 1024 + (size_t)p.stages * stage_bytes(prec, BN, mode) +
         (size_t)p.raw_depth * p.raw_slot_bytes +
         (p.epi_stage ? (size_t)(ytma ? EPI_TMA_BYTES : EPI_STG_BYTES) : 0);
}

// Offset of 16-byte chunk q of row r inside a 128-byte-swizzled K-major tile.
__device__ __forceinline__ uint32_t swz(int r, int q) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((q ^ (r & 7)) << 4));
}

struct TileCoord {
  int phase, m_tile, n_tile;
};

// Rows of the GEMM: a.M, or a.count maps (clamped to 0..a.N) when the count
// lives in device memory.
__device__ __forceinline__ int gemm_rows(const ConvArgs &a) {
  if (!a.count) return a.M;
  int n = *reinterpret_cast<const volatile int *>(a.count);
  n = n < 0 ? 0 : (n > a.N ? a.N : n);
  return n * a.Hrow * a.Wrow;
}
// Tile t of the persistent schedule (CTA b takes t = b, b + G, b + 2G, ...).
// Several phases (decoder): the phases of one (m, n) tile are consecutive in
// t, so they run side by side on neighbouring CTAs and read the same input
// rows while they are in L2.  When G is a multiple of the phase count, a
// CTA's phase also advances by one every round (t / G), so each CTA cycles
// through the light and heavy phases instead of always drawing the same one;
// the rotation stays a bijection because a tile's P consecutive t never
// straddle a multiple of G.
__device__ __forceinline__ TileCoord tile_coord(const ConvArgs &a, int t) {
  TileCoord c;
  const int P = a.num_phases;
  const int unit = t / P;
  int l = t - unit * P;
  if (P > 1 && gridDim.x % P == 0) l = (l + (int)(t / gridDim.x)) % P;
  c.phase = a.phase_order[l];
  c.m_tile = unit / a.n_tiles;
  c.n_tile = unit - c.m_tile * a.n_tiles;
  return c;
}

// --------------------------------------------------------- conversions
// fp32 -> tf32, round to nearest with ties away from zero, done on the bits:
// add half an ulp of the 10-bit mantissa and clear the 13 dropped bits
// (finite inputs).  Integer add/and run at full rate, unlike the conversion
// instruction.
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
  __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return (uint32_t)lo | ((uint32_t)hi << 16);
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// 16-byte shared-memory store / load as single vector instructions.
__device__ __forceinline__ void sts128(uint8_t *p, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(smem_u32(p)), "r"(x), "r"(y), "r"(z), "r"(w)
               : "memory");
}
__device__ __forceinline__ void sts128u(uint32_t addr, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}
__device__ __forceinline__ void sts128f(uint32_t addr, float x, float y, float z, float w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}
__device__ __forceinline__ float4 lds128f(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ uint4 lds128(const void *p) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(smem_u32(p))
               : "memory");
  return v;
}

// One 16-byte A chunk from its raw bytes (uint4 = 16 B; FP8 reads two).
template <int PREC>
__device__ __forceinline__ void convert_store(uint8_t *a0, uint8_t *a1, uint32_t off, const uint4 *raw) {
  if constexpr (PREC == PREC_TF32X3) {
    const uint4 u = lds128(raw);
    const float x[4] = {__uint_as_float(u.x), __uint_as_float(u.y), __uint_as_float(u.z), __uint_as_float(u.w)};
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float hf = tf32_rna(x[e]);
      h[e] = __float_as_uint(hf);
      l[e] = __float_as_uint(tf32_rna(x[e] - hf));
    }
    sts128(a0 + off, h[0], h[1], h[2], h[3]);
    sts128(a1 + off, l[0], l[1], l[2], l[3]);
  } else {  // bf16 / e4m3: stored in the operand type already
    const uint4 u = lds128(raw);
    sts128(a0 + off, u.x, u.y, u.z, u.w);
  }
}

// mbar_wait that also adds the cycles it waited to `acc` when profiling.
__device__ __forceinline__ bool pwait(const ConvArgs &a, unsigned long long &acc, uint32_t bar, uint32_t parity) {
  if (!a.prof) return mbar_wait(bar, parity, a.timeout_ns, a.status, ERR_TIMEOUT);
  const long long t0 = clock64();
  const bool ok = mbar_wait(bar, parity, a.timeout_ns, a.status, ERR_TIMEOUT);
  acc += (unsigned long long)(clock64() - t0);
  return ok;
}

// ------------------------------------------------------------ A producer
// The implicit-im2col rows of A reach the 128-byte-swizzled A tile of an MMA
// stage in one of three ways (ProdMode), chosen per layer on the host:
//
// PROD_TMA_DIRECT / PROD_TMA_CONVERT: one TMA load per K block fetches the
//   whole 128-row tile for one tap and 128 bytes of channels: the tile covers
//   whole output rows of whole maps, so its rows are a box of the NHWC
//   activation tensor -- for the stride-2 convolution a box with traversal
//   stride 2 in H and W starting at (2 i0 + u - 1, v - 1), for a decoder
//   phase a box starting at (a0 + di, dj).  Positions outside the map are
//   zero-filled by the TMA unit (the convolution's padding).  The TMA writes
//   the 128-byte swizzle itself.  DIRECT (bf16): into the A tile.  CONVERT:
//   into a raw slot, from which the eight producer warps write the tf32 hi/lo
//   (or e4m3) tiles at the same swizzled offsets.
// PROD_CPASYNC (any shape): each producer thread gathers 16-byte chunks of
//   4 rows with cp.async into its own part of a raw slot, R-1 K blocks ahead,
//   then converts them (8 lanes per 128-byte row).
struct RowInfo {
  int pix_base[4], ybase[4], xbase[4];
  bool vrow[4];
  int nkb, ntaps;
  unsigned long long taps;  // tap t: dy in bits 4t..4t+1, dx in bits 4t+2..4t+3 (offsets 0..2)
};

__device__ __forceinline__ unsigned long long pack_taps(const PhaseDesc &pd) {
  unsigned long long tp = 0;
#pragma unroll
  for (int q = 0; q < 9; ++q)
    if (q < pd.ntaps) tp |= (unsigned long long)((pd.dy[q] & 3) | ((pd.dx[q] & 3) << 2)) << (4 * q);
  return tp;
}

__device__ __forceinline__ void prod_setup(const ConvArgs &a, int M, int t, int pt, RowInfo &ri) {
  const TileCoord tc = tile_coord(a, t);
  // the phase's tap table, read once per tile into registers
  const PhaseDesc &pd = a.ph[tc.phase];
  ri.nkb = pd.num_kb;
  ri.ntaps = pd.ntaps;
  ri.taps = pack_taps(pd);
  const int rows_per_map = a.Hrow * a.Wrow;
  const int hw_in = a.Hin * a.Win;
  const int lane = pt & 31, pw = pt >> 5;
  const bool s2 = a.kind == LK_CONV;
  const int o1 = a.kind == LK_CONV1 ? 1 : 0;  // stride 1: taps at offsets -1..1 from the output pixel
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int r = (lane >> 3) + 4 * pw + 32 * it;
    const int m = tc.m_tile * BM + r;
    const bool v = m < M;
    const int n = v ? m / rows_per_map : 0;
    const int rem = v ? m - n * rows_per_map : 0;
    const int i = rem / a.Wrow, j = rem - (rem / a.Wrow) * a.Wrow;
    ri.vrow[it] = v;
    ri.pix_base[it] = n * hw_in;
    ri.ybase[it] = s2 ? 2 * i - 1 : i - o1;
    ri.xbase[it] = s2 ? 2 * j - 1 : j - o1;
  }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// PROD_CPASYNC step 1: this thread's copies of one K block (4 rows x 16
// bytes) into raw slot `slot`; layout [row][thread] of 16 bytes.
template <int PREC>
__device__ __forceinline__ void raw_issue(const ConvArgs &a, const RowInfo &ri, int kb, int pt, uint32_t slot) {
  using T = PrecTraits<PREC>;
  constexpr int E = 16 / T::ELEM;
  constexpr int BKE = KROW_BYTES / T::ELEM;
  constexpr int AB = sizeof(typename T::act_t);
  const int k0 = kb * BKE + (pt & 7) * E;
  int tap, c;
  if (a.cin_shift >= 0) {
    tap = k0 >> a.cin_shift;
    c = k0 & (a.Cin - 1);
  } else {
    tap = k0 / a.Cin;
    c = k0 - tap * a.Cin;
  }
  const bool vtap = tap < ri.ntaps;
  const unsigned tb = vtap ? (unsigned)(ri.taps >> (4 * tap)) & 15u : 0u;
  const int dy = (int)(tb & 3u), dx = (int)(tb >> 2);
  const uint8_t *xin = reinterpret_cast<const uint8_t *>(a.x);
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int yy = ri.ybase[it] + dy, xx = ri.xbase[it] + dx;
    const bool okp = ri.vrow[it] && vtap && (unsigned)yy < (unsigned)a.Hin && (unsigned)xx < (unsigned)a.Win;
    const uint8_t *src = okp ? xin + ((size_t)(ri.pix_base[it] + yy * a.Win + xx) * a.Cin + c) * AB : xin;
    cp_async16(slot + (uint32_t)(it * NUM_PROD_THREADS + pt) * 16u, src, okp ? 16u : 0u);
  }
}

// PROD_CPASYNC step 2: convert this thread's raw chunks into the A tile(s).
template <int PREC>
__device__ __forceinline__ void raw_convert_own(const ConvArgs &a, int pt, const uint8_t *slot, uint8_t *a0,
                                                uint8_t *a1) {
  const int lane = pt & 31, pw = pt >> 5;
  const uint4 *raw = reinterpret_cast<const uint4 *>(slot);
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int r = (lane >> 3) + 4 * pw + 32 * it;
    convert_store<PREC>(a0, a1, swz(r, lane & 7), raw + it * NUM_PROD_THREADS + pt);
  }
}

// With tap boxes the slot is tap-major: chunk (r, q) of the K block is at
// (q / 2) BM 32 + 32 r + 16 (q % 2); a quarter warp then takes 8 rows of one
// chunk, so the reads see at most 2-way bank conflicts and the swizzled
// writes none.
__device__ __forceinline__ const uint8_t *tap_chunk(const uint8_t *slot, int r, int q) {
  return slot + (q >> 1) * (BM * 32) + r * 32 + (q & 1) * 16;
}

// PROD_TMA_CONVERT step 2 for one group of four producer warps (128
// threads, gt = thread index in the group): the whole K block, 8 chunks of
// 128 rows, from the raw slot (the A tile's swizzled layout, or tap-major
// with TAPS) into the tf32 hi / lo (or e4m3) tiles.
template <int PREC, bool TAPS>
__device__ __forceinline__ void raw_convert_tma_group(int gt, const uint8_t *slot, uint8_t *a0, uint8_t *a1) {
  const int lane = gt & 31, gw = gt >> 5, q = lane & 7;
  if constexpr (TAPS) {
    const int rr = lane & 7, qq = lane >> 3;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int r = 32 * gw + 8 * (it & 3) + rr, qt = 4 * (it >> 2) + qq;
      convert_store<PREC>(a0, a1, swz(r, qt), reinterpret_cast<const uint4 *>(tap_chunk(slot, r, qt)));
    }
    return;
  }
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int r = (lane >> 3) + 4 * gw + 16 * it;
    convert_store<PREC>(a0, a1, swz(r, q), reinterpret_cast<const uint4 *>(slot + swz(r, q)));
  }
}

// PROD_TMA_CONVERT, split-tf32 over whole K-block boxes (the raw slot is
// already a 128-byte-swizzled K-major tile): the MMAs read A_hi from the raw
// slot itself -- the tensor core takes the top 19 bits of each fp32 element,
// i.e. A truncated to tf32 -- so only A_lo = A - trunc_tf32(A), exact in
// fp32, is written, into the stage's lo tile.
__device__ __forceinline__ void raw_convert_lo(int gt, const uint8_t *slot, uint8_t *a1) {
  const int lane = gt & 31, gw = gt >> 5, q = lane & 7;
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int r = (lane >> 3) + 4 * gw + 16 * it;
    const uint32_t off = swz(r, q);
    const uint4 u = lds128(slot + off);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
    uint32_t l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      l[e] = __float_as_uint(__uint_as_float(w[e]) - __uint_as_float(w[e] & 0xFFFFE000u));
    sts128(a1 + off, l[0], l[1], l[2], l[3]);
  }
}

// PROD_TMA_TMEM step 2: the warp's lane quarter (rows 32 q .. 32 q + 31,
// q = warp % 4) of the whole K block goes from the raw slot, split into tf32
// hi/lo, into the A stage's tensor-memory columns [0, 32) (hi) and
// [32, 64) (lo).
template <bool TAPS>
__device__ __forceinline__ void raw_convert_tmem(int q, int lane, const uint8_t *slot, uint32_t ta) {
  const int r = 32 * q + lane;
  const uint32_t t0 = ta + ((uint32_t)(32 * q) << 16);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint4 u = lds128(TAPS ? tap_chunk(slot, r, 4 * h + c) : slot + swz(r, 4 * h + c));
      const float x[4] = {__uint_as_float(u.x), __uint_as_float(u.y), __uint_as_float(u.z), __uint_as_float(u.w)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float hf = tf32_rna(x[e]);
        hi[4 * c + e] = __float_as_uint(hf);
        lo[4 * c + e] = __float_as_uint(tf32_rna(x[e] - hf));
      }
    }
    tmem_st16(t0 + 16 * h, hi);
    tmem_st16(t0 + 32 + 16 * h, lo);
  }
  tmem_wait_st();
}

// Box coordinates (channel, x, y, map) of the A rows of tile t, K block kb.
struct TmaCursor {
  int t, kb, nkb, ntaps, n0, r0;  // r0: first output row (conv) / input row (phase) of the tile
  unsigned long long taps;
};
__device__ __forceinline__ void tma_tile(const ConvArgs &a, TmaCursor &c) {
  const TileCoord tc = tile_coord(a, c.t);
  const PhaseDesc &pd = a.ph[tc.phase];
  c.nkb = pd.num_kb;
  c.ntaps = pd.ntaps;
  c.taps = pack_taps(pd);
  const int rows_per_map = a.Hrow * a.Wrow;
  const int m0 = tc.m_tile * BM;
  c.n0 = m0 / rows_per_map;
  c.r0 = (m0 - c.n0 * rows_per_map) / a.Wrow;
}
template <int PREC>
__device__ __forceinline__ void tma_issue(const ConvArgs &a, const TmaCursor &c, uint32_t dst, uint32_t bar) {
  using T = PrecTraits<PREC>;
  constexpr int BKE = KROW_BYTES / T::ELEM;
  if (a.tap_boxes) {
    // taps narrower than a K block -- 8 channels (FP32: 32 bytes, four per K
    // block; BF16: 16 bytes, eight), or 64 e4m3 channels (64 bytes, two) --
    // of the stride-2 or stride-1 conv, one box each, tap-major; a slot past
    // the last tap loads tap 0 again, against B rows packed as zero
    constexpr int TB = PREC == PREC_FP8 ? 64 : 8 * T::ELEM;  // bytes of one tap row (Cin 64 / 8)
    constexpr int TPB = KROW_BYTES / TB;                      // taps per K block
    const int ry = a.kind == LK_CONV ? 2 * c.r0 : c.r0;
#pragma unroll
    for (int t = 0; t < TPB; ++t) {
      const int tap = TPB * c.kb + t < c.ntaps ? TPB * c.kb + t : 0;
      const unsigned tb = (unsigned)(c.taps >> (4 * tap)) & 15u;
      const int dy = (int)(tb & 3u), dx = (int)(tb >> 2);
      tma_load_4d(dst + (uint32_t)(t * BM * TB), &a.tmap, 0, dx - 1, ry + dy - 1, c.n0, bar);
    }
    return;
  }
  const int kpt = a.Cin / BKE;  // K blocks per tap
  const int tap = c.kb / kpt;
  const int c0 = (c.kb - tap * kpt) * BKE;
  const unsigned tb = (unsigned)(c.taps >> (4 * tap)) & 15u;
  const int dy = (int)(tb & 3u), dx = (int)(tb >> 2);
  int x, y;
  if (a.kind == LK_CONV) {  // stride-2 box: rows 2 i + dy - 1, cols 2 j + dx - 1
    x = dx - 1;
    y = 2 * c.r0 + dy - 1;
  } else if (a.kind == LK_CONV1) {  // stride-1 box: rows i + dy - 1, cols j + dx - 1
    x = dx - 1;
    y = c.r0 + dy - 1;
    if (a.x2 && c0 >= a.C1) {  // the channels of the concatenated second input
      tma_load_4d(dst, &a.tmap2, c0 - a.C1, x, y, c.n0, bar);
      return;
    }
  } else {  // decoder phase: rows a + di, cols b + dj
    x = dx;
    y = c.r0 + dy;
  }
  tma_load_4d(dst, &a.tmap, c0, x, y, c.n0, bar);
}

// PROD_TMA_CONVERT / PROD_TMA_TMEM step 1, one thread: every raw box of the
// CTA's K blocks in order, each into ring slot j % R once the group that
// converted its previous occupant has released it.
template <int PREC>
__device__ __noinline__ void tma_issue_loop(const ConvArgs &a, uint32_t raw_u32, uint64_t *raw_full,
                                            uint64_t *raw_empty, int R, int slot_bytes, int total_tiles) {
  if ((int)blockIdx.x >= total_tiles) return;
  int total_kb = 0;
  for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) total_kb += a.ph[tile_coord(a, t).phase].num_kb;
  TmaCursor c;
  c.t = blockIdx.x;
  c.kb = 0;
  tma_tile(a, c);
  unsigned long long w_issue = 0;
  for (int j = 0; j < total_kb; ++j) {
    const int slot = j % R;
    if (!pwait(a, w_issue, smem_u32(&raw_empty[slot]), (uint32_t)(((j / R) & 1) ^ 1))) break;
    const uint32_t fb = smem_u32(&raw_full[slot]);
    mbar_arrive_expect_tx(fb, (uint32_t)(BM * KROW_BYTES));
    tma_issue<PREC>(a, c, raw_u32 + (uint32_t)(slot * slot_bytes), fb);
    if (++c.kb == c.nkb) {
      c.kb = 0;
      c.t += gridDim.x;
      if (c.t < total_tiles) tma_tile(a, c);
    }
  }
  if (a.prof) atomicAdd(&a.prof[PROF_PROD_ISSUE], w_issue * 8);  // reported per producer warp like the others
}

// PROD_TMA_CONVERT / PROD_TMA_TMEM producer loop (TAPS: the raw slots hold
// tap boxes, see tma_issue).
template <int PREC, bool TAPS, bool HI>
__device__ __forceinline__ void convert_loop(const ConvArgs &a, uint8_t *data, uint8_t *raw, uint64_t *full_bar,
                                             uint64_t *empty_bar, uint64_t *raw_full, uint64_t *raw_empty,
                                             int stages, int sbytes, int R, int slot_bytes, int total_kb,
                                             uint32_t tmem_base, unsigned long long &w_empty,
                                             unsigned long long &w_copy, unsigned long long &w_conv,
                                             unsigned long long &w_fence) {
  const int pt = threadIdx.x - PROD_WARP0 * 32;  // 0..255
  const int lane = pt & 31;
  const int a_bytes = BM * KROW_BYTES;
  // The raw boxes come from the TMA-issue warp (tma_issue_loop); the
  // producer warps form two groups of four -- one warp per tensor-memory
  // lane quarter -- that take alternate K blocks, so two blocks are being
  // converted at any time.  K block j uses raw slot j % R and MMA stage
  // j % stages; the barrier parities follow from j.
  const int g = (pt >> 5) >> 2, gw = (pt >> 5) & 3, gt = pt & 127;
  // A_hi read by the MMAs from the raw slot, which their commit releases
  const bool hiraw = HI && PREC == PREC_TF32X3 && !TAPS && a.hi_raw;
  for (int jc = g; jc < total_kb; jc += 2) {
    const int slot = jc % R, stage = jc % stages;
    if (!pwait(a, w_copy, smem_u32(&raw_full[slot]), (uint32_t)((jc / R) & 1))) break;
    if (!pwait(a, w_empty, smem_u32(&empty_bar[stage]), (uint32_t)(((jc / stages) & 1) ^ 1))) break;
    uint8_t *a0 = data + stage * sbytes;
    const long long tv0 = a.prof ? clock64() : 0;
    if constexpr (PREC == PREC_TF32X3) {
      if (a.prod_mode == PROD_TMA_TMEM)
        raw_convert_tmem<TAPS>(gw, lane, raw + slot * slot_bytes,
                               tmem_base + (uint32_t)(ts_a_col0(a.BN, a.kfold > 0) + stage * 64));
      else if (HI && hiraw)
        raw_convert_lo(gt, raw + slot * slot_bytes, a0 + a_bytes);
      else
        raw_convert_tma_group<PREC, TAPS>(gt, raw + slot * slot_bytes, a0, a0 + a_bytes);
    } else {
      raw_convert_tma_group<PREC, false>(gt, raw + slot * slot_bytes, a0, a0 + a_bytes);
    }
    const long long tv1 = a.prof ? clock64() : 0;
    fence_proxy_async_smem();  // A tile writes -> MMA; raw reads before the slot's next TMA write
    tc_fence_before();         // tensor-memory A stores -> MMA (PROD_TMA_TMEM)
    __syncwarp();
    if (a.prof) {
      w_conv += (unsigned long long)(tv1 - tv0);
      w_fence += (unsigned long long)(clock64() - tv1);
    }
    if (lane == 0) {
      mbar_arrive(smem_u32(&full_bar[stage]));
      if (!(HI && hiraw)) mbar_arrive(smem_u32(&raw_empty[slot]));
    }
  }
}

// Producer warps.  `raw` is the raw ring (unused in PROD_TMA_DIRECT).  HI:
// the decoder forms, where a.hi_raw may send A_hi to the MMAs from the raw
// slot (compiled apart, so the encoders' producers carry none of it).
template <int PREC, bool HI>
__device__ __noinline__ void run_producer(const ConvArgs &a, uint8_t *data, uint8_t *raw, uint64_t *full_bar,
                                          uint64_t *empty_bar, uint64_t *raw_full, uint64_t *raw_empty, int stages,
                                          int sbytes, int R, int slot_bytes, int M, int total_tiles,
                                          uint32_t tmem_base) {
  const int pt = threadIdx.x - PROD_WARP0 * 32;  // 0..255
  const int lane = pt & 31;
  const int a_bytes = BM * KROW_BYTES;
  const uint32_t raw_u32 = smem_u32(raw);
  const uint32_t data_u32 = smem_u32(data);
  if ((int)blockIdx.x >= total_tiles) return;
  int total_kb = 0;
  for (int t = blockIdx.x; t < total_tiles; t += gridDim.x) total_kb += a.ph[tile_coord(a, t).phase].num_kb;
  unsigned long long w_empty = 0, w_copy = 0, w_conv = 0, w_fence = 0, w_issue = 0;
  const long long t_start = a.prof ? clock64() : 0;

  if (a.prod_mode == PROD_TMA_DIRECT) {
    // one thread: wait for the stage, expect the box bytes, load into the A tile
    if (pt == 0) {
      TmaCursor c;
      c.t = blockIdx.x;
      c.kb = 0;
      tma_tile(a, c);
      int stage = 0;
      uint32_t phase = 0;
      for (int j = 0; j < total_kb; ++j) {
        if (!pwait(a, w_empty, smem_u32(&empty_bar[stage]), phase ^ 1)) break;
        const uint32_t fb = smem_u32(&full_bar[stage]);
        mbar_arrive_expect_tx(fb, (uint32_t)a_bytes);
        tma_issue<PREC>(a, c, data_u32 + stage * sbytes, fb);
        if (++stage == stages) {
          stage = 0;
          phase ^= 1;
        }
        if (++c.kb == c.nkb) {
          c.kb = 0;
          c.t += gridDim.x;
          if (c.t < total_tiles) tma_tile(a, c);
        }
      }
    }
  } else if (a.prod_mode == PROD_TMA_CONVERT || a.prod_mode == PROD_TMA_TMEM) {
    if (a.tap_boxes)
      convert_loop<PREC, true, HI>(a, data, raw, full_bar, empty_bar, raw_full, raw_empty, stages, sbytes, R, slot_bytes,
                               total_kb, tmem_base, w_empty, w_copy, w_conv, w_fence);
    else
      convert_loop<PREC, false, HI>(a, data, raw, full_bar, empty_bar, raw_full, raw_empty, stages, sbytes, R, slot_bytes,
                                total_kb, tmem_base, w_empty, w_copy, w_conv, w_fence);
  } else {
    // PROD_CPASYNC
    const int D = R - 1;
    int it_t = blockIdx.x, it_kb = 0;
    bool it_more = true;
    RowInfo ri;
    prod_setup(a, M, it_t, pt, ri);
    int islot = 0;
    auto issue = [&]() {
      const long long ti0 = a.prof ? clock64() : 0;
      if (it_more) {
        raw_issue<PREC>(a, ri, it_kb, pt, raw_u32 + (uint32_t)(islot * slot_bytes));
        if (++it_kb == ri.nkb) {
          it_kb = 0;
          it_t += gridDim.x;
          if (it_t < total_tiles)
            prod_setup(a, M, it_t, pt, ri);
          else
            it_more = false;
        }
      }
      cp_async_commit();  // one group per K block (empty past the end)
      if (++islot == R) islot = 0;
      if (a.prof) w_issue += (unsigned long long)(clock64() - ti0);
    };
    for (int j = 0; j < D; ++j) issue();
    int cslot = 0, stage = 0;
    uint32_t phase = 0;
    for (int jc = 0; jc < total_kb; ++jc) {
      issue();
      const long long tc0 = a.prof ? clock64() : 0;
      if (D >= 2)
        cp_async_wait<2>();
      else
        cp_async_wait<1>();
      if (a.prof) w_copy += (unsigned long long)(clock64() - tc0);
      if (!pwait(a, w_empty, smem_u32(&empty_bar[stage]), phase ^ 1)) break;
      uint8_t *a0 = data + stage * sbytes;
      const long long tv0 = a.prof ? clock64() : 0;
      raw_convert_own<PREC>(a, pt, raw + cslot * slot_bytes, a0, a0 + a_bytes);
      const long long tv1 = a.prof ? clock64() : 0;
      fence_proxy_async_smem();
      __syncwarp();
      if (a.prof) {
        w_conv += (unsigned long long)(tv1 - tv0);
        w_fence += (unsigned long long)(clock64() - tv1);
      }
      if (lane == 0) mbar_arrive(smem_u32(&full_bar[stage]));
      if (++stage == stages) {
        stage = 0;
        phase ^= 1;
      }
      if (++cslot == R) cslot = 0;
    }
    cp_async_wait_all();
  }
  if (a.prof && lane == 0) {
    atomicAdd(&a.prof[PROF_PROD_WAIT_EMPTY], w_empty);
    atomicAdd(&a.prof[PROF_PROD_WAIT_COPY], w_copy);
    atomicAdd(&a.prof[PROF_PROD_TOTAL], (unsigned long long)(clock64() - t_start));
    atomicAdd(&a.prof[PROF_PROD_CONVERT], w_conv);
    atomicAdd(&a.prof[PROF_PROD_FENCE], w_fence);
    atomicAdd(&a.prof[PROF_PROD_ISSUE], w_issue);
  }
}

// Accumulator columns [c, c+16) of a tile: the main accumulator, plus the
// correction accumulator BN columns further on for the split-tf32 path.
// t2: the second accumulator's address (split-tf32: the correction one, BN
// columns on; with accumulation chunks the running sum, or kNoAcc for a
// tile of one chunk).
constexpr uint32_t kNoAcc = 0xFFFFFFFFu;
template <int PREC, bool FOLD>
__device__ __forceinline__ void tmem_ld_acc(uint32_t taddr, uint32_t t2, float (&v)[16]) {
  if constexpr (PREC == PREC_TF32X3) {
    if (FOLD && t2 == kNoAcc) {
      tmem_ld16(taddr, v);
      return;
    }
    // both loads in flight, one wait
    uint32_t a[16], c[16];
    tmem_ld16_nowait(taddr, a);
    tmem_ld16_nowait(t2, c);
    tmem_wait_ld();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(a[e]) + __uint_as_float(c[e]);
  } else {
    tmem_ld16(taddr, v);
  }
}
template <bool FOLD>
__device__ __forceinline__ uint32_t acc_at(uint32_t t2, int c) {
  if constexpr (FOLD)
    return t2 == kNoAcc ? kNoAcc : t2 + (uint32_t)c;
  else
    return t2 + (uint32_t)c;
}

// 16 consecutive skip channels as raw 16-byte words (fp32: 4 words, bf16: 2,
// e4m3: 1).
template <int PREC>
__device__ __forceinline__ void load_skip(const typename PrecTraits<PREC>::act_t *p, uint4 (&s)[4]) {
  const uint4 *q = reinterpret_cast<const uint4 *>(p);
  constexpr int NW = PREC == PREC_TF32X3 ? 4 : (PREC == PREC_BF16 ? 2 : 1);
#pragma unroll
  for (int e = 0; e < NW; ++e) s[e] = q[e];
}

// Four e4m3 bytes of a word -> floats.
__device__ __forceinline__ void e4m3x4_to_f32(uint32_t w, float *f) {
  const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xFFFFu), __NV_E4M3);
  const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
  f[0] = a.x;
  f[1] = a.y;
  f[2] = b.x;
  f[3] = b.y;
}

// Epilogue of one 16-column chunk of one accumulator row: TMEM load (every
// lane: the load is warp-collective), dequantisation (FP8), bias, ReLU, the
// skip add, the calibration max (warp-collective), then for a valid row the
// NHWC store -- e4m3 with the consumer's scales when out_qinv is set.
// Store 16 values in the kernel's activation type (not e4m3).
template <int PREC>
__device__ __forceinline__ void store16(uint8_t *yb, const float (&v)[16]) {
  if constexpr (PREC == PREC_TF32X3) {
    float4 *q = reinterpret_cast<float4 *>(yb);
#pragma unroll
    for (int e = 0; e < 4; ++e) q[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
  } else {
    uint4 *q = reinterpret_cast<uint4 *>(yb);
#pragma unroll
    for (int e = 0; e < 2; ++e)
      q[e] = make_uint4(pack_bf16x2(v[8 * e], v[8 * e + 1]), pack_bf16x2(v[8 * e + 2], v[8 * e + 3]),
                        pack_bf16x2(v[8 * e + 4], v[8 * e + 5]), pack_bf16x2(v[8 * e + 6], v[8 * e + 7]));
  }
}

// The epilogue's rectifier: ReLU, or in the U-Net form (FOLD) LeakyReLU
// max(z, a.slope z), a.slope in [0, 1).  Compile-time: a select per element
// measured 5-40 % on the autoencoder's epilogue-bound layers.
template <bool FOLD>
__device__ __forceinline__ float act_fn(const ConvArgs &a, float z) {
  if constexpr (FOLD)
    return fmaxf(z, a.slope * z);
  else
    return fmaxf(z, 0.f);
}

// Zero v[e] where the mask tensor's value is not positive (16 channels at mb).
template <int PREC>
__device__ __forceinline__ void apply_mask(const uint8_t *mb, float (&v)[16]) {
  if constexpr (PREC == PREC_TF32X3) {
    const float4 *m = reinterpret_cast<const float4 *>(mb);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float4 q = m[e];
      if (!(q.x > 0.f)) v[4 * e] = 0.f;
      if (!(q.y > 0.f)) v[4 * e + 1] = 0.f;
      if (!(q.z > 0.f)) v[4 * e + 2] = 0.f;
      if (!(q.w > 0.f)) v[4 * e + 3] = 0.f;
    }
  } else {
    const uint4 *m = reinterpret_cast<const uint4 *>(mb);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const uint4 q = m[e];
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        if (!(bf16_lo(w[h]) > 0.f)) v[8 * e + 2 * h] = 0.f;
        if (!(bf16_hi(w[h]) > 0.f)) v[8 * e + 2 * h + 1] = 0.f;
      }
    }
  }
}

template <int PREC, bool FOLD>
__device__ __forceinline__ void epi_chunk(const ConvArgs &a, uint32_t taddr, int cc, int BN, int col0, bool vrow,
                                          bool has_skip, const uint4 (&sk)[4], uint8_t *yb, size_t eoff,
                                          uint32_t t2) {
  float v[16];
  tmem_ld_acc<PREC, FOLD>(taddr + cc * 16, acc_at<FOLD>(FOLD ? t2 : taddr + (uint32_t)BN, cc * 16), v);
  const float *bsc = a.bscale ? a.bscale + col0 : nullptr;
  const float4 *bias4 = reinterpret_cast<const float4 *>(a.bias + col0);
#pragma unroll
  for (int e4 = 0; e4 < 4; ++e4) {
    const float4 b = __ldg(bias4 + e4);
    const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float z = bsc ? v[4 * e4 + e] * __ldg(bsc + 4 * e4 + e) : v[4 * e4 + e];
      z += bb[e];
      if (a.relu) z = act_fn<FOLD>(a, z);
      v[4 * e4 + e] = z;
    }
  }
  if constexpr (PREC != PREC_FP8) {
    if (a.y2 && a.y2_pre_skip && vrow)
      store16<PREC>(reinterpret_cast<uint8_t *>(a.y2) + eoff * sizeof(typename PrecTraits<PREC>::act_t), v);
  }
  if (has_skip) {
    if constexpr (PREC == PREC_TF32X3) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        v[4 * e] += __uint_as_float(sk[e].x);
        v[4 * e + 1] += __uint_as_float(sk[e].y);
        v[4 * e + 2] += __uint_as_float(sk[e].z);
        v[4 * e + 3] += __uint_as_float(sk[e].w);
      }
    } else if constexpr (PREC == PREC_BF16) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        v[8 * e + 0] += bf16_lo(sk[e].x);
        v[8 * e + 1] += bf16_hi(sk[e].x);
        v[8 * e + 2] += bf16_lo(sk[e].y);
        v[8 * e + 3] += bf16_hi(sk[e].y);
        v[8 * e + 4] += bf16_lo(sk[e].z);
        v[8 * e + 5] += bf16_hi(sk[e].z);
        v[8 * e + 6] += bf16_lo(sk[e].w);
        v[8 * e + 7] += bf16_hi(sk[e].w);
      }
    } else {
      float f[16];
      e4m3x4_to_f32(sk[0].x, f);
      e4m3x4_to_f32(sk[0].y, f + 4);
      e4m3x4_to_f32(sk[0].z, f + 8);
      e4m3x4_to_f32(sk[0].w, f + 12);
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = fmaf(f[e], __ldg(a.skip_scale + col0 + e), v[e]);
    }
  }
  if (a.amax) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const unsigned m = __reduce_max_sync(0xffffffffu, vrow ? __float_as_uint(fabsf(v[e])) : 0u);
      if ((threadIdx.x & 31) == 0 && m) atomicMax(a.amax + col0 + e, m);
    }
  }
  if (!vrow) return;
  if constexpr (PREC != PREC_FP8) {
    constexpr int AB = sizeof(typename PrecTraits<PREC>::act_t);
    if (a.y2 && !a.y2_pre_skip) store16<PREC>(reinterpret_cast<uint8_t *>(a.y2) + eoff * AB, v);
    if (a.mask) apply_mask<PREC>(reinterpret_cast<const uint8_t *>(a.mask) + eoff * AB, v);
  }
  if (a.out_qinv) {
    const float *qi = a.out_qinv + col0;
    uint4 o;
    o.x = pack_e4m3x4(v[0] * __ldg(qi), v[1] * __ldg(qi + 1), v[2] * __ldg(qi + 2), v[3] * __ldg(qi + 3));
    o.y = pack_e4m3x4(v[4] * __ldg(qi + 4), v[5] * __ldg(qi + 5), v[6] * __ldg(qi + 6), v[7] * __ldg(qi + 7));
    o.z = pack_e4m3x4(v[8] * __ldg(qi + 8), v[9] * __ldg(qi + 9), v[10] * __ldg(qi + 10), v[11] * __ldg(qi + 11));
    o.w = pack_e4m3x4(v[12] * __ldg(qi + 12), v[13] * __ldg(qi + 13), v[14] * __ldg(qi + 14),
                      v[15] * __ldg(qi + 15));
    *reinterpret_cast<uint4 *>(yb) = o;
  } else if constexpr (PREC != PREC_FP8) {
    store16<PREC>(yb, v);
  }
}

// ---- staged epilogue: four consecutive elements at element offset e ----
// Load 4 values of an NHWC tensor of the kernel's activation type (FP8: e4m3
// times the channels' scales sc).
template <int PREC>
__device__ __forceinline__ float4 ld4(const void *base, size_t e, const float *sc) {
  if constexpr (PREC == PREC_TF32X3) {
    return *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(base) + e);
  } else if constexpr (PREC == PREC_BF16) {
    const uint2 u = *reinterpret_cast<const uint2 *>(reinterpret_cast<const __nv_bfloat16 *>(base) + e);
    return make_float4(bf16_lo(u.x), bf16_hi(u.x), bf16_lo(u.y), bf16_hi(u.y));
  } else {
    float f[4];
    e4m3x4_to_f32(*reinterpret_cast<const uint32_t *>(reinterpret_cast<const uint8_t *>(base) + e), f);
    return make_float4(f[0] * __ldg(sc), f[1] * __ldg(sc + 1), f[2] * __ldg(sc + 2), f[3] * __ldg(sc + 3));
  }
}
// Store 4 values in the kernel's activation type, or as e4m3 times qi.
template <int PREC>
__device__ __forceinline__ void st4(void *base, size_t e, float4 v, const float *qi) {
  if (qi) {
    *reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(base) + e) =
        pack_e4m3x4(v.x * __ldg(qi), v.y * __ldg(qi + 1), v.z * __ldg(qi + 2), v.w * __ldg(qi + 3));
  } else if constexpr (PREC == PREC_TF32X3) {
    *reinterpret_cast<float4 *>(reinterpret_cast<float *>(base) + e) = v;
  } else {
    *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(base) + e) =
        make_uint2(pack_bf16x2(v.x, v.y), pack_bf16x2(v.z, v.w));
  }
}

// One accumulator tile through the staging buffer.  Per 16-column chunk each
// lane takes its own row out of tensor memory (the load is warp-collective)
// and applies the dequantisation, bias, ReLU and the calibration maximum;
// the warp's 32 rows x 16 columns then go through shared memory so that four
// lanes cover one row and the skip load, the stores and the training mask /
// second output are 16-byte accesses to 64 contiguous bytes of each row
// (instead of 32 rows per warp instruction).
// FP32 encoder epilogue by TMA stores (y_tma: output rows contiguous, no
// skip, no training outputs).  Each 16-column chunk of the warp's 32 rows
// (bias, ReLU) goes into a 2 KB staging box -- row r at 64 r, its 16-byte
// chunk c at the 64-byte swizzle position c ^ ((r / 2) % 4) -- and one TMA
// store writes the box.  The warp's boxes form a ring (box counts chunks
// across tiles): a box is rewritten once the store that read it
// EPI_TMA_BOXES chunks ago is done, while the later ones are still in
// flight.  With a single box every chunk waited for the store just issued
// (e1 at 4096 maps: 0.167 ms).  Rows past M are clipped by the tensor map.
//
// Decoder phases (LK_CONVT): the warp's 32 rows are y_mw maps x y_rw phase
// rows x Wrow columns, i.e. a box of the output with element strides 2 in H
// and W starting at (2 i0 + oy, ox); the skip add reads each lane's own row
// (prefetched one chunk ahead, as in the other epilogues).
// EPI (compiled apart): EPI_E4 stores the tile as e4m3 with a.out_qinv (FP8
// contexts' encoder outputs); EPI_SKIP is the FP32 decoder form, whose skip
// comes by TMA when a.skip_tma; EPI_PAIR is EPI_SKIP for a phase pair,
// columns [Cout, 2 Cout) at the second output parity.
enum EpiForm { EPI_PLAIN = 0, EPI_E4 = 1, EPI_PAIR = 2, EPI_SKIP = 3 };
template <int PREC, bool FOLD, int EPI>
__device__ __forceinline__ bool epi_tile_tma(const ConvArgs &a, uint32_t taddr, int BN, int n0, int row0,
                                             const PhaseDesc &pd, uint32_t ring, int &box, unsigned long long &w_tfull,
                                             uint32_t tfull, uint32_t par, unsigned long long &w_ld, uint32_t t2,
                                             uint32_t skbar, uint32_t &skpar) {
  constexpr bool E4 = EPI == EPI_E4;
  const int lane = threadIdx.x & 31;
  const bool convt = a.kind == LK_CONVT;
  // box origin (convT) and this lane's skip row
  const int rows_per_map = a.Hrow * a.Wrow;
  const int bn0 = row0 / rows_per_map, bi0 = (row0 - bn0 * rows_per_map) / a.Wrow;
  const int m = row0 + lane;
  const bool vrow = m < a.M;
  const int n = m / rows_per_map, rem = m - n * rows_per_map;
  const int i = rem / a.Wrow, j = rem - (rem / a.Wrow) * a.Wrow;
  const size_t sbase = (((size_t)n * a.Hout + (2 * i + pd.oy)) * a.Wout + (2 * j + pd.ox)) * a.Cout + n0;
  // a phase pair (one tile, n0 = 0): columns [Cout, 2 Cout) are the output
  // parity (oy2, ox2), whose skip element is dsk past the first phase's
  constexpr bool pr = EPI == EPI_PAIR;
  const int dsk = pr ? ((pd.oy2 - pd.oy) * a.Wout + (pd.ox2 - pd.ox) - 1) * a.Cout : 0;
  // skip boxes by TMA (a.skip_tma): chunk cc's box of the ring, (box0 + cc)
  // mod EPI_TMA_BOXES, is loaded on that box's barrier -- the first
  // EPI_TMA_BOXES - 1 before the accumulator is waited for, each later one
  // once the store of the chunk before it has read its box -- and the chunk
  // adds the skip from there and stores the sum from the same box
  constexpr bool SKT = PREC == PREC_TF32X3 && !FOLD && (EPI == EPI_SKIP || EPI == EPI_PAIR);
  const bool skt = SKT && a.skip_tma;
  const int nch = BN / 16;
  const int box0 = box;
  auto issue_skip = [&](int cc) {  // lane 0
    const int b = (box0 + cc) % EPI_TMA_BOXES, c0 = n0 + cc * 16;
    const bool u = pr && c0 >= a.Cout;
    const uint32_t bar = skbar + 8u * (uint32_t)b;
    mbar_arrive_expect_tx(bar, EPI_TMA_BOX_BYTES);
    tma_load_4d(ring + (uint32_t)(b * EPI_TMA_BOX_BYTES), &a.ymap, u ? c0 - a.Cout : c0, u ? pd.ox2 : pd.ox,
                2 * bi0 + (u ? pd.oy2 : pd.oy), bn0, bar);
  };
  // after a failed wait: the loads still in flight, chunks [c1, c2), land
  // before the kernel returns (bounded waits, their failures only latched)
  auto drain_skip = [&](int c1, int c2) {
    if (lane == 0)
      for (int cc = c1; cc < c2 && cc < nch; ++cc) {
        const int b = (box0 + cc) % EPI_TMA_BOXES;
        mbar_wait(skbar + 8u * (uint32_t)b, (skpar >> b) & 1u, a.timeout_ns, a.status, ERR_TIMEOUT);
        skpar ^= 1u << b;
      }
  };
  if constexpr (SKT) {
    if (skt && lane == 0) {
      bulk_wait_read<0>();  // every box's last store has read it
      for (int cc = 0; cc < nch && cc < EPI_TMA_BOXES - 1; ++cc) issue_skip(cc);
    }
  }
  using act_t = typename PrecTraits<PREC>::act_t;
  const act_t *skp = a.skip && vrow && !skt ? reinterpret_cast<const act_t *>(a.skip) + sbase : nullptr;
  float4 sk[4];
  // 16 skip values of chunk cc (fp32: four 16-byte loads; bf16: two)
  auto load_sk = [&](int cc) {
    const act_t *sp = skp + cc * 16 + (cc * 16 >= a.Cout ? dsk : 0);
    if constexpr (PREC == PREC_BF16) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(sp) + h);
        sk[2 * h] = make_float4(bf16_lo(u.x), bf16_hi(u.x), bf16_lo(u.y), bf16_hi(u.y));
        sk[2 * h + 1] = make_float4(bf16_lo(u.z), bf16_hi(u.z), bf16_lo(u.w), bf16_hi(u.w));
      }
    } else {
#pragma unroll
      for (int e4 = 0; e4 < 4; ++e4) sk[e4] = __ldg(reinterpret_cast<const float4 *>(sp) + e4);
    }
  };
  if (skp) load_sk(0);
  // the fused 1x1 head (U-Net form): this lane's pixel's outputs, from the bias
  const bool head = FOLD && a.head_w != nullptr;
  float hacc[KHEAD_MAX];
  if constexpr (FOLD) {
#pragma unroll
    for (int o = 0; o < KHEAD_MAX; ++o) hacc[o] = head && o < a.head_cout ? __ldg(a.head_w + a.head_cout * a.Cout + o) : 0.f;
  }
  if (!pwait(a, w_tfull, tfull, par)) {
    if (skt) drain_skip(0, EPI_TMA_BOXES - 1);
    return false;
  }
  tc_fence_after();
  for (int cc = 0; cc < nch; ++cc) {
    const int col0 = n0 + cc * 16;
    float v[16];
    const long long tl0 = a.prof ? clock64() : 0;
    tmem_ld_acc<PREC, FOLD>(taddr + cc * 16, acc_at<FOLD>(FOLD ? t2 : taddr + (uint32_t)BN, cc * 16), v);
    if (a.prof) w_ld += (unsigned long long)(clock64() - tl0);
    const bool up = pr && col0 >= a.Cout;  // the pair's second phase
    const int ch0 = up ? col0 - a.Cout : col0;
    const float4 *bias4 = reinterpret_cast<const float4 *>(a.bias + ch0);
    if constexpr (PREC == PREC_FP8) {  // dequantise with the output columns' weight scales
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] *= __ldg(a.bscale + col0 + e);
    }
#pragma unroll
    for (int e4 = 0; e4 < 4; ++e4) {
      const float4 b = __ldg(bias4 + e4);
      const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float z = v[4 * e4 + e] + bb[e];
        if (a.relu) z = act_fn<FOLD>(a, z);
        v[4 * e4 + e] = z;
      }
    }
    if (skp) {
#pragma unroll
      for (int e4 = 0; e4 < 4; ++e4) {
        v[4 * e4] += sk[e4].x;
        v[4 * e4 + 1] += sk[e4].y;
        v[4 * e4 + 2] += sk[e4].z;
        v[4 * e4 + 3] += sk[e4].w;
      }
      if (cc + 1 < BN / 16) load_sk(cc + 1);
    }
    if constexpr (SKT) {
      if (skt) {  // this chunk's skip box (the waits count as the epilogue's input waits)
        const uint32_t bar = skbar + 8u * (uint32_t)box;
        if (!pwait(a, w_tfull, bar, (skpar >> box) & 1u)) {
          drain_skip(cc + 1, cc + EPI_TMA_BOXES - 1);
          return false;
        }
        skpar ^= 1u << box;
        const uint32_t sb = ring + (uint32_t)(box * EPI_TMA_BOX_BYTES) + (uint32_t)(lane * 64);
#pragma unroll
        for (int e4 = 0; e4 < 4; ++e4) {
          const float4 k = lds128f(sb + (uint32_t)((e4 ^ ((lane >> 1) & 3)) << 4));
          v[4 * e4] += k.x;
          v[4 * e4 + 1] += k.y;
          v[4 * e4 + 2] += k.z;
          v[4 * e4 + 3] += k.w;
        }
      }
    }
    if constexpr (FOLD) {
      if (head) {  // this chunk's 16 channels into the head's dot products; y is not stored
#pragma unroll
        for (int o = 0; o < KHEAD_MAX; ++o) {
          if (o >= a.head_cout) break;
          const float *wo = a.head_w + (size_t)o * a.Cout + col0;
#pragma unroll
          for (int e = 0; e < 16; ++e) hacc[o] = fmaf(__ldg(wo + e), v[e], hacc[o]);
        }
        continue;
      }
    }
    const uint32_t stg = ring + (uint32_t)(box * EPI_TMA_BOX_BYTES);
    box = box + 1 == EPI_TMA_BOXES ? 0 : box + 1;
    if (lane == 0) bulk_wait_read<EPI_TMA_BOXES - 1>();
    __syncwarp();
    if constexpr (E4) {
      // e4m3 with the consuming layer's inverse input scales: 16-byte rows,
      // no swizzle (a quarter warp's eight rows are 128 contiguous bytes)
      const float *qi = a.out_qinv + col0;
      float q[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) q[e] = v[e] * __ldg(qi + e);
      sts128u(stg + (uint32_t)(lane * 16), pack_e4m3x4(q[0], q[1], q[2], q[3]), pack_e4m3x4(q[4], q[5], q[6], q[7]),
              pack_e4m3x4(q[8], q[9], q[10], q[11]), pack_e4m3x4(q[12], q[13], q[14], q[15]));
    } else if constexpr (PREC == PREC_BF16) {
      // 32-byte rows, 32-byte swizzle: 16-byte chunk h at h ^ ((r / 4) % 2)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        sts128u(stg + (uint32_t)(lane * 32 + ((h ^ ((lane >> 2) & 1)) << 4)),
               pack_bf16x2(v[8 * h], v[8 * h + 1]), pack_bf16x2(v[8 * h + 2], v[8 * h + 3]),
               pack_bf16x2(v[8 * h + 4], v[8 * h + 5]), pack_bf16x2(v[8 * h + 6], v[8 * h + 7]));
    } else {
#pragma unroll
      for (int e4 = 0; e4 < 4; ++e4)
        sts128f(stg + (uint32_t)(lane * 64 + ((e4 ^ ((lane >> 1) & 3)) << 4)), v[4 * e4], v[4 * e4 + 1],
                v[4 * e4 + 2], v[4 * e4 + 3]);
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      if (convt)
        tma_store_4d(&a.ymap, stg, ch0, up ? pd.ox2 : pd.ox, 2 * bi0 + (up ? pd.oy2 : pd.oy), bn0);
      else
        tma_store_2d(&a.ymap, stg, col0, row0);
      bulk_commit();
      if constexpr (SKT) {
        if (skt && cc + EPI_TMA_BOXES - 1 < nch) {  // into the box of chunk cc - 1, once its store has read it
          bulk_wait_read<1>();
          issue_skip(cc + EPI_TMA_BOXES - 1);
        }
      }
    }
  }
  if constexpr (FOLD) {
    if (head && vrow) {
#pragma unroll
      for (int o = 0; o < KHEAD_MAX; ++o)
        if (o < a.head_cout) a.head_out[((size_t)n * a.head_cout + o) * rows_per_map + rem] = fmaxf(hacc[o], 0.f);
    }
  }
  return true;
}

template <int PREC, bool FOLD>
__device__ __forceinline__ bool epi_tile_staged(const ConvArgs &a, uint32_t taddr, int BN, int n0, size_t ebase,
                                                bool vrow, float *stg, unsigned long long &w_tfull, uint32_t tfull,
                                                uint32_t par, unsigned long long &w_ld, uint32_t t2) {
  const int lane = threadIdx.x & 31;
  size_t er[4];
  bool vr[4];
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int src = it * 8 + (lane >> 2);
    er[it] = ((size_t)__shfl_sync(0xffffffffu, (unsigned)(ebase >> 32), src) << 32) |
             (size_t)__shfl_sync(0xffffffffu, (unsigned)ebase, src);
    vr[it] = __shfl_sync(0xffffffffu, vrow ? 1 : 0, src) != 0;
  }
  const int q = lane & 3;
  float4 *stg4 = reinterpret_cast<float4 *>(stg);
  // skip values one chunk ahead: chunk 0's before the accumulator is ready,
  // each next chunk's as soon as the previous chunk has used its registers
  float4 sk[4];
  auto load_skip4 = [&](int cc) {
    const int col0 = n0 + cc * 16;
#pragma unroll
    for (int it = 0; it < 4; ++it)
      if (vr[it]) sk[it] = ld4<PREC>(a.skip, er[it] + col0 + 4 * q, a.skip_scale ? a.skip_scale + col0 + 4 * q : nullptr);
  };
  if (a.skip) load_skip4(0);
  if (!pwait(a, w_tfull, tfull, par)) return false;
  tc_fence_after();
  for (int cc = 0; cc < BN / 16; ++cc) {
    const int col0 = n0 + cc * 16;
    float v[16];
    const long long tl0 = a.prof ? clock64() : 0;
    tmem_ld_acc<PREC, FOLD>(taddr + cc * 16, acc_at<FOLD>(FOLD ? t2 : taddr + (uint32_t)BN, cc * 16), v);
    if (a.prof) w_ld += (unsigned long long)(clock64() - tl0);
    const float *bsc = a.bscale ? a.bscale + col0 : nullptr;
    const float4 *bias4 = reinterpret_cast<const float4 *>(a.bias + col0);
#pragma unroll
    for (int e4 = 0; e4 < 4; ++e4) {
      const float4 b = __ldg(bias4 + e4);
      const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float z = bsc ? v[4 * e4 + e] * __ldg(bsc + 4 * e4 + e) : v[4 * e4 + e];
        z += bb[e];
        if (a.relu) z = act_fn<FOLD>(a, z);
        v[4 * e4 + e] = z;
      }
    }
#pragma unroll
    for (int e4 = 0; e4 < 4; ++e4)
      stg4[lane * 5 + e4] = make_float4(v[4 * e4], v[4 * e4 + 1], v[4 * e4 + 2], v[4 * e4 + 3]);
    __syncwarp();
    float4 mx = make_float4(0.f, 0.f, 0.f, 0.f);  // calibration: max |stored value| of this lane's columns
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      if (!vr[it]) continue;
      const int r = it * 8 + (lane >> 2);
      float4 x = stg4[r * 5 + q];
      const size_t e = er[it] + col0 + 4 * q;  // er: the row's first element; col0 includes the N tile
      if constexpr (PREC != PREC_FP8) {
        if (a.y2 && a.y2_pre_skip) st4<PREC>(a.y2, e, x, nullptr);
      }
      if (a.skip) {
        x.x += sk[it].x;
        x.y += sk[it].y;
        x.z += sk[it].z;
        x.w += sk[it].w;
      }
      if constexpr (PREC != PREC_FP8) {
        if (a.y2 && !a.y2_pre_skip) st4<PREC>(a.y2, e, x, nullptr);
        if (a.mask) {
          const float4 mk = ld4<PREC>(a.mask, e, nullptr);
          if (!(mk.x > 0.f)) x.x = 0.f;
          if (!(mk.y > 0.f)) x.y = 0.f;
          if (!(mk.z > 0.f)) x.z = 0.f;
          if (!(mk.w > 0.f)) x.w = 0.f;
        }
      }
      if (a.amax) {
        mx.x = fmaxf(mx.x, fabsf(x.x));
        mx.y = fmaxf(mx.y, fabsf(x.y));
        mx.z = fmaxf(mx.z, fabsf(x.z));
        mx.w = fmaxf(mx.w, fabsf(x.w));
      }
      st4<PREC>(a.y, e, x, a.out_qinv ? a.out_qinv + col0 + 4 * q : nullptr);
    }
    if (a.skip && cc + 1 < BN / 16) load_skip4(cc + 1);
    if (a.amax) {  // lanes with the same q hold the same columns
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        mx.x = fmaxf(mx.x, __shfl_xor_sync(0xffffffffu, mx.x, o));
        mx.y = fmaxf(mx.y, __shfl_xor_sync(0xffffffffu, mx.y, o));
        mx.z = fmaxf(mx.z, __shfl_xor_sync(0xffffffffu, mx.z, o));
        mx.w = fmaxf(mx.w, __shfl_xor_sync(0xffffffffu, mx.w, o));
      }
      if (lane < 4) {
        unsigned *am = a.amax + col0 + 4 * q;
        if (mx.x > 0.f) atomicMax(am, __float_as_uint(mx.x));
        if (mx.y > 0.f) atomicMax(am + 1, __float_as_uint(mx.y));
        if (mx.z > 0.f) atomicMax(am + 2, __float_as_uint(mx.z));
        if (mx.w > 0.f) atomicMax(am + 3, __float_as_uint(mx.w));
      }
    }
    __syncwarp();
  }
  return true;
}

// MMA issue loop of one CTA (one thread): per tile (or accumulation chunk)
// wait for a free accumulator, per K block wait for the stage and issue its
// MMAs, then hand the accumulator to the epilogue.  TS: A from tensor memory
// (split-tf32).  FOLD (with TS): accumulation chunks, all three products of
// a K block into the chunk's one accumulator, the two small correction
// products first.
template <int PREC, bool TS, bool PROF, bool TAPA, bool FOLD, bool HIRAW>
__device__ __forceinline__ void mma_issue(const ConvArgs &a, uint32_t data_u32, int sbytes, int a_bytes,
                                          int b_bytes, int stages, int total_tiles, int nbufs, int acc_cols,
                                          uint32_t acc_base, uint32_t a_col0,
                                          uint32_t tmem_base, uint64_t *full_bar, uint64_t *empty_bar,
                                          uint64_t *tfull_bar, uint64_t *tempty_bar, unsigned long long &w_full,
                                          unsigned long long &w_tempty, uint32_t raw_u32, int R, int slot_bytes,
                                          uint64_t *raw_empty) {
  using T = PrecTraits<PREC>;
  const int BN = a.BN;
  const unsigned long long tmo = a.timeout_ns;
  int *const status = a.status;
  // the wait-time accounting is compiled in only where it is on (PROF)
  auto pwait = [&](const ConvArgs &, unsigned long long &acc, uint32_t bar, uint32_t parity) -> bool {
    if constexpr (PROF) {
      const long long t0 = clock64();
      const bool r = mbar_wait(bar, parity, tmo, status, ERR_TIMEOUT);
      acc += (unsigned long long)(clock64() - t0);
      return r;
    } else {
      return mbar_wait(bar, parity, tmo, status, ERR_TIMEOUT);
    }
  };
  bool ok = true;
  const uint32_t idesc = make_idesc(T::KIND, BM, BN);
  // TAPA, BF16 tap boxes: A is K-major without swizzle, 2 KB per 8-element
  // K group (one tap box), 128 bytes per 8-row group; a 16-element K step
  // spans two groups (4096 bytes = 256 units).  TAPA, FP8 tap boxes of 64
  // channels: two 64-byte-swizzled boxes of 8 KB (512 units) per K block, two
  // 32-element K steps in each (+2 units).
  constexpr bool TAP8 = TAPA && PREC == PREC_FP8;
  const uint64_t dA0 = TAP8 ? make_sdesc_sw64(data_u32)
                            : (TAPA ? make_sdesc_kmajor_plain(data_u32, BM * 16, 128) : make_sdesc_sw128(data_u32));
  constexpr uint32_t kA = TAPA ? 256u : 2u;
  auto a_step = [&](int k) -> uint32_t { return TAP8 ? (uint32_t)((k >> 1) * 512 + (k & 1) * 2) : kA * (uint32_t)k; };
  const uint32_t dstage = (uint32_t)sbytes >> 4, dAlo = (uint32_t)a_bytes >> 4;
  const uint64_t dB0 = make_sdesc_sw128(data_u32 + (uint32_t)(TS ? 0 : T::SPLIT * a_bytes));
  const uint32_t dBlo = (uint32_t)b_bytes >> 4;
  // HIRAW: A_hi is K block j's raw slot (j mod R), released by the commit
  const uint64_t dR0 = make_sdesc_sw128(raw_u32);
  const uint32_t dslot = (uint32_t)slot_bytes >> 4;
  int rslot = 0;
  int stage = 0;
  uint32_t phase = 0;
  int it = 0;  // accumulator units: tiles, or with a.kfold chunks of a.kfold K blocks of a tile
  for (int t = blockIdx.x; ok && t < total_tiles; t += gridDim.x) {
    const TileCoord tc = tile_coord(a, t);
    const int nkb = a.ph[tc.phase].num_kb;
    // FOLD: one accumulator unit per a.kfold K blocks; else the whole tile
    int k0 = 0;
    do {
      const int k1 = FOLD ? (k0 + a.kfold < nkb ? k0 + a.kfold : nkb) : nkb;
      const int buf = nbufs == 2 ? (it & 1) : 0;
      const uint32_t par = (uint32_t)((nbufs == 2 ? (it >> 1) : it) & 1);
      if (!pwait(a, w_tempty, smem_u32(&tempty_bar[buf]), par ^ 1)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + acc_base + (uint32_t)(buf * acc_cols);
      const uint32_t c_tmem = d_tmem + (uint32_t)BN;  // correction accumulator (split-tf32, not FOLD)
      for (int kb = k0; kb < k1; ++kb) {
        if (!pwait(a, w_full, smem_u32(&full_bar[stage]), phase)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // descriptors: the stage-0 A tile's plus fixed offsets in units of
        // the start-address field (bytes >> 4); the K step inside the
        // 128-byte swizzle row adds 32 bytes (2 units).  Keeping this to a
        // few adds matters: one thread issues every MMA, so its dependent
        // instruction latency bounds the MMA rate.
        const uint64_t sd = dA0 + (uint64_t)((uint32_t)stage * dstage);
        const uint64_t bd0 = dB0 + (uint64_t)((uint32_t)stage * dstage), bd1 = bd0 + dBlo;
        if constexpr (TS) {
          // A hi/lo from tensor memory: 8 tf32 columns per K step
          const uint32_t ta = tmem_base + a_col0 + (uint32_t)(stage * 64);
          const uint32_t acc0 = kb != k0;
          if constexpr (FOLD) {
            // A_hi B_lo and A_lo B_hi while the accumulator holds only small
            // terms (their rounding is then negligible), then A_hi B_hi
            tc_mma_ts_tf32(d_tmem, ta, bd1, idesc, acc0);
            tc_mma_ts_tf32(d_tmem, ta + 32, bd0, idesc, 1u);
#pragma unroll
            for (int k = 1; k < KROW_BYTES / 32; ++k) {
              tc_mma_ts_tf32(d_tmem, ta + 8 * k, bd1 + 2 * k, idesc, 1u);
              tc_mma_ts_tf32(d_tmem, ta + 32 + 8 * k, bd0 + 2 * k, idesc, 1u);
            }
#pragma unroll
            for (int k = 0; k < KROW_BYTES / 32; ++k) tc_mma_ts_tf32(d_tmem, ta + 8 * k, bd0 + 2 * k, idesc, 1u);
          } else {
            tc_mma_ts_tf32(d_tmem, ta, bd0, idesc, acc0);
            tc_mma_ts_tf32(c_tmem, ta, bd1, idesc, acc0);
            tc_mma_ts_tf32(c_tmem, ta + 32, bd0, idesc, 1u);
#pragma unroll
            for (int k = 1; k < KROW_BYTES / 32; ++k) {
              tc_mma_ts_tf32(d_tmem, ta + 8 * k, bd0 + 2 * k, idesc, 1u);
              tc_mma_ts_tf32(c_tmem, ta + 8 * k, bd1 + 2 * k, idesc, 1u);
              tc_mma_ts_tf32(c_tmem, ta + 32 + 8 * k, bd0 + 2 * k, idesc, 1u);
            }
          }
        } else {
          const uint64_t ad1 = sd + dAlo;
          const uint64_t ah = HIRAW ? dR0 + (uint64_t)((uint32_t)rslot * dslot) : sd;
          const uint32_t acc0 = kb != k0;
          if constexpr (HIRAW) {
            tc_mma<T::KIND>(d_tmem, ah, bd0, idesc, acc0);
            tc_mma<T::KIND>(c_tmem, ah, bd1, idesc, acc0);
            tc_mma<T::KIND>(c_tmem, ad1, bd0, idesc, 1u);
#pragma unroll
            for (int k = 1; k < KROW_BYTES / 32; ++k) {
              tc_mma<T::KIND>(d_tmem, ah + 2u * k, bd0 + 2 * k, idesc, 1u);
              tc_mma<T::KIND>(c_tmem, ah + 2u * k, bd1 + 2 * k, idesc, 1u);
              tc_mma<T::KIND>(c_tmem, ad1 + 2u * k, bd0 + 2 * k, idesc, 1u);
            }
          } else {
          tc_mma<T::KIND>(d_tmem, sd, bd0, idesc, acc0);
          if constexpr (PREC == PREC_TF32X3) {
            tc_mma<T::KIND>(c_tmem, sd, bd1, idesc, acc0);
            tc_mma<T::KIND>(c_tmem, ad1, bd0, idesc, 1u);
          }
#pragma unroll
          for (int k = 1; k < KROW_BYTES / 32; ++k) {
            tc_mma<T::KIND>(d_tmem, sd + a_step(k), bd0 + 2 * k, idesc, 1u);
            if constexpr (PREC == PREC_TF32X3) {
              tc_mma<T::KIND>(c_tmem, sd + kA * k, bd1 + 2 * k, idesc, 1u);
              tc_mma<T::KIND>(c_tmem, ad1 + kA * k, bd0 + 2 * k, idesc, 1u);
            }
          }
          }
        }
        tc_commit(smem_u32(&empty_bar[stage]));
        if constexpr (HIRAW) {
          tc_commit(smem_u32(&raw_empty[rslot]));
          rslot = rslot + 1 == R ? 0 : rslot + 1;
        }
        stage = stage + 1 == stages ? 0 : stage + 1;  // selects, not a branch
        phase ^= stage == 0 ? 1u : 0u;
      }
      if (!ok) break;
      tc_commit(smem_u32(&tfull_bar[buf]));
      ++it;
      k0 = k1;
    } while (FOLD && k0 < nkb);
  }
}

// YTMA: the FP32 encoder form whose epilogue stores tiles by TMA (a.y_tma),
// compiled apart so that the other layers carry none of its code.
// FOLD: the U-Net form -- accumulation chunks and LeakyReLU (TF32X3 with A
// in tensor memory only), compiled apart like YTMA.
template <int PREC, bool YTMA, bool FOLD, int EPI>
__global__ void __launch_bounds__(NUM_THREADS, 1) conv_tc_kernel(const __grid_constant__ ConvArgs a) {
  using T = PrecTraits<PREC>;
  const int BN = a.BN;
  constexpr bool fold = FOLD;
  const SmemPlan plan = smem_plan(PREC, BN, a.prod_mode, YTMA ? 1 : 0, fold ? 1 : 0);
  const int stages = plan.stages;
  const int a_bytes = BM * KROW_BYTES;
  const int b_bytes = BN * KROW_BYTES;
  const int sbytes = stage_bytes(PREC, BN, a.prod_mode);
  const bool ts = PREC == PREC_TF32X3 && a.prod_mode == PROD_TMA_TMEM;

  extern __shared__ uint8_t smem_raw[];
  // control block at the start, stage buffers from the next 1024-byte
  // boundary, raw ring after the stages
  uint8_t *ctrl = smem_raw;
  uint64_t *full_bar = reinterpret_cast<uint64_t *>(ctrl);  // [8]
  uint64_t *empty_bar = full_bar + 8;                        // [8]
  uint64_t *tfull_bar = empty_bar + 8;                       // [2]
  uint64_t *tempty_bar = tfull_bar + 2;                      // [2]
  uint64_t *stall_bar = tempty_bar + 2;                      // [1]
  uint64_t *raw_full = stall_bar + 1;                        // [RAW_MAX]
  uint64_t *raw_empty = raw_full + RAW_MAX;                  // [RAW_MAX]
  uint64_t *skip_bar = raw_empty + RAW_MAX;                  // [4 * EPI_TMA_BOXES]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(skip_bar + 4 * EPI_TMA_BOXES);
  static_assert((8 + 8 + 2 + 2 + 1 + 2 * RAW_MAX + 4 * EPI_TMA_BOXES) * 8 + 4 <= SMEM_CTRL, "control block");
  const uint32_t base_u32 = smem_u32(smem_raw);
  const uint32_t data_u32 = (base_u32 + SMEM_CTRL + 1023u) & ~1023u;
  uint8_t *data = smem_raw + (data_u32 - base_u32);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // Accumulator layout per tile buffer: BN columns, or for the split-tf32
  // path [hi*hi | hi*lo + lo*hi] (2 BN columns).  Keeping the two small
  // correction products out of the main accumulator matters: the tensor core
  // rounds the accumulator on every MMA, so three MMAs into one accumulator
  // triple its rounding error.  Two buffers when they fit in 512 columns.
  // With A in tensor memory (PROD_TMA_TMEM) the accumulators share the 512
  // columns with the A stages.  Accumulation chunks (fold): the running sum
  // at column 0, then two chunk buffers of BN columns, each taking all
  // three products (the correction products first).
  const int acc_cols = fold ? BN : T::SPLIT * BN;
  const uint32_t acc_base = fold ? (uint32_t)BN : 0u;
  const uint32_t a_col0 = (uint32_t)ts_a_col0(BN, fold ? 1 : 0);
  const int nbufs = fold ? 2 : (ts ? (2 * acc_cols <= TS_A_COL0 ? 2 : 1) : (2 * acc_cols <= 512 ? 2 : 1));
  const int need = ts ? 512 : nbufs * acc_cols;
  const uint32_t ncols =
      need <= 32 ? 32u : (need <= 64 ? 64u : (need <= 128 ? 128u : (need <= 256 ? 256u : 512u)));

  if (warp == MMA_WARP) {
    tmem_alloc(smem_u32(tmem_slot), ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    // full: the B loader's arrive + one per producer warp, or the A-TMA
    // thread's arrive in PROD_TMA_DIRECT
    // PROD_CPASYNC: all eight producer warps fill every stage; the TMA
    // convert modes: one group of four
    const uint32_t full_count = a.prod_mode == PROD_TMA_DIRECT
                                    ? 2u
                                    : (a.prod_mode == PROD_CPASYNC ? (uint32_t)(NUM_PROD_THREADS / 32 + 1) : 5u);
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), full_count);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull_bar[b]), 1);
      mbar_init(smem_u32(&tempty_bar[b]), 4);
    }
    mbar_init(smem_u32(stall_bar), 1);
    for (int r = 0; r < plan.raw_depth; ++r) {
      mbar_init(smem_u32(&raw_full[r]), 1);                        // the TMA thread's arrive
      // one arrive per warp of the converting group, or the MMAs' commit where
      // they read A_hi from the raw slot
      mbar_init(smem_u32(&raw_empty[r]), a.hi_raw ? 1u : 4u);
    }
    for (int b = 0; b < 4 * EPI_TMA_BOXES; ++b) mbar_init(smem_u32(&skip_bar[b]), 1);  // the epilogue lane's arrive
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // GEMM rows of this launch: fixed, or read from device memory (a graph
  // captured once serves every count up to a.N)
  const int M = gemm_rows(a);
  const int total_tiles = a.num_phases * ((M + BM - 1) / BM) * a.n_tiles;
  const unsigned long long tmo = a.timeout_ns;

  if (warp == MMA_WARP) {
    if (lane == 0) {
      bool ok = true;
      if (a.debug_stall) ok = mbar_wait(smem_u32(stall_bar), 0, tmo, a.status, ERR_TIMEOUT);
      unsigned long long w_full = 0, w_tempty = 0;
      const long long t_start = a.prof ? clock64() : 0;
      // one instantiation per A form: a branch between the forms inside the
      // issue loop measured ~110 cycles per MMA against 45-64 without
      if (ok) {
#define DRC_MMA_ISSUE(TSV, PROFV, TAPV, FOLDV, HIV)                                                              \
  mma_issue<PREC, TSV, PROFV, TAPV, FOLDV, HIV>(a, data_u32, sbytes, a_bytes, b_bytes, stages, total_tiles, nbufs,  \
                                                acc_cols, acc_base, a_col0, tmem_base, full_bar, empty_bar,         \
                                                tfull_bar, tempty_bar, w_full, w_tempty,                            \
                                                smem_u32(data + stages * sbytes), plan.raw_depth,                  \
                                                plan.raw_slot_bytes, raw_empty)
        constexpr bool kTS = PREC == PREC_TF32X3;
        constexpr bool kTAP = PREC == PREC_BF16 || PREC == PREC_FP8;  // tap boxes land in the A tile itself
        const bool tapa = kTAP && a.tap_boxes && a.prod_mode == PROD_TMA_DIRECT;
        // the decoder forms only (the encoders' form carries none of its code)
        constexpr bool kHI = kTS && (EPI == EPI_SKIP || EPI == EPI_PAIR);
        const bool hiraw = kHI && a.hi_raw;
        if (a.prof) {
          if constexpr (FOLD)
            DRC_MMA_ISSUE(kTS, true, false, kTS, false);
          else if (kTS && ts)
            DRC_MMA_ISSUE(kTS, true, false, false, false);
          else if (tapa)
            DRC_MMA_ISSUE(false, true, kTAP, false, false);
          else if (hiraw)
            DRC_MMA_ISSUE(false, true, false, false, kHI);
          else
            DRC_MMA_ISSUE(false, true, false, false, false);
        } else {
          if constexpr (FOLD)
            DRC_MMA_ISSUE(kTS, false, false, kTS, false);
          else if (kTS && ts)
            DRC_MMA_ISSUE(kTS, false, false, false, false);
          else if (tapa)
            DRC_MMA_ISSUE(false, false, kTAP, false, false);
          else if (hiraw)
            DRC_MMA_ISSUE(false, false, false, false, kHI);
          else
            DRC_MMA_ISSUE(false, false, false, false, false);
        }
#undef DRC_MMA_ISSUE
      }
      if (a.prof) {
        atomicAdd(&a.prof[PROF_MMA_WAIT_FULL], w_full);
        atomicAdd(&a.prof[PROF_MMA_WAIT_TEMPTY], w_tempty);
        atomicAdd(&a.prof[PROF_MMA_TOTAL], (unsigned long long)(clock64() - t_start));
        atomicAdd(&a.prof[PROF_CTAS], 1ull);
      }
    }
  } else if (warp == BLOAD_WARP) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      unsigned long long w_empty = 0;
      for (int t = blockIdx.x; ok && t < total_tiles; t += gridDim.x) {
        const TileCoord tc = tile_coord(a, t);
        const PhaseDesc &pd = a.ph[tc.phase];
        const int nkb = pd.num_kb;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!pwait(a, w_empty, smem_u32(&empty_bar[stage]), phase ^ 1)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          mbar_arrive_expect_tx(fb, (uint32_t)(T::SPLIT * b_bytes));
          const size_t off = (size_t)pd.b_off + ((size_t)tc.n_tile * nkb + kb) * (size_t)b_bytes;
          const uint32_t sb0 = data_u32 + stage * sbytes + (ts ? 0 : T::SPLIT * a_bytes);
          bulk_g2s(sb0, a.B + off, (uint32_t)b_bytes, fb);
          if constexpr (PREC == PREC_TF32X3) bulk_g2s(sb0 + b_bytes, a.B_lo + off, (uint32_t)b_bytes, fb);
          if (++stage == stages) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (a.prof) atomicAdd(&a.prof[PROF_BLOAD_WAIT_EMPTY], w_empty);
    }
  } else if (warp == TMA_ISSUE_WARP && (a.prod_mode == PROD_TMA_CONVERT || a.prod_mode == PROD_TMA_TMEM)) {
    if (lane == 0)
      tma_issue_loop<PREC>(a, smem_u32(data + stages * sbytes), raw_full, raw_empty, plan.raw_depth,
                           plan.raw_slot_bytes, total_tiles);
  } else if (warp >= PROD_WARP0) {
    run_producer<PREC, PREC == PREC_TF32X3 && (EPI == EPI_SKIP || EPI == EPI_PAIR)>(a, data, data + stages * sbytes, full_bar, empty_bar, raw_full, raw_empty, stages, sbytes,
                       plan.raw_depth, plan.raw_slot_bytes, M, total_tiles, tmem_base);
  } else if (warp >= EPI_WARP0 && warp < EPI_WARP0 + 4) {
    // ------------------------------------------------------------ epilogue
    const int eq = warp - EPI_WARP0;  // TMEM lane quarter
    const int row = eq * 32 + lane;
    const int rows_per_map = a.Hrow * a.Wrow;
    int it = 0;
    unsigned long long w_tfull = 0, w_ld = 0;
    const long long t_start = a.prof ? clock64() : 0;
    using act_t = typename T::act_t;
    uint8_t *yout = reinterpret_cast<uint8_t *>(a.y);
    const int out_elem = a.out_qinv ? 1 : (int)sizeof(act_t);  // e4m3, or the activation type
    const act_t *skip = reinterpret_cast<const act_t *>(a.skip);
    const int nch = BN / 16;
    float *epi_stg = reinterpret_cast<float *>(data + (size_t)stages * sbytes + (size_t)plan.raw_depth * plan.raw_slot_bytes);
    // this lane quarter's tensor-memory rows; with accumulation chunks the
    // running sum is at column 0
    const uint32_t lanebase = tmem_base + ((uint32_t)(eq * 32) << 16);
    int tma_box = 0;      // next box of this warp's TMA staging ring
    uint32_t skpar = 0;   // per box: parity of its next skip load
    bool failed = false;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++it) {
      const TileCoord tc = tile_coord(a, t);
      const PhaseDesc &pd = a.ph[tc.phase];
      // every chunk but the last: added into the running sum (round to
      // nearest), then the chunk buffer goes back to the MMA warp
      int nchunk = 1;
      if constexpr (FOLD) {
      nchunk = (pd.num_kb + a.kfold - 1) / a.kfold;
      for (int q = 0; q + 1 < nchunk; ++q, ++it) {
        const int fbuf = nbufs == 2 ? (it & 1) : 0;
        const uint32_t fpar = (uint32_t)((nbufs == 2 ? (it >> 1) : it) & 1);
        if (!pwait(a, w_tfull, smem_u32(&tfull_bar[fbuf]), fpar)) {
          failed = true;
          break;
        }
        tc_fence_after();
        const uint32_t faddr = lanebase + acc_base + (uint32_t)(fbuf * acc_cols);
        for (int cc = 0; cc < nch; ++cc) {
          uint32_t x[16], r[16];
          tmem_ld16_nowait(faddr + cc * 16, x);
          if (q > 0) tmem_ld16_nowait(lanebase + cc * 16, r);
          tmem_wait_ld();
          if (q > 0) {
#pragma unroll
            for (int e = 0; e < 16; ++e) x[e] = __float_as_uint(__uint_as_float(x[e]) + __uint_as_float(r[e]));
          }
          tmem_st16(lanebase + cc * 16, x);
        }
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[fbuf]));
      }
      }
      if (failed) break;
      const int buf = nbufs == 2 ? (it & 1) : 0;
      const uint32_t par = (uint32_t)((nbufs == 2 ? (it >> 1) : it) & 1);
      // the tile's accumulator and the one added to it: the correction
      // accumulator, or with chunks the running sum (none for one chunk)
      const uint32_t taddr = lanebase + acc_base + (uint32_t)(buf * acc_cols);
      const uint32_t t2 = PREC != PREC_TF32X3 ? kNoAcc : (!fold ? taddr + (uint32_t)BN : (nchunk > 1 ? lanebase : kNoAcc));
      const int m = tc.m_tile * BM + row;
      const bool vrow = m < M;
      const int n = vrow ? m / rows_per_map : 0;
      const int rem = vrow ? m - n * rows_per_map : 0;
      const int i = rem / a.Wrow, j = rem - (rem / a.Wrow) * a.Wrow;
      const size_t opix = a.kind == LK_CONVT
                              ? ((size_t)n * a.Hout + (2 * i + pd.oy)) * a.Wout + (2 * j + pd.ox)
                              : (size_t)m;
      const size_t ebase = opix * a.Cout + (size_t)tc.n_tile * BN;
      if (YTMA && plan.epi_stage) {
        if (!epi_tile_tma<PREC, FOLD, EPI>(a, taddr, BN, tc.n_tile * BN, tc.m_tile * BM + eq * 32, pd,
                                smem_u32(epi_stg) + (uint32_t)(eq * EPI_TMA_BOXES * EPI_TMA_BOX_BYTES), tma_box,
                                w_tfull, smem_u32(&tfull_bar[buf]), par, w_ld, t2,
                                smem_u32(&skip_bar[eq * EPI_TMA_BOXES]), skpar))
          break;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[buf]));
        continue;
      }
      if (plan.epi_stage) {
        if (!epi_tile_staged<PREC, FOLD>(a, taddr, BN, tc.n_tile * BN, opix * a.Cout, vrow, epi_stg + eq * 32 * 20, w_tfull,
                                   smem_u32(&tfull_bar[buf]), par, w_ld, t2))
          break;
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[buf]));
        continue;
      }
      // Per-row path: each lane stores its own row.  BF16 / FP8 load the
      // skip values of the first two 16-column chunks before the accumulator
      // is ready (their latency hides behind the tile's MMAs) and later
      // chunks two ahead; each element is read (skip) and written by this
      // thread only, so reading ahead of the in-place store is safe.  The
      // FP32 kernel only takes this path when the staging buffer does not
      // fit and loads each chunk's skip just before use (fewer registers).
      const bool has_skip = skip != nullptr && vrow;
      uint8_t *yb = yout + ebase * out_elem;
      if constexpr (PREC == PREC_TF32X3) {
        if (!pwait(a, w_tfull, smem_u32(&tfull_bar[buf]), par)) break;
        tc_fence_after();
        for (int cc = 0; cc < nch; ++cc) {
          uint4 sk[4];
          if (has_skip) load_skip<PREC>(skip + ebase + cc * 16, sk);
          epi_chunk<PREC, FOLD>(a, taddr, cc, BN, tc.n_tile * BN + cc * 16, vrow, has_skip, sk, yb + cc * 16 * out_elem,
                          ebase + cc * 16, t2);
        }
      } else {
        uint4 sk0[4], sk1[4];
        if (has_skip) {
          load_skip<PREC>(skip + ebase, sk0);
          if (nch > 1) load_skip<PREC>(skip + ebase + 16, sk1);
        }
        if (!pwait(a, w_tfull, smem_u32(&tfull_bar[buf]), par)) break;
        tc_fence_after();
        for (int cc = 0; cc < nch; cc += 2) {
          epi_chunk<PREC, FOLD>(a, taddr, cc, BN, tc.n_tile * BN + cc * 16, vrow, has_skip, sk0, yb + cc * 16 * out_elem,
                          ebase + cc * 16, t2);
          if (has_skip && cc + 2 < nch) load_skip<PREC>(skip + ebase + (cc + 2) * 16, sk0);
          if (cc + 1 < nch) {
            epi_chunk<PREC, FOLD>(a, taddr, cc + 1, BN, tc.n_tile * BN + (cc + 1) * 16, vrow, has_skip, sk1,
                            yb + (cc + 1) * 16 * out_elem, ebase + (cc + 1) * 16, t2);
            if (has_skip && cc + 3 < nch) load_skip<PREC>(skip + ebase + (cc + 3) * 16, sk1);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[buf]));
    }
    if (YTMA && plan.epi_stage && lane == 0) bulk_wait0();  // no store in flight at exit
    if (a.prof && lane == 0) {
      atomicAdd(&a.prof[PROF_EPI_WAIT_TFULL], w_tfull);
      atomicAdd(&a.prof[PROF_EPI_LD], w_ld);
      atomicAdd(&a.prof[PROF_EPI_TOTAL], (unsigned long long)(clock64() - t_start));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, ncols);
  }
}

template <int PREC, bool YTMA, bool FOLD, int EPI = EPI_PLAIN>
static cudaError_t launch_form(const ConvArgs &a, int grid, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<PREC, YTMA, FOLD, EPI>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  conv_tc_kernel<PREC, YTMA, FOLD, EPI><<<grid, NUM_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_conv(const ConvArgs &a, int prec, int num_sms, cudaStream_t st) {
  const int total = a.num_phases * a.m_tiles * a.n_tiles;
  if (total == 0) return cudaSuccess;
  const int grid = total < num_sms ? total : num_sms;
  // the U-Net form: accumulation chunks, LeakyReLU (its slope only there)
  const bool fold = a.kfold > 0;
  if (a.kfold < 0 || (fold && (prec != PREC_TF32X3 || a.prod_mode != PROD_TMA_TMEM || a.BN > KFOLD_MAX_BN)) ||
      (!fold && a.slope != 0.f) ||
      (a.head_w && (!fold || !a.y_tma || a.kind == LK_CONVT || a.n_tiles != 1 || a.head_cout < 1 ||
                    a.head_cout > KHEAD_MAX || !a.head_out)))
    return cudaErrorInvalidValue;
  // phase pairs: every phase of the launch, through the TMA-store epilogue
  // of the FP32 kernel, one tile of 2 Cout columns
  const bool pair = a.kind == LK_CONVT && a.num_phases > 0 && a.ph[0].pair;
  for (int p = 0; p < a.num_phases; ++p)
    if ((a.ph[p].pair != 0) != pair) return cudaErrorInvalidValue;
  if (pair && (prec != PREC_TF32X3 || fold || !a.y_tma || a.n_tiles != 1 || a.BN != 2 * a.Cout))
    return cudaErrorInvalidValue;
  const size_t smem = conv_smem_bytes(prec, a.BN, a.prod_mode, a.y_tma, fold ? 1 : 0);
  if (a.hi_raw) return cudaErrorInvalidValue;  // launch_conv's own decision
  switch (prec) {
    case PREC_TF32X3: {
      if (fold) return a.y_tma ? launch_form<PREC_TF32X3, true, true>(a, grid, smem, st)
                               : launch_form<PREC_TF32X3, false, true>(a, grid, smem, st);
      // the decoder forms: A_hi from the raw slot where A is in shared memory
      // over whole K-block boxes
      const bool dec = pair || (a.y_tma && a.skip_tma);
      if (dec && a.prod_mode == PROD_TMA_CONVERT && !a.tap_boxes) {
        ConvArgs b = a;
        b.hi_raw = 1;
        return pair ? launch_form<PREC_TF32X3, true, false, EPI_PAIR>(b, grid, smem, st)
                    : launch_form<PREC_TF32X3, true, false, EPI_SKIP>(b, grid, smem, st);
      }
      if (pair) return launch_form<PREC_TF32X3, true, false, EPI_PAIR>(a, grid, smem, st);
      if (a.y_tma && a.skip_tma) return launch_form<PREC_TF32X3, true, false, EPI_SKIP>(a, grid, smem, st);
      return a.y_tma ? launch_form<PREC_TF32X3, true, false>(a, grid, smem, st)
                     : launch_form<PREC_TF32X3, false, false>(a, grid, smem, st);
    }
    case PREC_BF16:
      if (a.y_tma && a.out_qinv) return launch_form<PREC_BF16, true, false, EPI_E4>(a, grid, smem, st);
      return a.y_tma ? launch_form<PREC_BF16, true, false>(a, grid, smem, st)
                     : launch_form<PREC_BF16, false, false>(a, grid, smem, st);
    default:  // FP8 TMA stores are always e4m3
      return a.y_tma ? launch_form<PREC_FP8, true, false, EPI_E4>(a, grid, smem, st)
                     : launch_form<PREC_FP8, false, false>(a, grid, smem, st);
  }
}

// ------------------------------------------------------ first-layer input
// One thread per pixel: 7 coalesced plane loads, log encode of channels 0..2,
// one 32-byte (fp32) or 16-byte (bf16) store of the 8-channel NHWC pixel.
// With a pass slot the input pointer, the map count and the encode flag come
// from device memory, and the kernel also clears the pass's payload.
template <bool BF16>
__global__ void nchw7_to_nhwc8_kernel(const float *__restrict__ in, void *__restrict__ out, long long hw, int N,
                                      int encode, float s, const PassSlot *slot) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot) {
    const int cnt = slot->count;
    N = cnt < 0 ? 0 : (cnt < N ? cnt : N);
    in = slot->in;
    encode = (slot->flags & SLOT_ENCODE) ? 1 : 0;
    if (slot->payload && g < 3ll * N) slot->payload[g] = 0.f;
  }
  if (g >= hw * N) return;
  const long long n = g / hw, p = g - n * hw;
  const float *src = in + n * 7 * hw + p;
  float v[8];
#pragma unroll
  for (int c = 0; c < 7; ++c) v[c] = __ldg(src + c * hw);
  v[7] = 0.f;
  if (encode) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = log1pf(s * v[c]);
  }
  if constexpr (BF16) {
    reinterpret_cast<uint4 *>(out)[g] =
        make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
  } else {
    float4 *o = reinterpret_cast<float4 *>(out) + 2 * g;
    o[0] = make_float4(v[0], v[1], v[2], v[3]);
    o[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
}

cudaError_t launch_nchw7_to_nhwc8(const float *in, void *out, long long hw, int N, bool bf16, bool encode,
                                  float exposure, cudaStream_t st, const PassSlot *slot) {
  long long total = hw * N;
  if (slot && total < 3ll * N) total = 3ll * N;  // payload clear
  if (total == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (bf16)
    nchw7_to_nhwc8_kernel<true><<<blocks, 256, 0, st>>>(in, out, hw, N, encode ? 1 : 0, exposure, slot);
  else
    nchw7_to_nhwc8_kernel<false><<<blocks, 256, 0, st>>>(in, out, hw, N, encode ? 1 : 0, exposure, slot);
  return cudaGetLastError();
}

// --------------------------------------------------------- weight packing
// One thread per 16-byte chunk of the packed B image: chunk (phase, n_tile,
// kb, row r, physical chunk p) holds logical chunk q = p ^ (r & 7) of row r,
// i.e. K elements kb*BKE + q*E .. + E - 1 of output column n_tile*BN + r.
__device__ float raw_weight(const PackArgs &p, const PhaseDesc &pd, int col, int k) {
  const int t = k / p.Cin, c = k - (k / p.Cin) * p.Cin;
  if (t >= pd.ntaps || c >= p.Cin_raw) return 0.f;
  if (p.kind == LK_CONV || p.kind == LK_CONV1)  // W[o][c][u][v], tap t = 3u + v
    return p.wraw[((size_t)col * p.Cin_raw + c) * 9 + t];
  // LK_CONVT: W[c][o][u][v] with the phase's kernel tap
  const int co = p.Cout_raw > 0 ? p.Cout_raw : p.Cout;
  if (pd.pair) {  // columns [co, 2 co): the pair's second phase
    const bool up = col >= co;
    const int o = up ? col - co : col, u = up ? pd.u2[t] : pd.u[t], v = up ? pd.v2[t] : pd.v[t];
    if (u < 0 || v < 0 || o >= co) return 0.f;
    return p.wraw[(((size_t)c * co + o) * 3 + u) * 3 + v];
  }
  if (col >= co) return 0.f;
  return p.wraw[(((size_t)c * co + col) * 3 + pd.u[t]) * 3 + pd.v[t]];
}

template <int PREC>
__global__ void pack_kernel(const __grid_constant__ PackArgs p) {
  using T = PrecTraits<PREC>;
  constexpr int E = 16 / T::ELEM;
  constexpr int BKE = KROW_BYTES / T::ELEM;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= p.total_chunks) return;
  const int chunks_per_tile = p.BN * (KROW_BYTES / 16);
  long long rem = gid;
  int ph = 0;
  for (; ph < p.num_phases; ++ph) {
    const long long nchunks = (long long)p.n_tiles * p.ph[ph].num_kb * chunks_per_tile;
    if (rem < nchunks) break;
    rem -= nchunks;
  }
  const PhaseDesc &pd = p.ph[ph];
  const long long tile = rem / chunks_per_tile;
  const int within = (int)(rem - tile * chunks_per_tile);
  const int n_tile = (int)(tile / pd.num_kb);
  const int kb = (int)(tile - (long long)n_tile * pd.num_kb);
  const int r = within / (KROW_BYTES / 16);
  const int pchunk = within - r * (KROW_BYTES / 16);
  const int q = pchunk ^ (r & 7);
  const int col = n_tile * p.BN + r;
  float w[E];
#pragma unroll
  for (int e = 0; e < E; ++e) w[e] = raw_weight(p, pd, col, kb * BKE + q * E + e);
  const size_t off = (size_t)pd.b_off + (size_t)tile * chunks_per_tile * 16 + (size_t)within * 16;
  if constexpr (PREC == PREC_TF32X3) {
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = tf32_rna(w[e]);
      l[e] = tf32_rna(w[e] - h[e]);
    }
    *reinterpret_cast<float4 *>(p.B + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(p.B_lo + off) = make_float4(l[0], l[1], l[2], l[3]);
  } else if constexpr (PREC == PREC_BF16) {
    uint4 o;
    o.x = pack_bf16x2(w[0], w[1]);
    o.y = pack_bf16x2(w[2], w[3]);
    o.z = pack_bf16x2(w[4], w[5]);
    o.w = pack_bf16x2(w[6], w[7]);
    *reinterpret_cast<uint4 *>(p.B + off) = o;
  } else {
    // W x (input channel scale) / (column scale): the layer's input is stored
    // as x / in_scale[c], so the product dequantises with bscale[col] alone
    const float inv = 1.0f / p.bscale[col];
    const int k0 = kb * BKE + q * E;
#pragma unroll
    for (int e = 0; e < E; ++e) w[e] *= p.in_scale ? __ldg(p.in_scale + (k0 + e) % p.Cin) : 1.f;
    uint4 o;
    o.x = pack_e4m3x4(w[0] * inv, w[1] * inv, w[2] * inv, w[3] * inv);
    o.y = pack_e4m3x4(w[4] * inv, w[5] * inv, w[6] * inv, w[7] * inv);
    o.z = pack_e4m3x4(w[8] * inv, w[9] * inv, w[10] * inv, w[11] * inv);
    o.w = pack_e4m3x4(w[12] * inv, w[13] * inv, w[14] * inv, w[15] * inv);
    *reinterpret_cast<uint4 *>(p.B + off) = o;
  }
}

// FP8: bscale[col] = max over the layer's taps and channels of
// |W[col][k] x in_scale[c]| / 448 (the e4m3 maximum), or 1 for a zero column.
// One block per output column.
__global__ void fp8_colscale_kernel(const __grid_constant__ PackArgs p) {
  const int col = blockIdx.x;
  float m = 0.f;
  for (int ph = 0; ph < p.num_phases; ++ph) {
    const PhaseDesc &pd = p.ph[ph];
    for (int k = threadIdx.x; k < pd.ntaps * p.Cin; k += blockDim.x) {
      const float sc = p.in_scale ? __ldg(p.in_scale + k % p.Cin) : 1.f;
      m = fmaxf(m, fabsf(raw_weight(p, pd, col, k) * sc));
    }
  }
  __shared__ float red[32];
  for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    m = fmaxf(m, red[0]);
    p.bscale[col] = m > 0.f ? m / 448.f : 1.f;
  }
}

cudaError_t launch_pack(const PackArgs &p, int prec, cudaStream_t st) {
  if (p.total_chunks == 0) return cudaSuccess;
  if (prec == PREC_FP8) {
    fp8_colscale_kernel<<<p.Cout, 256, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int threads = 256;
  const unsigned blocks = (unsigned)((p.total_chunks + threads - 1) / threads);
  switch (prec) {
    case PREC_TF32X3:
      pack_kernel<PREC_TF32X3><<<blocks, threads, 0, st>>>(p);
      break;
    case PREC_BF16:
      pack_kernel<PREC_BF16><<<blocks, threads, 0, st>>>(p);
      break;
    default:
      pack_kernel<PREC_FP8><<<blocks, threads, 0, st>>>(p);
      break;
  }
  return cudaGetLastError();
}

}  // namespace drc
