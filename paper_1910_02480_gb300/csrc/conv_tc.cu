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
//   D          = fp32 accumulator in tensor memory, double buffered so the
//                epilogue of tile i overlaps the MMAs of tile i+1.
// Warp roles (16 warps): 0 = MMA issuer + TMEM owner, 1 = B loader,
// 4..7 = epilogue (TMEM lane quarters 0..3), 8..15 = A producers.
// FP32 parity uses the split-tf32 product: x = hi + lo with hi, lo tf32, and
// D += A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped lo*lo term is below
// 2^-21 relative).  BF16 / FP8 use one product per K step.
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
  static constexpr int ELEM = 4;          // bytes per stored operand element
  static constexpr int KIND = KIND_TF32;
  static constexpr int SPLIT = 2;         // hi + lo copies of each operand tile
  using act_t = float;                    // activation storage
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
  using act_t = __nv_bfloat16;  // fp8 path keeps bf16 activations, quantised on load
};

constexpr int SMEM_BUDGET = 227 * 1024;
constexpr int SMEM_CTRL = 1024;  // barriers + TMEM slot, padded to the 1024-byte swizzle atom

__host__ __device__ inline int stage_bytes(int prec, int BN) {
  int split = prec == PREC_TF32X3 ? 2 : 1;
  return split * (BM * KROW_BYTES + BN * KROW_BYTES);
}

__host__ __device__ int conv_stages(int prec, int BN) {
  int s = (SMEM_BUDGET - SMEM_CTRL - 1024) / stage_bytes(prec, BN);
  return s > 8 ? 8 : s;
}
size_t conv_smem_bytes(int prec, int BN) {
  return (size_t)SMEM_CTRL + 1024 + (size_t)conv_stages(prec, BN) * stage_bytes(prec, BN);
}

// Offset of 16-byte chunk q of row r inside a 128-byte-swizzled K-major tile.
__device__ __forceinline__ uint32_t swz(int r, int q) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((q ^ (r & 7)) << 4));
}

struct TileCoord {
  int phase, m_tile, n_tile;
};
__device__ __forceinline__ TileCoord tile_coord(const ConvArgs &a, int t) {
  int per_phase = a.m_tiles * a.n_tiles;
  int p = t / per_phase;
  int rem = t - p * per_phase;
  TileCoord c;
  c.phase = a.phase_order[p];
  c.m_tile = rem / a.n_tiles;
  c.n_tile = rem - c.m_tile * a.n_tiles;
  return c;
}

// ----------------------------------------------------------------- loads
template <int PREC>
struct Chunk;  // one 16-byte slice of an operand row, as loaded
template <>
struct Chunk<PREC_TF32X3> {
  float4 v;
};
template <>
struct Chunk<PREC_BF16> {
  uint4 v;
};
template <>
struct Chunk<PREC_FP8> {
  uint4 v[2];  // 16 bf16 values, quantised to 16 e4m3 on store
};

__device__ __forceinline__ uint4 ldg16(const void *p) {
  return __ldg(reinterpret_cast<const uint4 *>(p));
}

template <int PREC>
__device__ __forceinline__ void load_chunk_nhwc(Chunk<PREC> &c, const uint8_t *src, bool ok) {
  if constexpr (PREC == PREC_TF32X3) {
    c.v = ok ? __ldg(reinterpret_cast<const float4 *>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
  } else if constexpr (PREC == PREC_BF16) {
    c.v = ok ? ldg16(src) : make_uint4(0, 0, 0, 0);
  } else {
    c.v[0] = ok ? ldg16(src) : make_uint4(0, 0, 0, 0);
    c.v[1] = ok ? ldg16(src + 16) : make_uint4(0, 0, 0, 0);
  }
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

// Store one chunk into the stage's A tile(s).
template <int PREC>
__device__ __forceinline__ void store_chunk(uint8_t *a0, uint8_t *a1, uint32_t off, const Chunk<PREC> &c,
                                            float qscale) {
  if constexpr (PREC == PREC_TF32X3) {
    float4 h, l;
    h.x = to_tf32(c.v.x);
    h.y = to_tf32(c.v.y);
    h.z = to_tf32(c.v.z);
    h.w = to_tf32(c.v.w);
    l.x = to_tf32(c.v.x - h.x);
    l.y = to_tf32(c.v.y - h.y);
    l.z = to_tf32(c.v.z - h.z);
    l.w = to_tf32(c.v.w - h.w);
    *reinterpret_cast<float4 *>(a0 + off) = h;
    *reinterpret_cast<float4 *>(a1 + off) = l;
  } else if constexpr (PREC == PREC_BF16) {
    *reinterpret_cast<uint4 *>(a0 + off) = c.v;
  } else {
    uint4 q;
    const uint4 &x = c.v[0];
    const uint4 &y = c.v[1];
    q.x = pack_e4m3x4(bf16_lo(x.x) * qscale, bf16_hi(x.x) * qscale, bf16_lo(x.y) * qscale,
                      bf16_hi(x.y) * qscale);
    q.y = pack_e4m3x4(bf16_lo(x.z) * qscale, bf16_hi(x.z) * qscale, bf16_lo(x.w) * qscale,
                      bf16_hi(x.w) * qscale);
    q.z = pack_e4m3x4(bf16_lo(y.x) * qscale, bf16_hi(y.x) * qscale, bf16_lo(y.y) * qscale,
                      bf16_hi(y.y) * qscale);
    q.w = pack_e4m3x4(bf16_lo(y.z) * qscale, bf16_hi(y.z) * qscale, bf16_lo(y.w) * qscale,
                      bf16_hi(y.w) * qscale);
    *reinterpret_cast<uint4 *>(a0 + off) = q;
  }
}

// Elements of the first layer's K (k = c*9 + tap, c < 7) gathered from the
// fp32 NCHW input, with the optional log encode of channels 0..2.
template <int PREC>
__device__ __forceinline__ void store_nchw7(uint8_t *a0, uint8_t *a1, uint32_t off, const float *vals,
                                            float qscale) {
  if constexpr (PREC == PREC_TF32X3) {
    Chunk<PREC_TF32X3> c;
    c.v = make_float4(vals[0], vals[1], vals[2], vals[3]);
    store_chunk<PREC_TF32X3>(a0, a1, off, c, qscale);
  } else if constexpr (PREC == PREC_BF16) {
    uint4 q;
    q.x = pack_bf16x2(vals[0], vals[1]);
    q.y = pack_bf16x2(vals[2], vals[3]);
    q.z = pack_bf16x2(vals[4], vals[5]);
    q.w = pack_bf16x2(vals[6], vals[7]);
    *reinterpret_cast<uint4 *>(a0 + off) = q;
  } else {
    uint4 q;
    q.x = pack_e4m3x4(vals[0] * qscale, vals[1] * qscale, vals[2] * qscale, vals[3] * qscale);
    q.y = pack_e4m3x4(vals[4] * qscale, vals[5] * qscale, vals[6] * qscale, vals[7] * qscale);
    q.z = pack_e4m3x4(vals[8] * qscale, vals[9] * qscale, vals[10] * qscale, vals[11] * qscale);
    q.w = pack_e4m3x4(vals[12] * qscale, vals[13] * qscale, vals[14] * qscale, vals[15] * qscale);
    *reinterpret_cast<uint4 *>(a0 + off) = q;
  }
}

// Accumulator columns [c, c+16) of a tile: the main accumulator, plus the
// correction accumulator BN columns further on for the split-tf32 path.
template <int PREC>
__device__ __forceinline__ void tmem_ld_acc(uint32_t taddr, int BN, float (&v)[16]) {
  tmem_ld16(taddr, v);
  if constexpr (PREC == PREC_TF32X3) {
    float c[16];
    tmem_ld16(taddr + (uint32_t)BN, c);
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] += c[e];
  }
}

// ------------------------------------------------------------- the kernel
template <int PREC>
__global__ void __launch_bounds__(NUM_THREADS, 1) conv_tc_kernel(const __grid_constant__ ConvArgs a) {
  using T = PrecTraits<PREC>;
  constexpr int E = 16 / T::ELEM;            // elements per 16-byte chunk
  constexpr int BKE = KROW_BYTES / T::ELEM;  // K elements per stage
  const int BN = a.BN;
  const int stages = conv_stages(PREC, BN);
  const int a_bytes = BM * KROW_BYTES;
  const int b_bytes = BN * KROW_BYTES;
  const int sbytes = stage_bytes(PREC, BN);

  extern __shared__ uint8_t smem_raw[];
  // control block at the start, stage buffers from the next 1024-byte boundary
  uint8_t *ctrl = smem_raw;
  uint64_t *full_bar = reinterpret_cast<uint64_t *>(ctrl);        // [8]
  uint64_t *empty_bar = full_bar + 8;                              // [8]
  uint64_t *tfull_bar = empty_bar + 8;                             // [2]
  uint64_t *tempty_bar = tfull_bar + 2;                            // [2]
  uint64_t *stall_bar = tempty_bar + 2;                            // [1]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(stall_bar + 1);
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
  const int acc_cols = T::SPLIT * BN;
  const int nbufs = 2 * acc_cols <= 512 ? 2 : 1;
  const int need = nbufs * acc_cols;
  const uint32_t ncols = need <= 32 ? 32u : (need <= 64 ? 64u : (need <= 128 ? 128u : (need <= 256 ? 256u : 512u)));

  if (warp == MMA_WARP) {
    tmem_alloc(smem_u32(tmem_slot), ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), NUM_PROD_THREADS / 32 + 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull_bar[b]), 1);
      mbar_init(smem_u32(&tempty_bar[b]), 4);
    }
    mbar_init(smem_u32(stall_bar), 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int total_tiles = a.num_phases * a.m_tiles * a.n_tiles;
  const unsigned long long tmo = a.timeout_ns;

  if (warp == MMA_WARP) {
    if (lane == 0) {
      bool ok = true;
      if (a.debug_stall) ok = mbar_wait(smem_u32(stall_bar), 0, tmo, a.status, ERR_TIMEOUT);
      const uint32_t idesc = make_idesc(T::KIND, BM, BN);
      int stage = 0;
      uint32_t phase = 0;
      int it = 0;
      for (int t = blockIdx.x; ok && t < total_tiles; t += gridDim.x, ++it) {
        const TileCoord tc = tile_coord(a, t);
        const int nkb = a.ph[tc.phase].num_kb;
        const int buf = nbufs == 2 ? (it & 1) : 0;
        const uint32_t par = (uint32_t)((nbufs == 2 ? (it >> 1) : it) & 1);
        if (!mbar_wait(smem_u32(&tempty_bar[buf]), par ^ 1, tmo, a.status, ERR_TIMEOUT)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(buf * acc_cols);
        const uint32_t c_tmem = d_tmem + (uint32_t)BN;  // correction accumulator (split-tf32)
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(smem_u32(&full_bar[stage]), phase, tmo, a.status, ERR_TIMEOUT)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa0 = data_u32 + stage * sbytes;
          const uint32_t sa1 = sa0 + a_bytes;                 // A lo (TF32X3)
          const uint32_t sb0 = sa0 + T::SPLIT * a_bytes;      // B (hi)
          const uint32_t sb1 = sb0 + b_bytes;                 // B lo (TF32X3)
#pragma unroll
          for (int k = 0; k < KROW_BYTES / 32; ++k) {
            const uint32_t acc = (kb | k) != 0;
            const uint64_t ad = make_sdesc_sw128(sa0 + k * 32);
            const uint64_t bd = make_sdesc_sw128(sb0 + k * 32);
            tc_mma<T::KIND>(d_tmem, ad, bd, idesc, acc);
            if constexpr (PREC == PREC_TF32X3) {
              tc_mma<T::KIND>(c_tmem, ad, make_sdesc_sw128(sb1 + k * 32), idesc, acc);
              tc_mma<T::KIND>(c_tmem, make_sdesc_sw128(sa1 + k * 32), bd, idesc, 1u);
            }
          }
          tc_commit(smem_u32(&empty_bar[stage]));
          if (++stage == stages) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        tc_commit(smem_u32(&tfull_bar[buf]));
      }
    }
  } else if (warp == BLOAD_WARP) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < total_tiles; t += gridDim.x) {
        const TileCoord tc = tile_coord(a, t);
        const PhaseDesc &pd = a.ph[tc.phase];
        const int nkb = pd.num_kb;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, tmo, a.status, ERR_TIMEOUT)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          mbar_arrive_expect_tx(fb, (uint32_t)(T::SPLIT * b_bytes));
          const size_t off = (size_t)pd.b_off + ((size_t)tc.n_tile * nkb + kb) * (size_t)b_bytes;
          const uint32_t sb0 = data_u32 + stage * sbytes + T::SPLIT * a_bytes;
          bulk_g2s(sb0, a.B + off, (uint32_t)b_bytes, fb);
          if constexpr (PREC == PREC_TF32X3) bulk_g2s(sb0 + b_bytes, a.B_lo + off, (uint32_t)b_bytes, fb);
          if (++stage == stages) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
    }
  } else if (warp >= PROD_WARP0) {
    // ------------------------------------------------------ A producers
    const int pt = threadIdx.x - PROD_WARP0 * 32;  // 0..255
    const int pw = pt >> 5;
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    const int rows_per_map = a.Hrow * a.Wrow;
    const int hw_in = a.Hin * a.Win;
    const float qscale = a.act_scale_in;
    for (int t = blockIdx.x; ok && t < total_tiles; t += gridDim.x) {
      const TileCoord tc = tile_coord(a, t);
      const PhaseDesc &pd = a.ph[tc.phase];
      const int nkb = pd.num_kb;
      if (a.kind == LK_CONV_NCHW7) {
        // one row per thread, half of the 16-byte chunks of that row
        const int r = pt & (BM - 1);
        const int qbase = (pt >> 7) * (KROW_BYTES / 16 / 2);
        const int m = tc.m_tile * BM + r;
        const bool vrow = m < a.M;
        const int n = vrow ? m / rows_per_map : 0;
        const int rem = m - n * rows_per_map;
        const int i = rem / a.Wrow, j = rem - (rem / a.Wrow) * a.Wrow;
        const int y0 = 2 * i - 1, x0 = 2 * j - 1;
        const float *xin = reinterpret_cast<const float *>(a.x) + (size_t)n * 7 * hw_in;
        for (int kb = 0; kb < nkb; ++kb) {
          float vals[KROW_BYTES / 16 / 2][E];
#pragma unroll
          for (int qq = 0; qq < KROW_BYTES / 16 / 2; ++qq) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int k = kb * BKE + (qbase + qq) * E + e;
              const int c = k / 9, tap = k - (k / 9) * 9;
              const int yy = y0 + tap / 3, xx = x0 + (tap - (tap / 3) * 3);
              float v = 0.f;
              if (vrow && k < 63 && yy >= 0 && yy < a.Hin && xx >= 0 && xx < a.Win) {
                v = __ldg(xin + (size_t)c * hw_in + yy * a.Win + xx);
                if (a.encode && c < 3) v = log1pf(a.exposure * v);
              }
              vals[qq][e] = v;
            }
          }
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, tmo, a.status, ERR_TIMEOUT)) {
            ok = false;
            break;
          }
          uint8_t *a0 = data + stage * sbytes;
          uint8_t *a1 = a0 + a_bytes;
#pragma unroll
          for (int qq = 0; qq < KROW_BYTES / 16 / 2; ++qq)
            store_nchw7<PREC>(a0, a1, swz(r, qbase + qq), vals[qq], qscale);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&full_bar[stage]));
          if (++stage == stages) {
            stage = 0;
            phase ^= 1;
          }
        }
      } else {
        // NHWC gather: 8 lanes cover one 128-byte operand row, 4 rows per warp,
        // 4 passes of 32 rows
        const int q = lane & 7;
        int pix_base[4], ybase[4], xbase[4];
        bool vrow[4];
#pragma unroll
        for (int it = 0; it < 4; ++it) {
          const int r = (lane >> 3) + 4 * pw + 32 * it;
          const int m = tc.m_tile * BM + r;
          vrow[it] = m < a.M;
          const int n = vrow[it] ? m / rows_per_map : 0;
          const int rem = vrow[it] ? m - n * rows_per_map : 0;
          const int i = rem / a.Wrow, j = rem - (rem / a.Wrow) * a.Wrow;
          pix_base[it] = n * hw_in;
          ybase[it] = a.kind == LK_CONV ? 2 * i - 1 : i;
          xbase[it] = a.kind == LK_CONV ? 2 * j - 1 : j;
        }
        const uint8_t *xin = reinterpret_cast<const uint8_t *>(a.x);
        const int ntaps = pd.ntaps;
        for (int kb = 0; kb < nkb; ++kb) {
          const int k0 = kb * BKE + q * E;
          const int tap = k0 / a.Cin;
          const int c = k0 - tap * a.Cin;
          const bool vtap = tap < ntaps;
          const int dy = vtap ? pd.dy[tap] : 0, dx = vtap ? pd.dx[tap] : 0;
          Chunk<PREC> ch[4];
#pragma unroll
          for (int it = 0; it < 4; ++it) {
            const int yy = ybase[it] + dy, xx = xbase[it] + dx;
            const bool okp = vrow[it] && vtap && yy >= 0 && yy < a.Hin && xx >= 0 && xx < a.Win;
            const size_t eoff = ((size_t)(pix_base[it] + (okp ? yy * a.Win + xx : 0)) * a.Cin + c);
            load_chunk_nhwc<PREC>(ch[it], xin + eoff * sizeof(typename T::act_t), okp);
          }
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1, tmo, a.status, ERR_TIMEOUT)) {
            ok = false;
            break;
          }
          uint8_t *a0 = data + stage * sbytes;
          uint8_t *a1 = a0 + a_bytes;
#pragma unroll
          for (int it = 0; it < 4; ++it) {
            const int r = (lane >> 3) + 4 * pw + 32 * it;
            store_chunk<PREC>(a0, a1, swz(r, q), ch[it], qscale);
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&full_bar[stage]));
          if (++stage == stages) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
    }
  } else if (warp >= EPI_WARP0 && warp < EPI_WARP0 + 4) {
    // ------------------------------------------------------------ epilogue
    const int eq = warp - EPI_WARP0;  // TMEM lane quarter
    const int row = eq * 32 + lane;
    const int rows_per_map = a.Hrow * a.Wrow;
    int it = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++it) {
      const TileCoord tc = tile_coord(a, t);
      const PhaseDesc &pd = a.ph[tc.phase];
      const int buf = nbufs == 2 ? (it & 1) : 0;
      const uint32_t par = (uint32_t)((nbufs == 2 ? (it >> 1) : it) & 1);
      if (!mbar_wait(smem_u32(&tfull_bar[buf]), par, tmo, a.status, ERR_TIMEOUT)) break;
      tc_fence_after();
      const int m = tc.m_tile * BM + row;
      const bool vrow = m < a.M;
      const int n = vrow ? m / rows_per_map : 0;
      const int rem = vrow ? m - n * rows_per_map : 0;
      const int i = rem / a.Wrow, j = rem - (rem / a.Wrow) * a.Wrow;
      const uint32_t taddr = tmem_base + ((uint32_t)(eq * 32) << 16) + (uint32_t)(buf * acc_cols);
      if (a.kind == LK_HEAD) {
        float v[16];
        tmem_ld_acc<PREC>(taddr, BN, v);
        float pay[3] = {0.f, 0.f, 0.f};
        float *out = reinterpret_cast<float *>(a.y);
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          const int orow = 2 * i + pp;
          const float band = vrow ? a.band[orow] : 0.f;
#pragma unroll
          for (int o = 0; o < 3; ++o) {
            float y0 = v[pp * 6 + o] + a.bias[o];
            float y1 = v[pp * 6 + 3 + o] + a.bias[o];
            if (a.relu) {
              y0 = fmaxf(y0, 0.f);
              y1 = fmaxf(y1, 0.f);
            }
            const float l0 = expm1f(y0) * a.inv_exposure;
            const float l1 = expm1f(y1) * a.inv_exposure;
            pay[o] += (l0 + l1) * band;
            if (vrow) {
              float2 w = a.decode ? make_float2(l0, l1) : make_float2(y0, y1);
              *reinterpret_cast<float2 *>(out + (((size_t)n * 3 + o) * a.Hout + orow) * a.Wout + 2 * j) = w;
            }
          }
        }
        if (a.payload) {
          const int n0 = __shfl_sync(0xffffffffu, n, 0);
          const bool uniform = __all_sync(0xffffffffu, vrow && n == n0);
          if (uniform) {
#pragma unroll
            for (int o = 0; o < 3; ++o) {
              float s = pay[o];
#pragma unroll
              for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
              pay[o] = s;
            }
            if (lane == 0)
              for (int o = 0; o < 3; ++o) atomicAdd(a.payload + (size_t)n0 * 3 + o, pay[o]);
          } else if (vrow) {
            for (int o = 0; o < 3; ++o) atomicAdd(a.payload + (size_t)n * 3 + o, pay[o]);
          }
        }
      } else {
        size_t opix;
        if (a.kind == LK_CONVT)
          opix = ((size_t)n * a.Hout + (2 * i + pd.oy)) * a.Wout + (2 * j + pd.ox);
        else
          opix = (size_t)m;
        using act_t = typename T::act_t;
        act_t *yout = reinterpret_cast<act_t *>(a.y);
        const act_t *skip = reinterpret_cast<const act_t *>(a.skip);
        for (int cc = 0; cc < BN / 16; ++cc) {
          float v[16];
          tmem_ld_acc<PREC>(taddr + cc * 16, BN, v);
          const int col0 = tc.n_tile * BN + cc * 16;
          if (!vrow) continue;
          const float *bsc = a.bscale ? a.bscale + col0 : nullptr;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            float z = bsc ? v[e] * bsc[e] : v[e];
            z += a.bias[col0 + e];
            if (a.relu) z = fmaxf(z, 0.f);
            v[e] = z;
          }
          const size_t eoff = opix * a.Cout + col0;
          if constexpr (PREC == PREC_TF32X3) {
            if (skip) {
              const float4 *sp = reinterpret_cast<const float4 *>(skip + eoff);
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                float4 s = sp[e];
                v[4 * e] += s.x;
                v[4 * e + 1] += s.y;
                v[4 * e + 2] += s.z;
                v[4 * e + 3] += s.w;
              }
            }
            float4 *yp = reinterpret_cast<float4 *>(yout + eoff);
#pragma unroll
            for (int e = 0; e < 4; ++e) yp[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
          } else {
            if (skip) {
              const uint4 *sp = reinterpret_cast<const uint4 *>(skip + eoff);
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                uint4 s = sp[e];
                v[8 * e + 0] += bf16_lo(s.x);
                v[8 * e + 1] += bf16_hi(s.x);
                v[8 * e + 2] += bf16_lo(s.y);
                v[8 * e + 3] += bf16_hi(s.y);
                v[8 * e + 4] += bf16_lo(s.z);
                v[8 * e + 5] += bf16_hi(s.z);
                v[8 * e + 6] += bf16_lo(s.w);
                v[8 * e + 7] += bf16_hi(s.w);
              }
            }
            uint4 *yp = reinterpret_cast<uint4 *>(yout + eoff);
#pragma unroll
            for (int e = 0; e < 2; ++e)
              yp[e] = make_uint4(pack_bf16x2(v[8 * e], v[8 * e + 1]), pack_bf16x2(v[8 * e + 2], v[8 * e + 3]),
                                 pack_bf16x2(v[8 * e + 4], v[8 * e + 5]), pack_bf16x2(v[8 * e + 6], v[8 * e + 7]));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[buf]));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem_base, ncols);
  }
}

cudaError_t launch_conv(const ConvArgs &a, int prec, int num_sms, cudaStream_t st) {
  const int total = a.num_phases * a.m_tiles * a.n_tiles;
  if (total == 0) return cudaSuccess;
  const int grid = total < num_sms ? total : num_sms;
  const size_t smem = conv_smem_bytes(prec, a.BN);
  cudaError_t e;
  switch (prec) {
    case PREC_TF32X3:
      e = cudaFuncSetAttribute(conv_tc_kernel<PREC_TF32X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      conv_tc_kernel<PREC_TF32X3><<<grid, NUM_THREADS, smem, st>>>(a);
      break;
    case PREC_BF16:
      e = cudaFuncSetAttribute(conv_tc_kernel<PREC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      conv_tc_kernel<PREC_BF16><<<grid, NUM_THREADS, smem, st>>>(a);
      break;
    default:
      e = cudaFuncSetAttribute(conv_tc_kernel<PREC_FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      conv_tc_kernel<PREC_FP8><<<grid, NUM_THREADS, smem, st>>>(a);
      break;
  }
  return cudaGetLastError();
}

// --------------------------------------------------------- weight packing
// One thread per 16-byte chunk of the packed B image: chunk (phase, n_tile,
// kb, row r, physical chunk p) holds logical chunk q = p ^ (r & 7) of row r,
// i.e. K elements kb*BKE + q*E .. + E - 1 of output column n_tile*BN + r.
__device__ float raw_weight(const PackArgs &p, const PhaseDesc &pd, int col, int k) {
  switch (p.kind) {
    case LK_CONV_NCHW7:
      return k < 63 ? p.wraw[(size_t)col * 63 + k] : 0.f;
    case LK_CONV: {
      const int tap = k / p.Cin, c = k - (k / p.Cin) * p.Cin;
      return tap < 9 ? p.wraw[((size_t)col * p.Cin + c) * 9 + tap] : 0.f;
    }
    case LK_CONVT: {
      const int t = k / p.Cin, c = k - (k / p.Cin) * p.Cin;
      if (t >= pd.ntaps) return 0.f;
      return p.wraw[(((size_t)c * p.Cout + col) * 3 + pd.u[t]) * 3 + pd.v[t]];
    }
    default: {  // LK_HEAD: column = pp*6 + qq*3 + o, K = neighbour*Cin + c
      if (col >= 12) return 0.f;
      const int pp = col / 6, qq = (col / 3) & 1, o = col % 3;
      const int nb = k / p.Cin, c = k - (k / p.Cin) * p.Cin;
      if (nb >= 4) return 0.f;
      const int di = nb >> 1, dj = nb & 1;
      // output row 2a+pp receives input row a+di through kernel row u with
      // 2(a+di) + u - 1 = 2a + pp, i.e. u = pp + 1 - 2 di (valid 0..2)
      const int u = pp + 1 - 2 * di, v = qq + 1 - 2 * dj;
      if (u < 0 || u > 2 || v < 0 || v > 2) return 0.f;
      return p.wraw[(((size_t)c * 3 + o) * 3 + u) * 3 + v];
    }
  }
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
    float4 h, l;
    h = make_float4(to_tf32(w[0]), to_tf32(w[1]), to_tf32(w[2]), to_tf32(w[3]));
    l = make_float4(to_tf32(w[0] - h.x), to_tf32(w[1] - h.y), to_tf32(w[2] - h.z), to_tf32(w[3] - h.w));
    *reinterpret_cast<float4 *>(p.B + off) = h;
    *reinterpret_cast<float4 *>(p.B_lo + off) = l;
  } else if constexpr (PREC == PREC_BF16) {
    uint4 o;
    o.x = pack_bf16x2(w[0], w[1]);
    o.y = pack_bf16x2(w[2], w[3]);
    o.z = pack_bf16x2(w[4], w[5]);
    o.w = pack_bf16x2(w[6], w[7]);
    *reinterpret_cast<uint4 *>(p.B + off) = o;
  } else {
    // per-column scale: the pack of the column's scale happens on the host
    // side of the planner (bscale), values are divided by it here
    const float inv = 1.0f / p.bscale[col];
    uint4 o;
    o.x = pack_e4m3x4(w[0] * inv, w[1] * inv, w[2] * inv, w[3] * inv);
    o.y = pack_e4m3x4(w[4] * inv, w[5] * inv, w[6] * inv, w[7] * inv);
    o.z = pack_e4m3x4(w[8] * inv, w[9] * inv, w[10] * inv, w[11] * inv);
    o.w = pack_e4m3x4(w[12] * inv, w[13] * inv, w[14] * inv, w[15] * inv);
    *reinterpret_cast<uint4 *>(p.B + off) = o;
  }
}

cudaError_t launch_pack(const PackArgs &p, int prec, cudaStream_t st) {
  if (p.total_chunks == 0) return cudaSuccess;
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
