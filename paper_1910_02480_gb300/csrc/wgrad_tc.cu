// wgrad_tc.cu -- weight gradient of a 3x3 stride-2 conv / transposed conv on
// the tensor cores (BF16 operands, fp32 accumulation), the training pass of
// Sec. 3.3 with the L1 loss of Eq. 7:
//   dW[m][q][u][v] += sum_{n,i,j} R[n,i,j,m] * Q[n, 2i+u-1, 2j+v-1, q]
// (R at the coarse resolution, Q at twice it; see backward.cu for which
// tensors they are).  K = pixels.  Both operands come straight from NHWC
// tensors, channels contiguous, so they are MN-major in shared memory.
//
// Wide form (Qc a multiple of 64): one GEMM per tap (u, v),
// D[m][q] = sum_k R[k][m] Q_uv[k][q].  A TMA box of 64 channels (128 bytes)
// x 64 pixels lands as eight 128-byte-swizzled atoms of 64 MN elements x 8 K
// rows, which the MMA reads with LBO = distance between MN atoms and SBO =
// distance between 8-row K groups (1024 bytes).  A = R (2-D map over
// [pixels][channels]), two boxes for M = 128; B = the tap's stride-2 box of
// Q (4-D map [C][W][H][N], element strides 1,2,2,1, the padding from the
// TMA's zero fill), the encoder convolution's A box.
//
// Narrow form (Qc = 8, the network input and the head's output gradient):
// all nine taps in one GEMM, D[8 tap + q][m] = sum_k Q_tap[k][q] R[k][m].
// A = the nine taps' boxes of 8 channels x 64 pixels (16 bytes x 64, no
// swizzle), placed 1024 bytes apart: in the no-swizzle MN-major layout a
// core matrix is 8 K rows x 16 bytes, here LBO = K-group stride (128 bytes)
// and SBO = MN-group stride (1024 bytes); rows 72..127 stay zero.  B = R in
// 64-channel swizzled boxes, N = up to 256 of its channels.
//
// One CTA = one tile and a range of 64-pixel K blocks; its fp32 tile is
// added to dW with atomics (split K).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "drc_status.cuh"
#include "ptx.cuh"
#include "wgrad_tc.cuh"

namespace drc {

namespace {

constexpr int WT_THREADS = 256;
constexpr int WT_KB = 64;               // pixels per K block
constexpr int WT_BOX = 64 * 64 * 2;     // bytes of one 64-channel x 64-pixel bf16 box
constexpr int WT_NARROW_A = 16 * 1024;  // narrow A: 16 MN groups of 8 rows x 64 pixels
constexpr int WT_MAX_STAGES = 6;
constexpr int WT_SMEM_BUDGET = 200 * 1024;

// MN-major, 128-byte swizzle: LBO = distance between 64-element MN atoms,
// SBO = distance between 8-row K groups.
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t mn_atom_bytes) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((mn_atom_bytes >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// MN-major, no swizzle, core matrices of 8 K rows x 16 bytes: LBO = distance
// between K groups, SBO = distance between 8-element MN groups.
__device__ __forceinline__ uint64_t sdesc_mn_plain(uint32_t saddr, uint32_t kgroup_bytes, uint32_t mngroup_bytes) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((kgroup_bytes >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((mngroup_bytes >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__host__ __device__ __forceinline__ uint32_t stage_bytes(bool narrow, int BN) {
  return narrow ? (uint32_t)WT_NARROW_A + (uint32_t)(BN / 64) * WT_BOX : 2u * WT_BOX + (uint32_t)(BN / 64) * WT_BOX;
}
__host__ __device__ __forceinline__ int num_stages(bool narrow, int BN) {
  const int s = WT_SMEM_BUDGET / (int)stage_bytes(narrow, BN);
  return s < WT_MAX_STAGES ? s : WT_MAX_STAGES;
}

template <bool NARROW>
__global__ void __launch_bounds__(WT_THREADS, 1) wgrad_tc_kernel(const __grid_constant__ WgradTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[WT_MAX_STAGES], empty_bar[WT_MAX_STAGES], done_bar;
  __shared__ uint32_t tmem_slot;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int nboxes = a.BN / 64;  // B boxes (wide: of Q; narrow: of R)
  const uint32_t a_bytes = NARROW ? (uint32_t)WT_NARROW_A : 2u * WT_BOX;
  const uint32_t sbytes = stage_bytes(NARROW, a.BN);
  const uint32_t load_bytes = NARROW ? 9u * 1024u + (uint32_t)nboxes * WT_BOX : sbytes;
  const int stages = num_stages(NARROW, a.BN);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this CTA's tile and K range; the tiles of one K range are neighbours, so
  // its R and Q blocks are fetched from DRAM once and re-read from L2
  const int tiles = (NARROW ? 1 : 9) * a.m_tiles * a.n_tiles;
  const int split = blockIdx.x / tiles, tile = blockIdx.x - split * tiles;
  if (split >= a.ksplit) return;
  const int tap = NARROW ? 0 : tile % 9;
  const int mt = NARROW ? 0 : (tile / 9) % a.m_tiles;
  const int nt = NARROW ? tile : tile / (9 * a.m_tiles);
  const int kb0 = split * a.kb_per_split;
  const int kb1 = min(kb0 + a.kb_per_split, a.total_kb);
  const int nkb = kb1 - kb0;
  if (nkb <= 0) return;  // block-uniform
  const uint32_t ncols = a.BN <= 64 ? 64u : (a.BN <= 128 ? 128u : 256u);
  if (warp == 2) {
    tmem_alloc(smem_u32(&tmem_slot), ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    fence_mbar_init();
  }
  if (NARROW) {  // the A rows 72..127 of every stage are zero for good
    uint8_t *sm = smem_raw + (base - smem_u32(smem_raw));
    for (int s = 0; s < stages; ++s)
      for (int i = threadIdx.x; i < (WT_NARROW_A - 9 * 1024) / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(sm + (size_t)s * sbytes + 9 * 1024)[i] = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const unsigned long long tmo = a.timeout_ns;
  const int m0 = mt * 128, n0c = nt * a.BN;  // first R channel (wide) / first B column
  const int hw = a.Hb * a.Wb;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int j = 0; j < nkb; ++j) {
      const int s = j % stages;
      if (!mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((j / stages) & 1) ^ 1), tmo, a.status, ERR_TIMEOUT))
        break;
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_arrive_expect_tx(fb, load_bytes);
      const uint32_t dst = base + (uint32_t)s * sbytes;
      const int p0 = (kb0 + j) * WT_KB;  // first pixel
      const int n0 = p0 / hw, r0 = (p0 - n0 * hw) / a.Wb;
      if (NARROW) {
        // A: the nine taps' 8-channel boxes of Q; B: R channels n0c ..
        for (int t = 0; t < 9; ++t) tma_load_4d(dst + 1024u * t, &a.mapQ, 0, t % 3 - 1, 2 * r0 + t / 3 - 1, n0, fb);
        for (int h = 0; h < nboxes; ++h)
          tma_load_2d(dst + a_bytes + (uint32_t)h * WT_BOX, &a.mapR, n0c + 64 * h, p0, fb);
      } else {
        // A: two boxes of R (channels m0 .. m0 + 127); B: the tap's box(es) of Q
        const int u = tap / 3, v = tap % 3;
        tma_load_2d(dst, &a.mapR, m0, p0, fb);
        tma_load_2d(dst + WT_BOX, &a.mapR, m0 + 64, p0, fb);
        for (int h = 0; h < nboxes; ++h)
          tma_load_4d(dst + a_bytes + (uint32_t)h * WT_BOX, &a.mapQ, n0c + 64 * h, v - 1, 2 * r0 + u - 1, n0, fb);
      }
      issued = j + 1;
    }
    // leave no copy in flight, whatever the MMA thread did (bounded waits)
    for (int j = issued > stages ? issued - stages : 0; j < issued; ++j)
      if (!mbar_wait(smem_u32(&full_bar[j % stages]), (uint32_t)((j / stages) & 1), tmo, a.status, ERR_TIMEOUT))
        break;
  } else if (warp == 1 && lane == 0) {
    // D[128][BN] += A[128][64] B[BN][64]^T per K block, 16 pixels per MMA
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                           ((uint32_t)(a.BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    for (int j = 0; j < nkb; ++j) {
      const int s = j % stages;
      if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((j / stages) & 1), tmo, a.status, ERR_TIMEOUT)) break;
      tc_fence_after();
      const uint32_t sa = base + (uint32_t)s * sbytes, sb = sa + a_bytes;
#pragma unroll
      for (int k = 0; k < WT_KB / 16; ++k) {  // 16 pixels = two 8-row K groups
        const uint64_t da = NARROW ? sdesc_mn_plain(sa + 256u * k, 128u, 1024u) : sdesc_mn(sa + 2048u * k, WT_BOX);
        tc_mma<KIND_F16>(tmem, da, sdesc_mn(sb + 2048u * k, WT_BOX), idesc, (j | k) != 0);
      }
      tc_commit(smem_u32(&empty_bar[s]));
    }
    tc_commit(smem_u32(&done_bar));
  } else if (warp >= 4) {
    // epilogue: lane quarter eq holds D rows 32 eq + lane
    const int eq = warp - 4, row = 32 * eq + lane;
    const bool ok = mbar_wait(smem_u32(&done_bar), 0u, tmo, a.status, ERR_TIMEOUT);
    tc_fence_after();
    if (ok) {
      for (int c0 = 0; c0 < a.BN; c0 += 16) {
        float d[16];
        tmem_ld16(tmem + ((uint32_t)(32 * eq) << 16) + (uint32_t)c0, d);
        if (NARROW) {  // row = 8 tap + q, column = R channel m
          const int t = row >> 3, q = row & 7;
          if (t < 9 && q < a.Qraw) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int m = n0c + c0 + e;
              if (m < a.Mr && d[e] != 0.f) atomicAdd(a.dW + ((size_t)m * a.Qraw + q) * 9 + t, d[e]);
            }
          }
        } else {  // row = R channel m, column = Q channel q
          const int m = m0 + row;
          if (m < a.Mr) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int q = n0c + c0 + e;
              if (q < a.Qraw && d[e] != 0.f) atomicAdd(a.dW + ((size_t)m * a.Qraw + q) * 9 + tap, d[e]);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}

}  // namespace

void wgrad_tc_box(int Hb, int Wb, int *rows, int *maps) {
  *rows = Hb < WT_KB / Wb ? Hb : WT_KB / Wb;
  *maps = *rows < Hb ? 1 : WT_KB / (Hb * Wb);
}

int wgrad_tc_form(int Hb, int Wb, int Mr, int Qc) {
  if (Hb < 1 || Wb < 1 || Wb > WT_KB || WT_KB % Wb) return WGRAD_TC_NONE;  // a K block = whole rows ...
  int rows, maps;
  wgrad_tc_box(Hb, Wb, &rows, &maps);
  if (rows < Hb ? Hb % rows != 0 : WT_KB % (Hb * Wb) != 0) return WGRAD_TC_NONE;  // ... of whole maps
  if (Qc >= 64 && Qc % 64 == 0 && Mr >= 128 && Mr % 128 == 0) return WGRAD_TC_WIDE;
  if (Qc == 8 && Mr >= 64 && Mr % 64 == 0) return WGRAD_TC_NARROW;
  return WGRAD_TC_NONE;
}

cudaError_t launch_wgrad_tc(const WgradTcArgs &in, int form, int num_sms, cudaStream_t st) {
  WgradTcArgs a = in;
  const long long K = (long long)a.N * a.Hb * a.Wb;
  if (K == 0) return cudaSuccess;
  const bool narrow = form == WGRAD_TC_NARROW;
  if (a.BN < 64 || a.BN > (narrow ? 256 : 128) || a.BN % 64) return cudaErrorInvalidValue;
  a.total_kb = (int)((K + WT_KB - 1) / WT_KB);
  const int tiles = (narrow ? 1 : 9) * a.m_tiles * a.n_tiles;
  // one CTA per SM (the stages take most of shared memory), one wave
  int ksplit = num_sms / tiles;
  if (ksplit > a.total_kb) ksplit = a.total_kb;
  if (ksplit < 1) ksplit = 1;
  a.kb_per_split = (a.total_kb + ksplit - 1) / ksplit;
  a.ksplit = (a.total_kb + a.kb_per_split - 1) / a.kb_per_split;
  const size_t smem = 1024 + (size_t)num_stages(narrow, a.BN) * stage_bytes(narrow, a.BN);
  cudaError_t e;
  if (narrow) {
    e = cudaFuncSetAttribute(wgrad_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    wgrad_tc_kernel<true><<<(unsigned)(tiles * a.ksplit), WT_THREADS, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(wgrad_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    wgrad_tc_kernel<false><<<(unsigned)(tiles * a.ksplit), WT_THREADS, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace drc
