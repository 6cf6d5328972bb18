// wgrad_tc.cu -- weight gradient of a 3x3 stride-2 conv / transposed conv on
// the tensor cores (BF16 operands, fp32 accumulation), the training pass of
// Sec. 3.3 with the L1 loss of Eq. 7:
//   dW[m][q][u][v] += sum_{n,i,j} R[n,i,j,m] * Q[n, 2i+u-1, 2j+v-1, q]
// (R at the coarse resolution, Q at twice it; see backward.cu for which
// tensors they are).  For each tap (u, v) this is a GEMM D[m][q] = sum_k
// A[m][k] B[q][k] with K = pixels.  Both operands come straight from NHWC
// tensors, channels contiguous, so they are MN-major: a TMA box of 64
// channels (128 bytes) x 64 pixels lands in shared memory as eight
// 128-byte-swizzled atoms of 64 MN elements x 8 K rows, which the MMA reads
// with LBO = distance between MN atoms and SBO = distance between 8-row K
// groups (1024 bytes).  A = R (2-D map over [pixels][channels]); B = the
// tap's stride-2 box of Q (4-D map [C][W][H][N], element strides 1,2,2,1,
// the padding from the TMA's zero fill), exactly the encoder convolution's A
// box.  One CTA = one (tap, m tile, q tile) and a range of 64-pixel K
// blocks; its fp32 tile is added to dW with atomics (split K).
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
constexpr int WT_KB = 64;          // pixels per K block
constexpr int WT_BOX = 64 * 64 * 2;  // bytes of one 64-channel x 64-pixel bf16 box
constexpr int WT_STAGES = 6;

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

__global__ void __launch_bounds__(WT_THREADS, 1) wgrad_tc_kernel(const __grid_constant__ WgradTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[WT_STAGES], empty_bar[WT_STAGES], done_bar;
  __shared__ uint32_t tmem_slot;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int qboxes = a.BNq / 64;
  const uint32_t a_bytes = 2 * WT_BOX, b_bytes = (uint32_t)qboxes * WT_BOX, sbytes = a_bytes + b_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this CTA's tile and K range
  const int tiles = 9 * a.m_tiles * a.n_tiles;
  // the tiles of one K range are neighbours, so its R and Q blocks are
  // fetched from DRAM once and re-read from L2 by the other taps
  const int split = blockIdx.x / tiles, tile = blockIdx.x - split * tiles;
  if (split >= a.ksplit) return;
  const int tap = tile % 9, mt = (tile / 9) % a.m_tiles, nt = tile / (9 * a.m_tiles);
  const int kb0 = split * a.kb_per_split;
  const int kb1 = min(kb0 + a.kb_per_split, a.total_kb);
  const int nkb = kb1 - kb0;
  if (nkb <= 0) return;  // block-uniform
  const uint32_t ncols = a.BNq <= 64 ? 64u : 128u;
  if (warp == 2) {
    tmem_alloc(smem_u32(&tmem_slot), ncols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < WT_STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&done_bar), 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const unsigned long long tmo = a.timeout_ns;
  const int u = tap / 3, v = tap % 3;
  const int m0 = mt * 128, q0 = nt * a.BNq;
  const int hw = a.Hb * a.Wb;

  if (warp == 0 && lane == 0) {
    // TMA: per K block two boxes of R (channels m0 .. m0 + 127) and the tap's
    // box(es) of Q
    int issued = 0;
    for (int j = 0; j < nkb; ++j) {
      const int s = j % WT_STAGES;
      if (!mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((j / WT_STAGES) & 1) ^ 1), tmo, a.status, ERR_TIMEOUT))
        break;
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_arrive_expect_tx(fb, sbytes);
      const uint32_t dst = base + (uint32_t)s * sbytes;
      const int p0 = (kb0 + j) * WT_KB;  // first pixel
      tma_load_2d(dst, &a.mapR, m0, p0, fb);
      tma_load_2d(dst + WT_BOX, &a.mapR, m0 + 64, p0, fb);
      const int n0 = p0 / hw, r0 = (p0 - n0 * hw) / a.Wb;
      for (int h = 0; h < qboxes; ++h)
        tma_load_4d(dst + a_bytes + (uint32_t)h * WT_BOX, &a.mapQ, q0 + 64 * h, v - 1, 2 * r0 + u - 1, n0, fb);
      issued = j + 1;
    }
    // leave no copy in flight, whatever the MMA thread did (bounded waits)
    for (int j = issued > WT_STAGES ? issued - WT_STAGES : 0; j < issued; ++j)
      if (!mbar_wait(smem_u32(&full_bar[j % WT_STAGES]), (uint32_t)((j / WT_STAGES) & 1), tmo, a.status,
                     ERR_TIMEOUT))
        break;
  } else if (warp == 1 && lane == 0) {
    // MMA: D[128][BNq] += A[128][64] B[BNq][64]^T per K block, 16 pixels per MMA
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                           ((uint32_t)(a.BNq >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    bool ok = true;
    for (int j = 0; j < nkb && ok; ++j) {
      const int s = j % WT_STAGES;
      if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((j / WT_STAGES) & 1), tmo, a.status, ERR_TIMEOUT)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = base + (uint32_t)s * sbytes, sb = sa + a_bytes;
#pragma unroll
      for (int k = 0; k < WT_KB / 16; ++k)  // 16 pixels = two 8-row K groups = 2048 bytes
        tc_mma<KIND_F16>(tmem, sdesc_mn(sa + 2048u * k, WT_BOX), sdesc_mn(sb + 2048u * k, WT_BOX), idesc,
                         (j | k) != 0);
      tc_commit(smem_u32(&empty_bar[s]));
    }
    tc_commit(smem_u32(&done_bar));
  } else if (warp >= 4) {
    // epilogue: lane quarter eq holds rows m0 + 32 eq + lane
    const int eq = warp - 4, row = 32 * eq + lane, m = m0 + row;
    const bool ok = mbar_wait(smem_u32(&done_bar), 0u, tmo, a.status, ERR_TIMEOUT);
    tc_fence_after();
    if (ok) {
      for (int c0 = 0; c0 < a.BNq; c0 += 16) {
        float d[16];
        tmem_ld16(tmem + ((uint32_t)(32 * eq) << 16) + (uint32_t)c0, d);
        if (m < a.Mr) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int q = q0 + c0 + e;
            if (q < a.Qraw && d[e] != 0.f) atomicAdd(a.dW + ((size_t)m * a.Qraw + q) * 9 + tap, d[e]);
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

bool wgrad_tc_supported(int Hb, int Wb, int Mr, int Qc) {
  if (Qc < 64 || Qc % 64 || Mr < 128 || Mr % 128 || Hb < 1 || Wb < 1) return false;
  if (Wb > WT_KB || WT_KB % Wb) return false;  // a K block = whole rows ...
  int rows, maps;
  wgrad_tc_box(Hb, Wb, &rows, &maps);
  if (rows < Hb) return Hb % rows == 0;  // ... of one map
  return WT_KB % (Hb * Wb) == 0;         // ... or whole maps
}

cudaError_t launch_wgrad_tc(const WgradTcArgs &in, int num_sms, cudaStream_t st) {
  WgradTcArgs a = in;
  const long long K = (long long)a.N * a.Hb * a.Wb;
  if (K == 0) return cudaSuccess;
  a.total_kb = (int)((K + WT_KB - 1) / WT_KB);
  const int tiles = 9 * a.m_tiles * a.n_tiles;
  // one CTA per SM (the stages take most of shared memory), one wave
  int ksplit = num_sms / tiles;
  if (ksplit > a.total_kb) ksplit = a.total_kb;
  if (ksplit < 1) ksplit = 1;
  a.kb_per_split = (a.total_kb + ksplit - 1) / ksplit;
  a.ksplit = (a.total_kb + a.kb_per_split - 1) / a.kb_per_split;
  const size_t smem = 1024 + (size_t)WT_STAGES * (2 * WT_BOX + (size_t)(a.BNq / 64) * WT_BOX);
  cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  wgrad_tc_kernel<<<(unsigned)(tiles * a.ksplit), WT_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace drc
