// head.cu -- the output layer of the autoencoder (Sec. 3.3): a 3x3 transposed
// convolution, stride 2, from the first decoder activation t_1 (C channels,
// H/2 x W/2, NHWC) to the 3 radiance channels (H x W, NCHW), with the
// optional final ReLU and log decode, and the per-map irradiance payload
// E/pi (Eq. 2 with a white Lambertian BRDF).
//
// With 3 output channels a tensor-core tile would be 3/16 useful, so this
// layer is plain fp32 FMA (exact fp32 rounding, no split needed), in two
// steps per CTA.  A CTA covers a 16 x 16 block of t_1 pixels of one map plus
// the row and column below / right of it (17 x 17, one thread per pixel):
//   1. D[p][r] = sum_c x[p][c] W[c][r] for the 27 r = (o, u, v): the input is
//      read once (4 channels per vector load).  For C <= 64 (CI > 0) the
//      weights come with the launch parameters and, the channel loop being
//      unrolled, every FMA reads its weight as a constant-bank operand (no
//      load instruction); wider layers stage the weights in shared memory
//      (7 float4 broadcasts per channel);
//   2. every output pixel of the block's 32 x 32 sums the 1, 2 or 4 entries of
//      D that reach it (output row 2a + p gathers t_1 row a + d through tap u
//      with 2(a + d) + u - 1 = 2a + p), adds the bias, and is written as
//      coalesced rows of the NCHW planes with the decode and the payload.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstdint>
#include <cuda_runtime.h>

#include "head.cuh"

namespace drc {

constexpr int HT = 16;          // t_1 block edge per CTA
constexpr int HE = HT + 1;       // with the halo row / column
constexpr int HPIX = HE * HE;    // pixels of D per CTA
constexpr int HTHREADS = 320;    // >= HPIX, whole warps
constexpr int HCC = 128;         // input channels per staged weight chunk
// Four consecutive channels (16-byte fp32 / 8-byte bf16 aligned: C and the
// channel offset are multiples of 4).
template <typename ActT>
__device__ __forceinline__ float4 load_act4(const ActT *p, const float *scale);
template <>
__device__ __forceinline__ float4 load_act4<float>(const float *p, const float *) {
  return __ldg(reinterpret_cast<const float4 *>(p));
}
template <>
__device__ __forceinline__ float4 load_act4<__nv_bfloat16>(const __nv_bfloat16 *p, const float *) {
  const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                     __uint_as_float(u.y & 0xffff0000u));
}
// e4m3 (4-byte aligned: C and the channel offset are multiples of 4), times
// the channels' scales.
template <>
__device__ __forceinline__ float4 load_act4<uint8_t>(const uint8_t *p, const float *scale) {
  const uint32_t w = __ldg(reinterpret_cast<const unsigned int *>(p));
  const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xFFFFu), __NV_E4M3);
  const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
  const float4 s = __ldg(reinterpret_cast<const float4 *>(scale));
  return make_float4(a.x * s.x, a.y * s.y, b.x * s.z, b.y * s.w);
}

template <typename ActT, int CI>
__global__ void __launch_bounds__(HTHREADS, 2) head_kernel(const __grid_constant__ HeadArgs a) {
  __shared__ float4 ws[HCC * 7];  // W[c][r] of one channel chunk, r = 9 o + 3 u + v (27 used of 28)
  __shared__ float ds[27 * HPIX];  // D[r][pixel]
  __shared__ float red[3][HTHREADS / 32];
  const int tiles_x = (a.Wh + HT - 1) / HT, tiles_y = (a.Hh + HT - 1) / HT;
  const int tile = blockIdx.x % (tiles_x * tiles_y);
  const int n = blockIdx.x / (tiles_x * tiles_y);
  float *out = a.out, *payload = a.payload;
  int decode = a.decode;
  if (a.slot) {  // block-uniform: the whole block leaves before any barrier
    if (n >= a.slot->count) return;
    out = a.slot->out;
    payload = a.slot->payload;
    decode = (a.slot->flags & SLOT_DECODE) ? 1 : 0;
  }
  const int a0 = (tile / tiles_x) * HT, b0 = (tile % tiles_x) * HT;
  const int tid = threadIdx.x;
  // step 1: D for this thread's pixel (zero outside the map)
  const int pi = tid / HE, pj = tid - (tid / HE) * HE;
  const bool vpix = tid < HPIX && a0 + pi < a.Hh && b0 + pj < a.Wh;
  const ActT *xp = reinterpret_cast<const ActT *>(a.x) +
                   (((size_t)n * a.Hh + (vpix ? a0 + pi : 0)) * a.Wh + (vpix ? b0 + pj : 0)) * a.C;
  float acc[27];
#pragma unroll
  for (int r = 0; r < 27; ++r) acc[r] = 0.f;
  if constexpr (CI > 0) {
    if (vpix) {
#pragma unroll
      for (int c = 0; c < CI; c += 4) {
        const float4 x4 = load_act4<ActT>(xp + c, a.in_scale ? a.in_scale + c : nullptr);
        const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int r = 0; r < 27; ++r) acc[r] = fmaf(xv[e], a.wk[(c + e) * 27 + r], acc[r]);
      }
    }
  }
  for (int c0 = 0; CI == 0 && c0 < a.C; c0 += HCC) {
    const int cn = min(HCC, a.C - c0);
    __syncthreads();
    for (int e = tid; e < cn * 7; e += HTHREADS) {
      const int c = e / 7, q = e - c * 7;
      const float *wc = a.w + (size_t)(c0 + c) * 27 + 4 * q;
      ws[e] = make_float4(__ldg(wc), __ldg(wc + 1), __ldg(wc + 2), q < 6 ? __ldg(wc + 3) : 0.f);
    }
    __syncthreads();
    if (vpix) {
      for (int c = 0; c < cn; c += 4) {
        const float4 x4 = load_act4<ActT>(xp + c0 + c, a.in_scale ? a.in_scale + c0 + c : nullptr);
        const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4 *wr = ws + (c + e) * 7;
#pragma unroll
          for (int q = 0; q < 7; ++q) {
            const float4 w = wr[q];
            acc[4 * q] = fmaf(xv[e], w.x, acc[4 * q]);
            if (4 * q + 1 < 27) acc[4 * q + 1] = fmaf(xv[e], w.y, acc[4 * q + 1]);
            if (4 * q + 2 < 27) acc[4 * q + 2] = fmaf(xv[e], w.z, acc[4 * q + 2]);
            if (4 * q + 3 < 27) acc[4 * q + 3] = fmaf(xv[e], w.w, acc[4 * q + 3]);
          }
        }
      }
    }
  }
  if (tid < HPIX) {
#pragma unroll
    for (int r = 0; r < 27; ++r) ds[r * HPIX + tid] = acc[r];
  }
  __syncthreads();
  // step 2: the block's output pixels
  const int H = 2 * a.Hh, W = 2 * a.Wh;
  const float bias[3] = {__ldg(a.bias), __ldg(a.bias + 1), __ldg(a.bias + 2)};
  float pay[3] = {0.f, 0.f, 0.f};
  for (int e = tid; e < 4 * HT * HT; e += HTHREADS) {
    const int li = e / (2 * HT), lj = e - (e / (2 * HT)) * (2 * HT);  // local output row / column
    const int P = 2 * a0 + li, Q = 2 * b0 + lj;
    if (P >= H || Q >= W) continue;
    const int ar = li >> 1, pr = li & 1, bc = lj >> 1, qc = lj & 1;
    // (t_1 row offset, kernel row) pairs reaching output parity pr
    const int nr = pr ? 2 : 1, nc = qc ? 2 : 1;
    float y[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      float s = bias[o];
      for (int rr = 0; rr < nr; ++rr) {
        const int da = pr ? (rr == 0 ? 0 : 1) : 0, u = pr ? (rr == 0 ? 2 : 0) : 1;
        for (int cc = 0; cc < nc; ++cc) {
          const int db = qc ? (cc == 0 ? 0 : 1) : 0, v = qc ? (cc == 0 ? 2 : 0) : 1;
          s += ds[(o * 9 + u * 3 + v) * HPIX + (ar + da) * HE + (bc + db)];
        }
      }
      y[o] = a.relu ? fmaxf(s, 0.f) : s;
    }
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float L = expm1f(y[o]) * a.inv_exposure;
      if (payload) pay[o] += L * a.band[P];
      out[(((size_t)n * 3 + o) * H + P) * W + Q] = decode ? L : y[o];
    }
  }
  if (payload) {
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      float v = pay[o];
      for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
      if (lane == 0) red[o][warp] = v;
    }
    __syncthreads();
    if (tid < 3) {
      float v = 0.f;
      for (int w = 0; w < HTHREADS / 32; ++w) v += red[tid][w];
      atomicAdd(payload + (size_t)n * 3 + tid, v);
    }
  }
}

template <typename ActT>
void head_dispatch(const HeadArgs &a, unsigned tiles, cudaStream_t st) {
  switch (a.inline_w ? a.C : 0) {
    case 16: head_kernel<ActT, 16><<<tiles, HTHREADS, 0, st>>>(a); break;
    case 32: head_kernel<ActT, 32><<<tiles, HTHREADS, 0, st>>>(a); break;
    case 48: head_kernel<ActT, 48><<<tiles, HTHREADS, 0, st>>>(a); break;
    case 64: head_kernel<ActT, 64><<<tiles, HTHREADS, 0, st>>>(a); break;
    default: head_kernel<ActT, 0><<<tiles, HTHREADS, 0, st>>>(a); break;
  }
}

cudaError_t launch_head(const HeadArgs &a, int prec, cudaStream_t st) {
  const long long tiles = (long long)((a.Hh + HT - 1) / HT) * ((a.Wh + HT - 1) / HT) * a.N;
  if (tiles == 0) return cudaSuccess;
  if (prec == 1)
    head_dispatch<__nv_bfloat16>(a, (unsigned)tiles, st);
  else if (prec == 2)
    head_dispatch<uint8_t>(a, (unsigned)tiles, st);
  else
    head_dispatch<float>(a, (unsigned)tiles, st);
  return cudaGetLastError();
}

}  // namespace drc
