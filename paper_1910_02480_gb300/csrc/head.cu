// head.cu -- the output layer of the autoencoder (Sec. 3.3): a 3x3 transposed
// convolution, stride 2, from the first decoder activation t_1 (C channels,
// H/2 x W/2, NHWC) to the 3 radiance channels (H x W, NCHW), with the
// optional final ReLU and log decode, and the per-map irradiance payload
// E/pi (Eq. 2 with a white Lambertian BRDF).
//
// With 3 output channels a tensor-core tile would be 3/16 useful, so this
// layer is plain fp32 FMA (exact fp32 rounding, no split needed).  One CTA
// covers an 8x8 block of t_1 pixels of one map = 16x16 output pixels: each
// warp handles one output parity phase, so all lanes of a warp share the same
// taps and read the same weights (shared-memory broadcast).  Channels are
// staged 64 at a time: the 9x9 input window transposed to [c][pixel] and the
// weights as [tap][c] float4 (o = 0..2).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstdint>
#include <cuda_runtime.h>

#include "head.cuh"

namespace drc {

constexpr int HT = 8;        // t_1 block edge per CTA
constexpr int HWIN = HT + 1; // input window edge (odd phases read one more)
constexpr int HC = 64;       // channels staged per pass

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

template <typename ActT>
__global__ void __launch_bounds__(256, 4) head_kernel(const __grid_constant__ HeadArgs a) {
  __shared__ float xs[HC * HWIN * HWIN];
  __shared__ float4 ws[9 * HC];
  __shared__ float red[3][8];
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
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pp = (warp >> 1) >> 1, qq = (warp >> 1) & 1;  // output parity of this warp
  const int idx = (warp & 1) * 32 + lane;
  const int ai = idx / HT, bi = idx % HT;
  const bool valid = a0 + ai < a.Hh && b0 + bi < a.Wh;
  // taps of this phase: output row 2a+pp gathers input row a+di through
  // kernel row u with 2(a+di) + u - 1 = 2a + pp
  int nr, nc, ru[2], rd[2], cu[2], cd[2];
  if (pp == 0) {
    nr = 1;
    ru[0] = 1;
    rd[0] = 0;
  } else {
    nr = 2;
    ru[0] = 0;
    rd[0] = 1;
    ru[1] = 2;
    rd[1] = 0;
  }
  if (qq == 0) {
    nc = 1;
    cu[0] = 1;
    cd[0] = 0;
  } else {
    nc = 2;
    cu[0] = 0;
    cd[0] = 1;
    cu[1] = 2;
    cd[1] = 0;
  }
  const ActT *x = reinterpret_cast<const ActT *>(a.x) + (size_t)n * a.Hh * a.Wh * a.C;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  for (int c0 = 0; c0 < a.C; c0 += HC) {
    const int cn = min(HC, a.C - c0);
    __syncthreads();
    // 81 pixels x 16 four-channel groups: all loads issued before any store
    constexpr int NG = HWIN * HWIN * (HC / 4);
    constexpr int PER = (NG + 255) / 256;
    float4 v[PER];
#pragma unroll
    for (int it = 0; it < PER; ++it) {
      const int e = threadIdx.x + it * 256;
      const int pix = e / (HC / 4), g = e % (HC / 4);
      const int y = a0 + pix / HWIN, xx = b0 + pix % HWIN;
      v[it] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < NG && 4 * g < cn && y < a.Hh && xx < a.Wh)
        v[it] = load_act4<ActT>(x + ((size_t)y * a.Wh + xx) * a.C + c0 + 4 * g, a.in_scale + c0 + 4 * g);
    }
#pragma unroll
    for (int it = 0; it < PER; ++it) {
      const int e = threadIdx.x + it * 256;
      if (e < NG) {
        const int pix = e / (HC / 4), g = e % (HC / 4);
        xs[(4 * g + 0) * HWIN * HWIN + pix] = v[it].x;
        xs[(4 * g + 1) * HWIN * HWIN + pix] = v[it].y;
        xs[(4 * g + 2) * HWIN * HWIN + pix] = v[it].z;
        xs[(4 * g + 3) * HWIN * HWIN + pix] = v[it].w;
      }
    }
    for (int e = threadIdx.x; e < 9 * HC; e += blockDim.x) {
      const int t = e / HC, c = e % HC;
      float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c < cn) {
        const float *wc = a.w + (size_t)(c0 + c) * 27 + t;  // W[c][o][u][v], t = 3u + v
        w = make_float4(__ldg(wc), __ldg(wc + 9), __ldg(wc + 18), 0.f);
      }
      ws[t * HC + c] = w;
    }
    __syncthreads();
    for (int r = 0; r < nr; ++r)
      for (int s = 0; s < nc; ++s) {
        const int pix = (ai + rd[r]) * HWIN + (bi + cd[s]);
        const float4 *wt = ws + (ru[r] * 3 + cu[s]) * HC;
#pragma unroll 8
        for (int c = 0; c < HC; ++c) {
          const float xv = xs[c * HWIN * HWIN + pix];
          const float4 w = wt[c];
          acc0 = fmaf(xv, w.x, acc0);
          acc1 = fmaf(xv, w.y, acc1);
          acc2 = fmaf(xv, w.z, acc2);
        }
      }
  }
  float y[3] = {acc0 + a.bias[0], acc1 + a.bias[1], acc2 + a.bias[2]};
  const int p = 2 * (a0 + ai) + pp, q = 2 * (b0 + bi) + qq;
  const int H = 2 * a.Hh, W = 2 * a.Wh;
  float pay[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    if (a.relu) y[o] = fmaxf(y[o], 0.f);
    const float L = expm1f(y[o]) * a.inv_exposure;
    pay[o] = (valid && payload) ? L * a.band[p] : 0.f;
    if (valid) out[(((size_t)n * 3 + o) * H + p) * W + q] = decode ? L : y[o];
  }
  if (payload) {
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      float v = pay[o];
      for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
      if (lane == 0) red[o][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      float v = 0.f;
      for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
      atomicAdd(payload + (size_t)n * 3 + threadIdx.x, v);
    }
  }
}

cudaError_t launch_head(const HeadArgs &a, int prec, cudaStream_t st) {
  const long long tiles = (long long)((a.Hh + HT - 1) / HT) * ((a.Wh + HT - 1) / HT) * a.N;
  if (tiles == 0) return cudaSuccess;
  if (prec == 1)
    head_kernel<__nv_bfloat16><<<(unsigned)tiles, 256, 0, st>>>(a);
  else if (prec == 2)
    head_kernel<uint8_t><<<(unsigned)tiles, 256, 0, st>>>(a);
  else
    head_kernel<float><<<(unsigned)tiles, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace drc
