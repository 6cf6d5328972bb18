// head.cu -- the output layer of the autoencoder (Sec. 3.3): a 3x3 transposed
// convolution, stride 2, from the first decoder activation t_1 (C channels,
// H/2 x W/2, NHWC) to the 3 radiance channels (H x W, NCHW), with the
// optional final ReLU and log decode, and the per-map irradiance payload
// E/pi (Eq. 2 with a white Lambertian BRDF).
//
// With 3 output channels a tensor-core tile would be 3/16 useful, so this
// layer is plain fp32 FMA (exact fp32 rounding, no split needed), in two
// steps per CTA.  A CTA covers a 16 x 16 block of t_1 pixels of one map, one
// thread per pixel:
//   1. D[p][r] = sum_c x[p][c] W[c][r] for the 27 r = (o, u, v): the input is
//      read once (4 channels per vector load).  For C <= 64 (CI > 0) the
//      weights come with the launch parameters and, the channel loop being
//      unrolled, every FMA reads its weight as a constant-bank operand (no
//      load instruction); wider layers stage the weights in shared memory
//      (7 float4 broadcasts per channel).  The row below and the column right
//      of the block (the halo, which the block's last output rows / columns
//      also gather) get a second pass only where they lie inside the map;
//   2. each thread writes the 2 x 2 output quad (2a + p, 2b + q) of its t_1
//      pixel (a, b): output row 2a + p gathers t_1 row a + d through tap u
//      with 2(a + d) + u - 1 = 2a + p, so the quad reads D at (a, b) (four
//      taps), (a, b + 1) and (a + 1, b) (two each) and (a + 1, b + 1) (one),
//      adds the bias, and stores two float2 rows per output channel
//      (coalesced rows of the NCHW planes) with the decode and the payload.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstdint>
#include <cuda_runtime.h>

#include "head.cuh"

namespace drc {

constexpr int HT = 16;           // t_1 block edge per CTA
constexpr int HE = HT + 1;       // with the halo row / column
constexpr int HPIX = HE * HE;    // entries of D per CTA
constexpr int HTHREADS = HT * HT;  // one thread per t_1 pixel of the block
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

// Step 1 for one t_1 pixel, channels [c0, c0 + cn): acc[r] += x[c] W[c][r].
// CI > 0: all CI channels, weights from the launch parameters; CI == 0: the
// chunk staged in ws.
template <typename ActT, int CI>
__device__ __forceinline__ void head_d(const HeadArgs &a, const ActT *xp, const float4 *ws, int c0, int cn,
                                       float (&acc)[27]) {
  if constexpr (CI > 0) {
#pragma unroll
    for (int c = 0; c < CI; c += 4) {
      const float4 x4 = load_act4<ActT>(xp + c, a.in_scale ? a.in_scale + c : nullptr);
      const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int r = 0; r < 27; ++r) acc[r] = fmaf(xv[e], a.wk[(c + e) * 27 + r], acc[r]);
    }
  } else {
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

template <typename ActT, int CI>
__global__ void __launch_bounds__(HTHREADS, 4) head_kernel(const __grid_constant__ HeadArgs a) {
  __shared__ float4 ws[CI > 0 ? 1 : HCC * 7];  // W[c][r] of one channel chunk, r = 9 o + 3 u + v (27 of 28)
  __shared__ float ds[27 * HPIX];              // D[r][pixel], pixel = row * HE + column
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
  const ActT *x = reinterpret_cast<const ActT *>(a.x);
  // step 1, pass 0: the block's own pixels; pass 1 (only where the halo row
  // or column lies inside the map): threads 0..32 take the halo, row HT
  // (h < 16), column HT (16 <= h < 32) and the corner (h = 32)
  const bool halo_in = a0 + HT < a.Hh || b0 + HT < a.Wh;  // block-uniform
  for (int pass = 0; pass < (halo_in ? 2 : 1); ++pass) {
    int pi, pj;
    if (pass == 0) {
      pi = tid / HT;
      pj = tid - pi * HT;
    } else {
      pi = tid < 16 ? HT : (tid < 32 ? tid - 16 : HT);
      pj = tid < 16 ? tid : HT;
    }
    const bool mine = pass == 0 || tid <= 32;
    const bool vpix = mine && a0 + pi < a.Hh && b0 + pj < a.Wh;
    const ActT *xp = x + (((size_t)n * a.Hh + (vpix ? a0 + pi : 0)) * a.Wh + (vpix ? b0 + pj : 0)) * a.C;
    float acc[27];
#pragma unroll
    for (int r = 0; r < 27; ++r) acc[r] = 0.f;
    if constexpr (CI > 0) {
      if (vpix) head_d<ActT, CI>(a, xp, ws, 0, CI, acc);
    } else {
      for (int c0 = 0; c0 < a.C; c0 += HCC) {
        const int cn = min(HCC, a.C - c0);
        __syncthreads();
        for (int e = tid; e < cn * 7; e += HTHREADS) {
          const int c = e / 7, q = e - c * 7;
          const float *wc = a.w + (size_t)(c0 + c) * 27 + 4 * q;
          ws[e] = make_float4(__ldg(wc), __ldg(wc + 1), __ldg(wc + 2), q < 6 ? __ldg(wc + 3) : 0.f);
        }
        __syncthreads();
        if (vpix) head_d<ActT, CI>(a, xp, ws, c0, cn, acc);
      }
    }
    if (mine) {
#pragma unroll
      for (int r = 0; r < 27; ++r) ds[r * HPIX + pi * HE + pj] = acc[r];
    }
  }
  if (!halo_in && tid <= 32) {  // halo outside the map: zero
    const int pi = tid < 16 ? HT : (tid < 32 ? tid - 16 : HT), pj = tid < 16 ? tid : HT;
#pragma unroll
    for (int r = 0; r < 27; ++r) ds[r * HPIX + pi * HE + pj] = 0.f;
  }
  __syncthreads();
  // step 2: this thread's output quad
  const int H = 2 * a.Hh, W = 2 * a.Wh;
  const int ar = tid / HT, bc = tid - ar * HT;
  float pay[3] = {0.f, 0.f, 0.f};
  if (a0 + ar < a.Hh && b0 + bc < a.Wh) {
    const int P = 2 * (a0 + ar), Q = 2 * (b0 + bc);
    const float *d00 = ds + ar * HE + bc;  // D at (a, b); + 1: (a, b + 1); + HE: (a + 1, b)
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const float *d = d00 + o * 9 * HPIX;
      const float b = __ldg(a.bias + o);
      float y[4];
      y[0] = b + d[(3 + 1) * HPIX];
      y[1] = b + d[(3 + 2) * HPIX] + d[(3 + 0) * HPIX + 1];
      y[2] = b + d[(6 + 1) * HPIX] + d[(0 + 1) * HPIX + HE];
      y[3] = b + d[(6 + 2) * HPIX] + d[(6 + 0) * HPIX + 1] + d[(0 + 2) * HPIX + HE] + d[(0 + 0) * HPIX + HE + 1];
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (a.relu) y[e] = fmaxf(y[e], 0.f);
        const float L = expm1f(y[e]) * a.inv_exposure;
        pay[o] += L * a.band[P + (e >> 1)];
        v[e] = decode ? L : y[e];
      }
      float *op = out + (((size_t)n * 3 + o) * H + P) * W + Q;
      *reinterpret_cast<float2 *>(op) = make_float2(v[0], v[1]);
      *reinterpret_cast<float2 *>(op + W) = make_float2(v[2], v[3]);
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
