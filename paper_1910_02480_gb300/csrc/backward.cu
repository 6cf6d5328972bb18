// backward.cu -- the kernels of the training backward pass that are not
// tensor-core convolutions: the L1 loss and its gradient, the output head's
// backward, the weight-gradient GEMM shared by every conv and transposed conv,
// bias gradients, and the input gradient (Sec. 3.3 training with the L1 loss
// of Eq. 7).  The data-gradients of the encoder and decoder layers run on the
// tensor-core conv kernel (conv_tc.cu) with a second packing of the weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "backward.cuh"

namespace drc {

namespace {

template <typename T>
__device__ __forceinline__ float ldf(const T *p);
template <>
__device__ __forceinline__ float ldf<float>(const float *p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}
template <typename T>
__device__ __forceinline__ T stf(float v);
template <>
__device__ __forceinline__ float stf<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 stf<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// L1 loss mean |out - target| and dL/dout = sign(out - target) / numel
// (sign(0) = 0), or dL/dout given (GRAD_OUT); zero where the output ReLU was
// inactive.  g is written NHWC with 4 channels (the 4th zero), and when g8 is
// given also as bf16 NHWC with 8 channels (5 zero).
__global__ void l1_grad_kernel(const float *__restrict__ out, const float *__restrict__ target, int N, int H, int W,
                               int grad_out, int out_relu, float inv_numel, float *__restrict__ g4,
                               __nv_bfloat16 *__restrict__ g8, float *__restrict__ loss) {
  const long long hw = (long long)H * W;
  const long long total = (long long)N * hw;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (pix < total) {
    const long long n = pix / hw, p = pix - n * hw;
    float gv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      const long long i = (n * 3 + o) * hw + p;
      const float y = out[i], t = target[i];
      float gi;
      if (grad_out) {
        gi = t;
      } else {
        const float d = y - t;
        l += fabsf(d);
        gi = d > 0.f ? inv_numel : (d < 0.f ? -inv_numel : 0.f);
      }
      if (out_relu && !(y > 0.f)) gi = 0.f;
      gv[o] = gi;
    }
    reinterpret_cast<float4 *>(g4)[pix] = make_float4(gv[0], gv[1], gv[2], 0.f);
    if (g8) {
      const __nv_bfloat162 a = __floats2bfloat162_rn(gv[0], gv[1]), b = __floats2bfloat162_rn(gv[2], 0.f);
      reinterpret_cast<uint4 *>(g8)[pix] = make_uint4(*reinterpret_cast<const uint32_t *>(&a),
                                                      *reinterpret_cast<const uint32_t *>(&b), 0u, 0u);
    }
  }
  if (!grad_out && loss) {
    __shared__ float red[32];
    for (int d = 16; d > 0; d >>= 1) l += __shfl_xor_sync(0xffffffffu, l, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      atomicAdd(loss, s * inv_numel);
    }
  }
}

// Head backward, data part: dt1[n,i,j,c] = sum_{o,u,v} W[c][o][u][v] *
// g[n, 2i+u-1, 2j+v-1, o] (g zero outside the map).  The head weights,
// transposed to [27][C], sit in shared memory once per block; a thread takes
// 8 channels of HB_P neighbouring t_1 pixels of a row (C/8 threads per pixel
// group, 16-byte bf16 accesses), so each 16-byte weight read from shared
// memory serves HB_P pixels, and reads the pixels' g vectors itself.
// Writes gt (unmasked, nullable) and gz = gt x [mask > 0] (mask nullable).
template <typename ActT>
__device__ __forceinline__ void load8(const ActT *p, float (&v)[8]);
template <>
__device__ __forceinline__ void load8<float>(const float *p, float (&v)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4 *>(p)), b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
  v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
}
template <>
__device__ __forceinline__ void load8<__nv_bfloat16>(const __nv_bfloat16 *p, float (&v)[8]) {
  const uint4 r = __ldg(reinterpret_cast<const uint4 *>(p));
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    v[2 * e] = __uint_as_float(w[e] << 16);
    v[2 * e + 1] = __uint_as_float(w[e] & 0xFFFF0000u);
  }
}
template <typename ActT>
__device__ __forceinline__ void store8(ActT *p, const float (&v)[8]);
template <>
__device__ __forceinline__ void store8<float>(float *p, const float (&v)[8]) {
  reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4 *>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
template <>
__device__ __forceinline__ void store8<__nv_bfloat16>(__nv_bfloat16 *p, const float (&v)[8]) {
  uint32_t w[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    w[e] = *reinterpret_cast<const uint32_t *>(&h);
  }
  *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

constexpr int HB_P = 4;  // t_1 pixels per thread (along a row)
template <typename ActT>
__global__ void __launch_bounds__(256) head_bwd_kernel(const float *__restrict__ g4, const float *__restrict__ Wh,
                                                       const ActT *__restrict__ mask, ActT *__restrict__ gt,
                                                       ActT *__restrict__ gz, int N, int Hh, int Wh_, int C) {
  extern __shared__ float4 wt4[];  // [27][C / 4], row r = 9 o + 3 u + v
  float *wt = reinterpret_cast<float *>(wt4);
  for (int e = threadIdx.x; e < 27 * C; e += blockDim.x) {
    const int c = e / 27, r = e - c * 27;  // W[c][o][u][v]
    wt[r * C + c] = __ldg(Wh + e);
  }
  __syncthreads();
  const int tpg = C / 8, gpb = (int)blockDim.x / tpg;  // threads per pixel group, groups per block step
  const int lg = threadIdx.x / tpg, c0 = 8 * (threadIdx.x - lg * tpg);
  if (lg >= gpb) return;
  const int gpr = (Wh_ + HB_P - 1) / HB_P;  // pixel groups per t_1 row
  const long long groups = (long long)N * Hh * gpr;
  const int H = 2 * Hh, W = 2 * Wh_, C4 = C / 4;
  for (long long gi = (long long)blockIdx.x * gpb + lg; gi < groups; gi += (long long)gridDim.x * gpb) {
    const long long row = gi / gpr;  // n * Hh + i
    const int j0 = HB_P * (int)(gi - row * gpr);
    const long long n = row / Hh;
    const int i = (int)(row - n * Hh);
    float acc[HB_P][8];
#pragma unroll
    for (int p = 0; p < HB_P; ++p)
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[p][e] = 0.f;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int y = 2 * i + u - 1;
      if ((unsigned)y >= (unsigned)H) continue;
      const float4 *grow = reinterpret_cast<const float4 *>(g4) + (n * H + y) * W;
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        float w[3][8];  // the tap's weights of output channels o = 0..2, channels c0 .. c0 + 7
#pragma unroll
        for (int o = 0; o < 3; ++o) {
          const float4 lo = wt4[(9 * o + 3 * u + v) * C4 + c0 / 4], hi = wt4[(9 * o + 3 * u + v) * C4 + c0 / 4 + 1];
          w[o][0] = lo.x, w[o][1] = lo.y, w[o][2] = lo.z, w[o][3] = lo.w;
          w[o][4] = hi.x, w[o][5] = hi.y, w[o][6] = hi.z, w[o][7] = hi.w;
        }
#pragma unroll
        for (int p = 0; p < HB_P; ++p) {
          const int x = 2 * (j0 + p) + v - 1;
          if ((unsigned)x >= (unsigned)W) continue;
          const float4 g = __ldg(grow + x);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            acc[p][e] = fmaf(g.z, w[2][e], fmaf(g.y, w[1][e], fmaf(g.x, w[0][e], acc[p][e])));
        }
      }
    }
#pragma unroll
    for (int p = 0; p < HB_P; ++p) {
      if (j0 + p >= Wh_) break;
      const size_t off = ((size_t)row * Wh_ + j0 + p) * C + c0;
      if (gt) store8<ActT>(gt + off, acc[p]);
      if (mask) {
        float m[8];
        load8<ActT>(mask + off, m);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (!(m[e] > 0.f)) acc[p][e] = 0.f;
      }
      store8<ActT>(gz + off, acc[p]);
    }
  }
}

// Weight gradient of a 3x3 stride-2 conv / transposed conv as one GEMM:
//   dW[m][q][u][v] += sum_{n,i,j} R[n,i,j,m] * Q[n, 2i+u-1, 2j+v-1, q]
// R: NHWC at the coarse resolution (Hb x Wb, Mr channels), Q: NHWC at twice
// it (Qc stored channels, Qraw of them in the weights).  For a conv R is the
// output gradient and Q the input; for a transposed conv R is the input and
// Q the output gradient -- the packed weight layouts [Cout][Cin][3][3] and
// [Cin][Cout][3][3] are then both [m][q][3][3].
// Tiles: 64 rows (m) x 64 columns (tap-major: col = 9-tap index x Qc + q) per
// block, 16 pixels of K per step, 4 x 4 outputs per thread; each block sums
// a range of pixels and adds its tile to dW with atomics (split K).
// KAHAN (the FP32 path): the 16-pixel partial sums are added with Kahan
// compensation, and each block writes its tile as (sum, -compensation)
// pairs to part[split][element]; wgrad_reduce_kernel then adds the splits'
// pairs in a fixed order, again compensated, into dW -- L1 gradients carry
// random signs, so these sums cancel heavily and plain fp32 accumulation over
// thousands of pixels loses ~1e-4 of the result.  Otherwise the tile goes
// to dW with fp32 atomics.
constexpr int WG_T = 64, WG_K = 16;
template <typename ActR, typename ActQ, bool KAHAN>
__global__ void __launch_bounds__(256) wgrad_kernel(const ActR *__restrict__ R, const ActQ *__restrict__ Q, int N,
                                                    int Hb, int Wb, int Mr, int Qc, int Qraw, long long k_per_block,
                                                    float *__restrict__ dW, float2 *__restrict__ part) {
  __shared__ float As[WG_K][WG_T + 4];
  __shared__ float Bs[WG_K][WG_T + 4];
  const int m0 = blockIdx.x * WG_T, c0 = blockIdx.y * WG_T;
  const long long K = (long long)N * Hb * Wb;
  const long long k_begin = (long long)blockIdx.z * k_per_block;
  const long long k_end = k_begin + k_per_block < K ? k_begin + k_per_block : K;
  const int ncols = 9 * Qc;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int H = 2 * Hb, W = 2 * Wb;
  float acc[4][4] = {}, comp[4][4] = {};
  for (long long k0 = k_begin; k0 < k_end; k0 += WG_K) {
    // 16 x 64 of R and of the gathered Q: 4 elements per thread each,
    // consecutive threads along the channel axis
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = threadIdx.x + 256 * e;
      const int kk = idx >> 6, cc = idx & 63;
      const long long k = k0 + kk;
      float av = 0.f, bv = 0.f;
      if (k < k_end) {
        const int m = m0 + cc;
        if (m < Mr) av = ldf<ActR>(R + (size_t)k * Mr + m);
        const int col = c0 + cc;
        if (col < ncols) {
          const int tap = col / Qc, q = col - tap * Qc;
          const long long n = k / ((long long)Hb * Wb);
          const int rem = (int)(k - n * Hb * Wb);
          const int i = rem / Wb, j = rem - (rem / Wb) * Wb;
          const int y = 2 * i + tap / 3 - 1, x = 2 * j + tap % 3 - 1;
          if ((unsigned)y < (unsigned)H && (unsigned)x < (unsigned)W)
            bv = ldf<ActQ>(Q + (((size_t)n * H + y) * W + x) * Qc + q);
        }
      }
      As[kk][cc] = av;
      Bs[kk][cc] = bv;
    }
    __syncthreads();
    float part[4][4] = {};
#pragma unroll
    for (int kk = 0; kk < WG_K; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a[r] = As[kk][ty * 4 + r];
        b[r] = Bs[kk][tx * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) part[r][s] = fmaf(a[r], b[s], part[r][s]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if constexpr (KAHAN) {
          const float y = part[r][s] - comp[r][s];
          const float t = acc[r][s] + y;
          comp[r][s] = (t - acc[r][s]) - y;
          acc[r][s] = t;
        } else {
          acc[r][s] += part[r][s];
        }
      }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int m = m0 + ty * 4 + r;
    if (m >= Mr) continue;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int col = c0 + tx * 4 + s;
      if (col >= ncols) continue;
      const int tap = col / Qc, q = col - tap * Qc;
      if (q >= Qraw) continue;
      if constexpr (KAHAN)
        part[(size_t)blockIdx.z * ((size_t)Mr * Qraw * 9) + ((size_t)m * Qraw + q) * 9 + tap] =
            make_float2(acc[r][s], -comp[r][s]);
      else
        atomicAdd(dW + ((size_t)m * Qraw + q) * 9 + tap, acc[r][s]);
    }
  }
}

// db[c] += sum over pixels of T[pix][c], c < Craw.  A thread sums one
// 16-byte group of V channels over every L-th pixel of the block's range
// (G = C / V groups side by side, L = 256 / G pixel lanes, four loads in
// flight); the L partial rows are then added through shared memory and the
// block total goes to db with one atomic per channel.  KAHAN (the FP32
// path): Kahan-compensated partial sums, and each block's totals as
// (sum, correction) pairs in part[block][channel], added over the blocks by
// the compensated reduction.
template <typename Act, bool KAHAN>
__global__ void __launch_bounds__(256) colsum_kernel(const Act *__restrict__ T, long long npix, int C, int Craw,
                                                     long long pix_per_block, float *__restrict__ db,
                                                     float2 *__restrict__ part) {
  constexpr int V = 16 / sizeof(Act);
  extern __shared__ float cs_part[];  // [L][C] sums, then [L][C] compensations
  const int G = C / V, L = 256 / G;
  const int sub = threadIdx.x / G, g = threadIdx.x - sub * G;
  const long long p0 = (long long)blockIdx.x * pix_per_block;
  const long long p1 = p0 + pix_per_block < npix ? p0 + pix_per_block : npix;
  float s[V], cp[V];
#pragma unroll
  for (int e = 0; e < V; ++e) s[e] = cp[e] = 0.f;
  auto add = [&](const float (&x)[V]) {
#pragma unroll
    for (int e = 0; e < V; ++e) {
      if constexpr (KAHAN) {
        const float y = x[e] - cp[e];
        const float t = s[e] + y;
        cp[e] = (t - s[e]) - y;
        s[e] = t;
      } else {
        s[e] += x[e];
      }
    }
  };
  auto load = [&](long long p, float (&x)[V]) {
    if constexpr (V == 8) {
      load8<Act>(T + (size_t)p * C + g * V, x);
    } else {
      const float4 a = __ldg(reinterpret_cast<const float4 *>(T + (size_t)p * C + g * V));
      x[0] = a.x, x[1] = a.y, x[2] = a.z, x[3] = a.w;
    }
  };
  if (sub < L) {
    long long p = p0 + sub;
    for (; p + 3ll * L < p1; p += 4ll * L) {
      float x0[V], x1[V], x2[V], x3[V];
      load(p, x0);
      load(p + L, x1);
      load(p + 2ll * L, x2);
      load(p + 3ll * L, x3);
      add(x0);
      add(x1);
      add(x2);
      add(x3);
    }
    for (; p < p1; p += L) {
      float x0[V];
      load(p, x0);
      add(x0);
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
      cs_part[sub * C + g * V + e] = s[e];
      if constexpr (KAHAN) cs_part[(L + sub) * C + g * V + e] = cp[e];
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < Craw; c += blockDim.x) {
    if constexpr (KAHAN) {
      // the lanes' sums, Kahan-added, and their compensations, summed apart
      float t = 0.f, tc = 0.f, low = 0.f;
      for (int l = 0; l < L; ++l) {
        const float y = cs_part[l * C + c] - tc;
        const float u = t + y;
        tc = (u - t) - y;
        t = u;
        low -= cs_part[(L + l) * C + c];
      }
      part[(size_t)blockIdx.x * Craw + c] = make_float2(t, low - tc);
    } else {
      float t = 0.f;
      for (int l = 0; l < L; ++l) t += cs_part[l * C + c];
      atomicAdd(db + c, t);
    }
  }
}

// out[i] = sum over the S splits of the pairs part[s][i] = (sum, correction):
// the sums Kahan-added in split order, the corrections summed apart and
// added at the end.  Deterministic; overwrites out.
__global__ void compensated_reduce_kernel(const float2 *__restrict__ part, long long n, int S, float *__restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f, c = 0.f, low = 0.f;
  for (int k = 0; k < S; ++k) {
    const float2 v = part[(size_t)k * n + i];
    const float y = v.x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
    low += v.y;
  }
  out[i] = s + (low - c);
}

// Input gradient: NHWC16 (7 real channels) -> [N][7][H][W], through the log
// encode d/dx log1p(s x) = s / (1 + s x) of channels 0..2 when it was applied.
template <typename Act>
__global__ void dinput_kernel(const Act *__restrict__ g16, const float *__restrict__ x_raw, long long hw, int N,
                              int encode, float s, float *__restrict__ dinput) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= hw * N) return;
  const long long n = g / hw, p = g - n * hw;
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    float v = ldf<Act>(g16 + (size_t)g * 16 + c);
    const size_t i = ((size_t)n * 7 + c) * hw + p;
    if (encode && c < 3) v *= s / (1.f + s * x_raw[i]);
    dinput[i] = v;
  }
}

}  // namespace

cudaError_t launch_l1_grad(const float *out, const float *target, int N, int H, int W, bool grad_out, bool out_relu,
                           float *g4, void *g8, float *loss, cudaStream_t st) {
  const long long total = (long long)N * H * W;
  if (total == 0) return cudaSuccess;
  const float inv = 1.0f / (float)(3.0 * (double)total);
  l1_grad_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(out, target, N, H, W, grad_out ? 1 : 0,
                                                                  out_relu ? 1 : 0, inv, g4,
                                                                  static_cast<__nv_bfloat16 *>(g8), loss);
  return cudaGetLastError();
}

cudaError_t launch_head_bwd(const float *g4, const float *Whead, const void *mask, void *gt, void *gz, int N, int Hh,
                            int Wh, int C, bool bf16, int num_sms, cudaStream_t st) {
  const long long total = (long long)N * Hh * Wh;
  if (total == 0) return cudaSuccess;
  if (C % 8 || C > 2048) return cudaErrorInvalidValue;
  const size_t smem = (size_t)27 * C * sizeof(float);
  const long long gpb = 256 / (C / 8), groups = (long long)N * Hh * ((Wh + HB_P - 1) / HB_P);
  long long blocks = (groups + gpb - 1) / gpb;
  if (blocks > 8ll * num_sms) blocks = 8ll * num_sms;
  cudaError_t e;
  if (bf16) {
    e = cudaFuncSetAttribute(head_bwd_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    head_bwd_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, smem, st>>>(
        g4, Whead, static_cast<const __nv_bfloat16 *>(mask), static_cast<__nv_bfloat16 *>(gt),
        static_cast<__nv_bfloat16 *>(gz), N, Hh, Wh, C);
  } else {
    e = cudaFuncSetAttribute(head_bwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    head_bwd_kernel<float><<<(unsigned)blocks, 256, smem, st>>>(g4, Whead, static_cast<const float *>(mask),
                                                                static_cast<float *>(gt), static_cast<float *>(gz),
                                                                N, Hh, Wh, C);
  }
  return cudaGetLastError();
}

// Split-K shape of the SIMT weight gradient: enough K splits for about four
// blocks per SM, at least 256 pixels each.
static void wgrad_shape(long long K, int Mr, int Qc, int num_sms, int &gx, int &gy, long long &kpb, unsigned &gz) {
  gx = (Mr + WG_T - 1) / WG_T;
  gy = (9 * Qc + WG_T - 1) / WG_T;
  long long splits = (4ll * num_sms + gx * gy - 1) / (gx * gy);
  if (splits < 1) splits = 1;
  kpb = (K + splits - 1) / splits;
  if (kpb < 256) kpb = 256;
  kpb = (kpb + WG_K - 1) / WG_K * WG_K;
  gz = (unsigned)((K + kpb - 1) / kpb);
}

size_t wgrad_partial_elems(int N, int Hb, int Wb, int Mr, int Qc, int Qraw, int num_sms) {
  const long long K = (long long)N * Hb * Wb;
  if (K == 0) return 0;
  int gx, gy;
  long long kpb;
  unsigned gz;
  wgrad_shape(K, Mr, Qc, num_sms, gx, gy, kpb, gz);
  return (size_t)gz * Mr * Qraw * 9;
}

template <bool KAHAN>
static cudaError_t wgrad_dispatch(const void *R, bool r_bf16, const void *Q, bool q_bf16, int N, int Hb, int Wb,
                                  int Mr, int Qc, int Qraw, float *dW, float2 *part, int num_sms, cudaStream_t st) {
  const long long K = (long long)N * Hb * Wb;
  if (K == 0) return cudaSuccess;
  int gx, gy;
  long long kpb;
  unsigned gz;
  wgrad_shape(K, Mr, Qc, num_sms, gx, gy, kpb, gz);
  const dim3 grid(gx, gy, gz);
  using bf = __nv_bfloat16;
  if (r_bf16 && q_bf16)
    wgrad_kernel<bf, bf, KAHAN><<<grid, 256, 0, st>>>(static_cast<const bf *>(R), static_cast<const bf *>(Q), N, Hb,
                                                      Wb, Mr, Qc, Qraw, kpb, dW, part);
  else if (!r_bf16 && !q_bf16)
    wgrad_kernel<float, float, KAHAN><<<grid, 256, 0, st>>>(static_cast<const float *>(R),
                                                            static_cast<const float *>(Q), N, Hb, Wb, Mr, Qc, Qraw,
                                                            kpb, dW, part);
  else if (r_bf16)
    wgrad_kernel<bf, float, KAHAN><<<grid, 256, 0, st>>>(static_cast<const bf *>(R), static_cast<const float *>(Q), N,
                                                         Hb, Wb, Mr, Qc, Qraw, kpb, dW, part);
  else
    wgrad_kernel<float, bf, KAHAN><<<grid, 256, 0, st>>>(static_cast<const float *>(R), static_cast<const bf *>(Q), N,
                                                         Hb, Wb, Mr, Qc, Qraw, kpb, dW, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !KAHAN) return e;
  const long long n = (long long)Mr * Qraw * 9;
  compensated_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, n, (int)gz, dW);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const void *R, bool r_bf16, const void *Q, bool q_bf16, int N, int Hb, int Wb, int Mr,
                         int Qc, int Qraw, float *dW, float2 *part, int num_sms, cudaStream_t st) {
  return part ? wgrad_dispatch<true>(R, r_bf16, Q, q_bf16, N, Hb, Wb, Mr, Qc, Qraw, dW, part, num_sms, st)
              : wgrad_dispatch<false>(R, r_bf16, Q, q_bf16, N, Hb, Wb, Mr, Qc, Qraw, dW, nullptr, num_sms, st);
}

static void colsum_shape(long long npix, int C, bool bf16, int num_sms, int &L, long long &ppb, unsigned &blocks) {
  const int V = bf16 ? 8 : 4;
  L = 256 / (C / V);
  ppb = (npix + 2ll * num_sms - 1) / (2ll * num_sms);
  if (ppb < 4ll * L) ppb = 4ll * L;
  blocks = (unsigned)((npix + ppb - 1) / ppb);
}

size_t colsum_partial_elems(long long npix, int C, int Craw, bool bf16, int num_sms) {
  if (npix == 0) return 0;
  int L;
  long long ppb;
  unsigned blocks;
  colsum_shape(npix, C, bf16, num_sms, L, ppb, blocks);
  return (size_t)blocks * Craw;
}

cudaError_t launch_colsum(const void *T, bool bf16, long long npix, int C, int Craw, float *db, float2 *part,
                          int num_sms, cudaStream_t st) {
  if (npix == 0) return cudaSuccess;
  const int V = bf16 ? 8 : 4;
  if (C % V || C / V > 256) return cudaErrorInvalidValue;
  int L;
  long long ppb;
  unsigned blocks;
  colsum_shape(npix, C, bf16, num_sms, L, ppb, blocks);
  const size_t smem = (size_t)(part ? 2 : 1) * L * C * sizeof(float);
  using bf = __nv_bfloat16;
  if (part) {
    if (bf16)
      colsum_kernel<bf, true><<<blocks, 256, smem, st>>>(static_cast<const bf *>(T), npix, C, Craw, ppb, db, part);
    else
      colsum_kernel<float, true><<<blocks, 256, smem, st>>>(static_cast<const float *>(T), npix, C, Craw, ppb, db,
                                                            part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    compensated_reduce_kernel<<<(unsigned)((Craw + 255) / 256), 256, 0, st>>>(part, Craw, (int)blocks, db);
  } else {
    if (bf16)
      colsum_kernel<bf, false><<<blocks, 256, smem, st>>>(static_cast<const bf *>(T), npix, C, Craw, ppb, db, nullptr);
    else
      colsum_kernel<float, false><<<blocks, 256, smem, st>>>(static_cast<const float *>(T), npix, C, Craw, ppb, db,
                                                             nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_dinput(const void *g16, bool bf16, const float *x_raw, long long hw, int N, bool encode,
                          float exposure, float *dinput, cudaStream_t st) {
  const long long total = hw * N;
  if (total == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (bf16)
    dinput_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(g16), x_raw, hw, N,
                                                         encode ? 1 : 0, exposure, dinput);
  else
    dinput_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(g16), x_raw, hw, N, encode ? 1 : 0,
                                                 exposure, dinput);
  return cudaGetLastError();
}

}  // namespace drc
