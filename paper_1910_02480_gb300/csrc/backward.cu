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
// inactive.  g is written NHWC with 4 channels (the 4th zero).
__global__ void l1_grad_kernel(const float *__restrict__ out, const float *__restrict__ target, int N, int H, int W,
                               int grad_out, int out_relu, float inv_numel, float *__restrict__ g4,
                               float *__restrict__ loss) {
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
// g[n, 2i+u-1, 2j+v-1, o] (g zero outside the map).  A block takes 16 t_1
// pixels; the 27 g values of each are staged in shared memory and the head
// weights, transposed to [27][C], too; a warp covers 32 channels of a pixel
// (coalesced stores).  Writes gt (unmasked, nullable) and gz = gt x [mask > 0]
// (mask nullable).
constexpr int HB_PIX = 16;
template <typename ActT>
__global__ void __launch_bounds__(256) head_bwd_kernel(const float *__restrict__ g4, const float *__restrict__ Wh,
                                                       const ActT *__restrict__ mask, ActT *__restrict__ gt,
                                                       ActT *__restrict__ gz, int N, int Hh, int Wh_, int C) {
  extern __shared__ float hb_smem[];
  float *wt = hb_smem;            // [27][C]
  float *gs = hb_smem + 27 * C;   // [HB_PIX][27]
  for (int e = threadIdx.x; e < 27 * C; e += blockDim.x) {
    const int c = e / 27, r = e - c * 27;  // W[c][o][u][v], r = 9 o + 3 u + v
    wt[r * C + c] = __ldg(Wh + e);
  }
  const long long total = (long long)N * Hh * Wh_;
  const long long p0 = (long long)blockIdx.x * HB_PIX;
  const int H = 2 * Hh, W = 2 * Wh_;
  for (int e = threadIdx.x; e < HB_PIX * 27; e += blockDim.x) {
    const int lp = e / 27, r = e - lp * 27;
    const long long pix = p0 + lp;
    float v = 0.f;
    if (pix < total) {
      const int o = r / 9, u = (r / 3) % 3, vv = r % 3;
      const long long n = pix / ((long long)Hh * Wh_);
      const int rem = (int)(pix - n * Hh * Wh_);
      const int i = rem / Wh_, j = rem - (rem / Wh_) * Wh_;
      const int y = 2 * i + u - 1, x = 2 * j + vv - 1;
      if ((unsigned)y < (unsigned)H && (unsigned)x < (unsigned)W) v = g4[((n * H + y) * W + x) * 4 + o];
    }
    gs[e] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int lp = warp; lp < HB_PIX; lp += blockDim.x >> 5) {
    const long long pix = p0 + lp;
    if (pix >= total) break;
    const float *gp = gs + lp * 27;
    for (int c = lane; c < C; c += 32) {
      float acc = 0.f;
#pragma unroll
      for (int r = 0; r < 27; ++r) acc = fmaf(wt[r * C + c], gp[r], acc);
      const size_t off = (size_t)pix * C + c;
      if (gt) gt[off] = stf<ActT>(acc);
      if (mask && !(ldf<ActT>(mask + off) > 0.f)) acc = 0.f;
      gz[off] = stf<ActT>(acc);
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
// AccT = double (the FP32 path): the 16-pixel partial sums are added with
// Kahan compensation and the block totals into an fp64 buffer -- L1
// gradients carry random signs, so these sums cancel heavily and plain fp32
// accumulation over thousands of pixels loses ~1e-4 of the result.
constexpr int WG_T = 64, WG_K = 16;
template <typename ActR, typename ActQ, typename AccT>
__global__ void __launch_bounds__(256) wgrad_kernel(const ActR *__restrict__ R, const ActQ *__restrict__ Q, int N,
                                                    int Hb, int Wb, int Mr, int Qc, int Qraw, long long k_per_block,
                                                    AccT *__restrict__ dW) {
  constexpr bool KAHAN = sizeof(AccT) == 8;
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
        atomicAdd(dW + ((size_t)m * Qraw + q) * 9 + tap, (double)acc[r][s] - (double)comp[r][s]);
      else
        atomicAdd(dW + ((size_t)m * Qraw + q) * 9 + tap, acc[r][s]);
    }
  }
}

// db[c] += sum over pixels of T[pix][c], c < Craw.  256 threads: up to 256
// channels side by side (coalesced), 256 / that many pixel lanes.
template <typename Act, typename AccT>
__global__ void __launch_bounds__(256) colsum_kernel(const Act *__restrict__ T, long long npix, int C, int Craw,
                                                     long long pix_per_block, AccT *__restrict__ db) {
  const long long p0 = (long long)blockIdx.x * pix_per_block;
  const long long p1 = p0 + pix_per_block < npix ? p0 + pix_per_block : npix;
  const int cs = C < 256 ? C : 256;
  const int lanes = 256 / cs;
  const int cl = threadIdx.x % cs, sub = threadIdx.x / cs;
  if (sub >= lanes) return;
  for (int c = cl; c < C; c += cs) {
    float s = 0.f, comp = 0.f;  // Kahan-compensated (the compensation is dropped for fp32 totals)
    for (long long p = p0 + sub; p < p1; p += lanes) {
      const float y = ldf<Act>(T + (size_t)p * C + c) - comp;
      const float t = s + y;
      comp = (t - s) - y;
      s = t;
    }
    if (c < Craw) atomicAdd(db + c, (AccT)s - (AccT)comp);
  }
}

// dweights (fp32) = the fp64 accumulation buffer.
__global__ void to_f32_kernel(const double *__restrict__ a, long long n, float *__restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)a[i];
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
                           float *g4, float *loss, cudaStream_t st) {
  const long long total = (long long)N * H * W;
  if (total == 0) return cudaSuccess;
  const float inv = 1.0f / (float)(3.0 * (double)total);
  l1_grad_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(out, target, N, H, W, grad_out ? 1 : 0,
                                                                  out_relu ? 1 : 0, inv, g4, loss);
  return cudaGetLastError();
}

cudaError_t launch_head_bwd(const float *g4, const float *Whead, const void *mask, void *gt, void *gz, int N, int Hh,
                            int Wh, int C, bool bf16, cudaStream_t st) {
  const long long total = (long long)N * Hh * Wh;
  if (total == 0) return cudaSuccess;
  const size_t smem = (size_t)(27 * C + HB_PIX * 27) * sizeof(float);
  const unsigned blocks = (unsigned)((total + HB_PIX - 1) / HB_PIX);
  cudaError_t e;
  if (bf16) {
    e = cudaFuncSetAttribute(head_bwd_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    head_bwd_kernel<__nv_bfloat16><<<blocks, 256, smem, st>>>(
        g4, Whead, static_cast<const __nv_bfloat16 *>(mask), static_cast<__nv_bfloat16 *>(gt),
        static_cast<__nv_bfloat16 *>(gz), N, Hh, Wh, C);
  } else {
    e = cudaFuncSetAttribute(head_bwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    head_bwd_kernel<float><<<blocks, 256, smem, st>>>(g4, Whead, static_cast<const float *>(mask),
                                                      static_cast<float *>(gt), static_cast<float *>(gz), N, Hh, Wh, C);
  }
  return cudaGetLastError();
}

template <typename AccT>
cudaError_t wgrad_dispatch(const void *R, bool r_bf16, const void *Q, bool q_bf16, int N, int Hb, int Wb, int Mr,
                           int Qc, int Qraw, AccT *dW, int num_sms, cudaStream_t st) {
  const long long K = (long long)N * Hb * Wb;
  if (K == 0) return cudaSuccess;
  const int gx = (Mr + WG_T - 1) / WG_T, gy = (9 * Qc + WG_T - 1) / WG_T;
  // enough K splits for about four blocks per SM, at least 256 pixels each
  long long splits = (4ll * num_sms + gx * gy - 1) / (gx * gy);
  if (splits < 1) splits = 1;
  long long kpb = (K + splits - 1) / splits;
  if (kpb < 256) kpb = 256;
  kpb = (kpb + WG_K - 1) / WG_K * WG_K;
  const unsigned gz = (unsigned)((K + kpb - 1) / kpb);
  const dim3 grid(gx, gy, gz);
  using bf = __nv_bfloat16;
  if (r_bf16 && q_bf16)
    wgrad_kernel<bf, bf, AccT><<<grid, 256, 0, st>>>(static_cast<const bf *>(R), static_cast<const bf *>(Q), N, Hb,
                                                     Wb, Mr, Qc, Qraw, kpb, dW);
  else if (!r_bf16 && !q_bf16)
    wgrad_kernel<float, float, AccT><<<grid, 256, 0, st>>>(static_cast<const float *>(R),
                                                           static_cast<const float *>(Q), N, Hb, Wb, Mr, Qc, Qraw,
                                                           kpb, dW);
  else if (r_bf16)
    wgrad_kernel<bf, float, AccT><<<grid, 256, 0, st>>>(static_cast<const bf *>(R), static_cast<const float *>(Q), N,
                                                        Hb, Wb, Mr, Qc, Qraw, kpb, dW);
  else
    wgrad_kernel<float, bf, AccT><<<grid, 256, 0, st>>>(static_cast<const float *>(R), static_cast<const bf *>(Q), N,
                                                        Hb, Wb, Mr, Qc, Qraw, kpb, dW);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const void *R, bool r_bf16, const void *Q, bool q_bf16, int N, int Hb, int Wb, int Mr,
                         int Qc, int Qraw, float *dW, double *dW64, int num_sms, cudaStream_t st) {
  return dW64 ? wgrad_dispatch<double>(R, r_bf16, Q, q_bf16, N, Hb, Wb, Mr, Qc, Qraw, dW64, num_sms, st)
              : wgrad_dispatch<float>(R, r_bf16, Q, q_bf16, N, Hb, Wb, Mr, Qc, Qraw, dW, num_sms, st);
}

cudaError_t launch_colsum(const void *T, bool bf16, long long npix, int C, int Craw, float *db, double *db64,
                          int num_sms, cudaStream_t st) {
  if (npix == 0) return cudaSuccess;
  long long ppb = (npix + 2ll * num_sms - 1) / (2ll * num_sms);
  if (ppb < 64) ppb = 64;
  const unsigned blocks = (unsigned)((npix + ppb - 1) / ppb);
  using bf = __nv_bfloat16;
  if (db64) {
    if (bf16)
      colsum_kernel<bf, double><<<blocks, 256, 0, st>>>(static_cast<const bf *>(T), npix, C, Craw, ppb, db64);
    else
      colsum_kernel<float, double><<<blocks, 256, 0, st>>>(static_cast<const float *>(T), npix, C, Craw, ppb, db64);
  } else {
    if (bf16)
      colsum_kernel<bf, float><<<blocks, 256, 0, st>>>(static_cast<const bf *>(T), npix, C, Craw, ppb, db);
    else
      colsum_kernel<float, float><<<blocks, 256, 0, st>>>(static_cast<const float *>(T), npix, C, Craw, ppb, db);
  }
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const double *a, long long n, float *out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, out);
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
