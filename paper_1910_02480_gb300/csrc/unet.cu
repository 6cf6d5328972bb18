// unet.cu -- the paper's own network form (Sec. 3.3, "Neural network") on
// the CUDA cores in FP32: a U-Net whose encoder stages take two 3x3
// convolutions (doubling the depth) and whose decoder stages take two 3x3
// transposed convolutions (halving it), with batch normalisation and
// LeakyReLU between, 2x2 max pooling down, 2x bilinear upsampling up,
// concatenated skips, and a 1x1 convolution with ReLU at the end.
//
// Readings (the paper's network diagram is missing): stride 1 and padding 1
// for every 3x3 layer; levels l = 0..L of depth base 2^l, the deepest one the
// bottleneck; a decoder stage concatenates the upsampled deeper features
// (first) with its level's encoder output (second); the output stage (level
// 0 of the decoder) has no batch normalisation; PyTorch's conventions, the
// paper's framework: LeakyReLU slope 0.01, batch-normalisation eps 1e-5,
// bilinear sampling at half-pixel centres.
//
// The forward pass:
//   1. unet_fold_kernel, per 3x3 layer: batch normalisation at inference is
//      an affine map per output channel, folded into the weights and bias;
//      a stride-1 transposed convolution is the convolution with the kernel
//      turned by 180 degrees and its channel axes swapped.  Every 3x3 layer
//      is then one convolution with weights laid out [Cin][9][Cout].
//   2. unet_conv3x3_kernel: a block computes 16 output channels of up to 256
//      output pixels -- a 16 x 16 tile of one map, or whole small maps, up to
//      64 of them (the deepest levels are 4 x 4).  Input channels go in
//      chunks of 8: the halo tile and the chunk's weights are staged in
//      shared memory, each thread accumulates its pixel's 16 outputs.  The
//      concatenated skip is read from its two sources directly.
//   3. unet_maxpool2_kernel, unet_upsample2_kernel, unet_head_kernel: one
//      thread per output element / pixel.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "unet.cuh"

namespace drc {

namespace {

constexpr float kLreluSlope = 0.01f;
constexpr float kBnEps = 1e-5f;
constexpr int UTHREADS = 256;
constexpr int UCC = 8;          // input channels per staged chunk
constexpr int UCOB = 16;        // output channels per block
constexpr int UMPB_MAX = 64;    // maps per block at most
constexpr int UXS_MAX = 9216;   // staged input floats: UCC x maps x (TH + 2) x (TW + 2) <= 8 x 1152

using LayerDesc = UnetLayer;

std::vector<LayerDesc> unet_layers(const UnetShape &u, size_t *n_src, size_t *n_dst) {
  std::vector<LayerDesc> L;
  size_t src = 0, dst = 0;
  auto add = [&](int kind, int cin, int cout, int bn) {
    L.push_back(LayerDesc{kind, cin, cout, bn, src, dst});
    const size_t nw = (kind == 2 ? 1 : 9) * (size_t)cin * cout;
    src += nw + cout + (bn ? 4 * (size_t)cout : 0);
    dst += nw + cout;
  };
  for (int l = 0; l <= u.levels; ++l) {
    const int c = u.base << l, ci = l == 0 ? u.cin : u.base << (l - 1);
    add(0, ci, c, 1);
    add(0, c, c, 1);
  }
  for (int l = u.levels - 1; l >= 0; --l) {
    const int c = u.base << l;
    add(1, 3 * c, c, l > 0);
    add(1, c, c, l > 0);
  }
  add(2, u.base, u.cout, 0);
  if (n_src) *n_src = src;
  if (n_dst) *n_dst = dst;
  return L;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct UnetBufs {
  float *fold = nullptr;
  float *enc_a[8] = {}, *enc[8] = {}, *pool[8] = {}, *up[8] = {}, *dec_a[8] = {}, *dec[8] = {};
};

// Byte layout of the workspace; with base == nullptr only the size.
size_t unet_carve(const UnetShape &u, int N, int H, int W, char *base, UnetBufs *b) {
  size_t n_dst = 0;
  unet_layers(u, nullptr, &n_dst);
  size_t off = 0;
  auto take = [&](size_t floats) -> float * {
    float *p = base ? reinterpret_cast<float *>(base + off) : nullptr;
    off += align256(floats * sizeof(float));
    return p;
  };
  float *f = take(n_dst);
  if (b) b->fold = f;
  for (int l = 0; l <= u.levels; ++l) {
    const size_t px = (size_t)N * (H >> l) * (W >> l);
    const size_t c = (size_t)u.base << l;
    float *ea = take(px * c), *e = take(px * c);
    float *pl = l > 0 ? take(px * (c / 2)) : nullptr;
    float *up = nullptr, *da = nullptr, *d = nullptr;
    if (l < u.levels) {
      up = take(px * 2 * c);
      da = take(px * c);
      d = take(px * c);
    }
    if (b) {
      b->enc_a[l] = ea;
      b->enc[l] = e;
      b->pool[l] = pl;
      b->up[l] = up;
      b->dec_a[l] = da;
      b->dec[l] = d;
    }
  }
  return off;
}

// CONV_FORM: the 3x3 layers' destination is [o][c][u][v] (the tensor-core
// packer's input); otherwise [c][t][o] (the CUDA-core kernel's).
template <bool CONV_FORM>
__global__ void unet_fold_kernel(const float *P, int kind, int cin, int cout, int bn, size_t src, size_t dst,
                                 float *F) {
  const size_t nw = (kind == 2 ? 1 : 9) * (size_t)cin * cout;
  const float *Wt = P + src, *b = Wt + nw;
  const float *g = b + cout, *be = g + cout, *mu = be + cout, *var = mu + cout;
  float *dw = F + dst, *db = dw + nw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nw + cout; e += (size_t)gridDim.x * blockDim.x) {
    if (e < nw) {
      int o;
      float val;
      if (kind == 2) {  // head: [o][c], unchanged
        o = (int)(e / cin);
        val = Wt[e];
      } else if (CONV_FORM) {  // destination [o][c][u][v]
        o = (int)(e / (9 * (size_t)cin));
        const int c = (int)((e / 9) % cin), t = (int)(e % 9), u = t / 3, v = t - 3 * (t / 3);
        val = kind == 0 ? Wt[e] : Wt[(((size_t)c * cout + o) * 3 + (2 - u)) * 3 + (2 - v)];
      } else {  // destination [c][t][o], t = 3 u + v
        o = (int)(e % cout);
        const size_t ct = e / cout;
        const int t = (int)(ct % 9), c = (int)(ct / 9), u = t / 3, v = t - 3 * (t / 3);
        val = kind == 0 ? Wt[(((size_t)o * cin + c) * 3 + u) * 3 + v]
                        : Wt[(((size_t)c * cout + o) * 3 + (2 - u)) * 3 + (2 - v)];
      }
      dw[e] = bn ? val * (g[o] / sqrtf(var[o] + kBnEps)) : val;
    } else {
      const int o = (int)(e - nw);
      db[o] = bn ? (b[o] - mu[o]) * (g[o] / sqrtf(var[o] + kBnEps)) + be[o] : b[o];
    }
  }
}

__global__ void __launch_bounds__(UTHREADS) unet_conv3x3_kernel(const float *x1, int C1, const float *x2, int C2,
                                                                int N, int H, int W, const float *wr,
                                                                const float *bias, int Cout, float slope, float *y,
                                                                int TH, int TW, int MPB, int tiles_x) {
  __shared__ float xs[UXS_MAX];
  __shared__ __align__(16) float ws[UCC * 9 * UCOB];
  const int Cin = C1 + C2;
  const int tile = blockIdx.x, o0 = blockIdx.y * UCOB, n0 = blockIdx.z * MPB;
  const int ty0 = (tile / tiles_x) * TH, tx0 = (tile - (tile / tiles_x) * tiles_x) * TW;
  const int tid = threadIdx.x, P = TH * TW;
  const int m = tid / P, pp = tid - m * P, ty = pp / TW, tx = pp - (pp / TW) * TW;
  const int n = n0 + m, i = ty0 + ty, j = tx0 + tx;
  const bool active = m < MPB && n < N && i < H && j < W;
  const int SW = TW + 2, plane = (TH + 2) * SW, staged = UCC * MPB * plane;
  float acc[UCOB];
#pragma unroll
  for (int o = 0; o < UCOB; ++o) acc[o] = 0.f;
  for (int c0 = 0; c0 < Cin; c0 += UCC) {
    for (int e = tid; e < staged; e += UTHREADS) {  // [c][map][row][col], halo of 1
      const int c = e / (MPB * plane);
      int r = e - c * (MPB * plane);
      const int mm = r / plane;
      r -= mm * plane;
      const int sr = r / SW, sc = r - (r / SW) * SW;
      const int cc = c0 + c, nn = n0 + mm, gi = ty0 + sr - 1, gj = tx0 + sc - 1;
      float v = 0.f;
      if (cc < Cin && nn < N && gi >= 0 && gi < H && gj >= 0 && gj < W)
        v = cc < C1 ? __ldg(x1 + (((size_t)nn * C1 + cc) * H + gi) * W + gj)
                    : __ldg(x2 + (((size_t)nn * C2 + (cc - C1)) * H + gi) * W + gj);
      xs[e] = v;
    }
    for (int e = tid; e < UCC * 9 * UCOB; e += UTHREADS) {  // [c][t][o]
      const int c = e / (9 * UCOB), t = (e / UCOB) % 9, o = e % UCOB;
      const int cc = c0 + c, oo = o0 + o;
      ws[e] = cc < Cin && oo < Cout ? __ldg(wr + ((size_t)cc * 9 + t) * Cout + oo) : 0.f;
    }
    __syncthreads();
    if (active) {
      // the chunk's 72 terms into a partial sum, then into the total: a
      // serial fp32 sum of all 9 Cin terms (6912 at the widest layer) rounds
      // about sqrt(9 Cin) times the unit, the two levels about
      // sqrt(72) + sqrt(Cin / 8)
      float part[UCOB];
#pragma unroll
      for (int o = 0; o < UCOB; ++o) part[o] = 0.f;
      for (int c = 0; c < UCC; ++c) {
        const float *xp = xs + (c * MPB + m) * plane + ty * SW + tx;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const float xv = xp[(t / 3) * SW + t % 3];
          const float4 *wp = reinterpret_cast<const float4 *>(ws + (c * 9 + t) * UCOB);
#pragma unroll
          for (int q = 0; q < UCOB / 4; ++q) {
            const float4 w4 = wp[q];
            part[4 * q] = fmaf(xv, w4.x, part[4 * q]);
            part[4 * q + 1] = fmaf(xv, w4.y, part[4 * q + 1]);
            part[4 * q + 2] = fmaf(xv, w4.z, part[4 * q + 2]);
            part[4 * q + 3] = fmaf(xv, w4.w, part[4 * q + 3]);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < UCOB; ++o) acc[o] += part[o];
    }
    __syncthreads();
  }
  if (!active) return;
#pragma unroll
  for (int o = 0; o < UCOB; ++o) {
    const int oo = o0 + o;
    if (oo < Cout) {
      float z = acc[o] + __ldg(bias + oo);
      z = z >= 0.f ? z : slope * z;
      y[(((size_t)n * Cout + oo) * H + i) * W + j] = z;
    }
  }
}

__global__ void unet_maxpool2_kernel(const float *x, int NC, int H, int W, float *y) {
  const int Ho = H / 2, Wo = W / 2;
  const size_t total = (size_t)NC * Ho * Wo;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t nc = e / ((size_t)Ho * Wo);
    const int r = (int)(e - nc * Ho * Wo), i = r / Wo, j = r - (r / Wo) * Wo;
    const float *s = x + nc * H * W + (size_t)(2 * i) * W + 2 * j;
    y[e] = fmaxf(fmaxf(__ldg(s), __ldg(s + 1)), fmaxf(__ldg(s + W), __ldg(s + W + 1)));
  }
}

// source row of output row p: s = (p + 1/2) / 2 - 1/2 = p / 2 - 1/4 (exact in
// fp32), clamped at 0; the next row clamped at the last
__device__ __forceinline__ void up_src(int p, int n, int &i0, int &i1, float &f) {
  const float s = fmaxf(0.5f * (float)p - 0.25f, 0.f);
  i0 = (int)s;
  i1 = i0 + 1 < n ? i0 + 1 : n - 1;
  f = s - (float)i0;
}

__global__ void unet_upsample2_kernel(const float *x, int NC, int H, int W, float *y) {
  const int Ho = 2 * H, Wo = 2 * W;
  const size_t total = (size_t)NC * Ho * Wo;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t nc = e / ((size_t)Ho * Wo);
    const int r = (int)(e - nc * Ho * Wo), p = r / Wo, q = r - (r / Wo) * Wo;
    int i0, i1, j0, j1;
    float fi, fj;
    up_src(p, H, i0, i1, fi);
    up_src(q, W, j0, j1, fj);
    const float *s = x + nc * H * W;
    const float top = (1.f - fj) * __ldg(s + (size_t)i0 * W + j0) + fj * __ldg(s + (size_t)i0 * W + j1);
    const float bot = (1.f - fj) * __ldg(s + (size_t)i1 * W + j0) + fj * __ldg(s + (size_t)i1 * W + j1);
    y[e] = (1.f - fi) * top + fi * bot;
  }
}

__global__ void unet_head_kernel(const float *d, int N, int C, int HW, const float *wh, const float *bh, int Cout,
                                 float *out) {
  const size_t total = (size_t)N * HW;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t n = e / HW, px = e - n * HW;
    const float *dp = d + n * C * HW + px;
    for (int o = 0; o < Cout; ++o) {
      float acc = __ldg(bh + o);
      for (int c = 0; c < C; ++c) acc = fmaf(__ldg(wh + (size_t)o * C + c), __ldg(dp + (size_t)c * HW), acc);
      out[(n * Cout + o) * HW + px] = fmaxf(acc, 0.f);
    }
  }
}

// ---- tensor-core form: NHWC helpers (one thread per 4 channels of an
// output pixel, or per pixel) ----

__global__ void unet_stage_nhwc_kernel(const float *in, int N, int cin, long long hw, int cs, float *out) {
  const long long total = (long long)N * hw;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long n = g / hw, p = g - n * hw;
    const float *src = in + n * cin * hw + p;
    float4 *dst = reinterpret_cast<float4 *>(out + g * cs);
    for (int q = 0; q < cs / 4; ++q) {
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = 4 * q + e < cin ? __ldg(src + (4 * q + e) * hw) : 0.f;
      dst[q] = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

__global__ void unet_pool_nhwc_kernel(const float4 *x, int N, int H, int W, int C4, float4 *y) {
  const int Ho = H / 2, Wo = W / 2;
  const long long total = (long long)N * Ho * Wo * C4;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long pix = e / C4;
    const int c4 = (int)(e - pix * C4);
    const long long n = pix / ((long long)Ho * Wo);
    const int r = (int)(pix - n * Ho * Wo), i = r / Wo, j = r - (r / Wo) * Wo;
    const float4 *s = x + ((n * H + 2 * i) * W + 2 * j) * C4 + c4;
    const float4 a = __ldg(s), b = __ldg(s + C4), c = __ldg(s + (size_t)W * C4), d = __ldg(s + (size_t)W * C4 + C4);
    y[e] = make_float4(fmaxf(fmaxf(a.x, b.x), fmaxf(c.x, d.x)), fmaxf(fmaxf(a.y, b.y), fmaxf(c.y, d.y)),
                       fmaxf(fmaxf(a.z, b.z), fmaxf(c.z, d.z)), fmaxf(fmaxf(a.w, b.w), fmaxf(c.w, d.w)));
  }
}

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float f) {
  return make_float4((1.f - f) * a.x + f * b.x, (1.f - f) * a.y + f * b.y, (1.f - f) * a.z + f * b.z,
                     (1.f - f) * a.w + f * b.w);
}

__global__ void unet_up_nhwc_kernel(const float4 *x, int N, int h, int w, int C4, float4 *y) {
  const int Ho = 2 * h, Wo = 2 * w;
  const long long total = (long long)N * Ho * Wo * C4;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long pix = e / C4;
    const int c4 = (int)(e - pix * C4);
    const long long n = pix / ((long long)Ho * Wo);
    const int r = (int)(pix - n * Ho * Wo), p = r / Wo, q = r - (r / Wo) * Wo;
    int i0, i1, j0, j1;
    float fi, fj;
    up_src(p, h, i0, i1, fi);
    up_src(q, w, j0, j1, fj);
    const float4 *s = x + n * h * w * C4 + c4;
    const float4 top = lerp4(__ldg(s + ((size_t)i0 * w + j0) * C4), __ldg(s + ((size_t)i0 * w + j1) * C4), fj);
    const float4 bot = lerp4(__ldg(s + ((size_t)i1 * w + j0) * C4), __ldg(s + ((size_t)i1 * w + j1) * C4), fj);
    y[e] = lerp4(top, bot, fi);
  }
}

// Output channels in groups of four, each group one pass over the pixel's C
// channels (C a multiple of 4).
__global__ void unet_head_nhwc_kernel(const float *d, int N, long long hw, int C, const float *wh, const float *bh,
                                      int cout, float *out) {
  const long long total = (long long)N * hw;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long n = g / hw, p = g - n * hw;
    const float4 *dp = reinterpret_cast<const float4 *>(d + g * C);
    for (int o0 = 0; o0 < cout; o0 += 4) {
      float acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = o0 + q < cout ? __ldg(bh + o0 + q) : 0.f;
      for (int c4 = 0; c4 < C / 4; ++c4) {
        const float4 v = __ldg(dp + c4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (o0 + q >= cout) break;
          const float *wr = wh + (size_t)(o0 + q) * C + 4 * c4;
          acc[q] = fmaf(__ldg(wr), v.x, acc[q]);
          acc[q] = fmaf(__ldg(wr + 1), v.y, acc[q]);
          acc[q] = fmaf(__ldg(wr + 2), v.z, acc[q]);
          acc[q] = fmaf(__ldg(wr + 3), v.w, acc[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (o0 + q < cout) out[(n * cout + o0 + q) * hw + p] = fmaxf(acc[q], 0.f);
    }
  }
}

unsigned grid_for(size_t work) {
  size_t g = (work + 255) / 256;
  if (g < 1) g = 1;
  if (g > 8192) g = 8192;
  return (unsigned)g;
}

cudaError_t conv_launch(const float *x1, int C1, const float *x2, int C2, int N, int H, int W, const float *F,
                        const LayerDesc &L, float *y, cudaStream_t st, Tracer *tr) {
  const int TH = H < 16 ? H : 16, TW = W < 16 ? W : 16, P = TH * TW;
  int MPB = UTHREADS / P;
  if (MPB > UMPB_MAX) MPB = UMPB_MAX;
  if (MPB < 1 || UCC * MPB * (TH + 2) * (TW + 2) > UXS_MAX) return cudaErrorInvalidValue;
  const int tiles_x = (W + TW - 1) / TW, tiles_y = (H + TH - 1) / TH;
  const unsigned gz = (unsigned)((N + MPB - 1) / MPB);
  if (gz > 65535u) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)(tiles_x * tiles_y), (unsigned)((L.cout + UCOB - 1) / UCOB), gz);
  const float *wr = F + L.dst, *bias = wr + 9 * (size_t)L.cin * L.cout;
  DRC_TRACED(tr, "unet conv", st,
             (unet_conv3x3_kernel<<<grid, UTHREADS, 0, st>>>(x1, C1, x2, C2, N, H, W, wr, bias, L.cout, kLreluSlope,
                                                             y, TH, TW, MPB, tiles_x)));
  return cudaGetLastError();
}

}  // namespace

size_t unet_param_count(const UnetShape &u) {
  size_t n = 0;
  unet_layers(u, &n, nullptr);
  return n;
}

size_t unet_workspace_bytes(const UnetShape &u, int N, int H, int W) { return unet_carve(u, N, H, W, nullptr, nullptr); }

cudaError_t unet_forward(const UnetShape &u, const float *params, const float *in, float *out, int N, int H, int W,
                         void *workspace, cudaStream_t st, Tracer *tr) {
  const std::vector<LayerDesc> L = unet_layers(u, nullptr, nullptr);
  UnetBufs b;
  unet_carve(u, N, H, W, static_cast<char *>(workspace), &b);
  cudaError_t e;
  for (const LayerDesc &d : L) {
    const size_t work = (d.kind == 2 ? 1 : 9) * (size_t)d.cin * d.cout + d.cout;
    DRC_TRACED(tr, "unet fold", st,
               (unet_fold_kernel<false><<<grid_for(work), 256, 0, st>>>(params, d.kind, d.cin, d.cout, d.bn, d.src,
                                                                        d.dst, b.fold)));
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  size_t li = 0;
  const float *x = in;
  int ci = u.cin;
  for (int l = 0; l <= u.levels; ++l) {
    const int h = H >> l, w = W >> l, c = u.base << l;
    if (l > 0) {
      const int ph = H >> (l - 1), pw = W >> (l - 1);
      const size_t work = (size_t)N * ci * h * w;
      DRC_TRACED(tr, "unet pool", st,
                 (unet_maxpool2_kernel<<<grid_for(work), 256, 0, st>>>(b.enc[l - 1], N * ci, ph, pw, b.pool[l])));
      x = b.pool[l];
    }
    if ((e = conv_launch(x, ci, nullptr, 0, N, h, w, b.fold, L[li++], b.enc_a[l], st, tr)) != cudaSuccess) return e;
    if ((e = conv_launch(b.enc_a[l], c, nullptr, 0, N, h, w, b.fold, L[li++], b.enc[l], st, tr)) != cudaSuccess)
      return e;
    ci = c;
  }
  const float *d = b.enc[u.levels];
  for (int l = u.levels - 1; l >= 0; --l) {
    const int h = H >> l, w = W >> l, c = u.base << l;
    const size_t work = (size_t)N * 2 * c * h * w;
    DRC_TRACED(tr, "unet up", st,
               (unet_upsample2_kernel<<<grid_for(work), 256, 0, st>>>(d, N * 2 * c, h / 2, w / 2, b.up[l])));
    if ((e = conv_launch(b.up[l], 2 * c, b.enc[l], c, N, h, w, b.fold, L[li++], b.dec_a[l], st, tr)) != cudaSuccess)
      return e;
    if ((e = conv_launch(b.dec_a[l], c, nullptr, 0, N, h, w, b.fold, L[li++], b.dec[l], st, tr)) != cudaSuccess)
      return e;
    d = b.dec[l];
  }
  const LayerDesc &hd = L[li];
  const float *wh = b.fold + hd.dst, *bh = wh + (size_t)hd.cin * hd.cout;
  DRC_TRACED(tr, "unet head", st,
             (unet_head_kernel<<<grid_for((size_t)N * H * W), 256, 0, st>>>(d, N, u.base, H * W, wh, bh, u.cout,
                                                                           out)));
  return cudaGetLastError();
}

std::vector<UnetLayer> unet_layer_table(const UnetShape &u) { return unet_layers(u, nullptr, nullptr); }

int unet_tc_in_channels(const UnetShape &u) { return u.cin <= 8 ? 8 : u.cin; }

bool unet_tc_shape_ok(const UnetShape &u, int H, int W) {
  if (u.base % 32 || (u.cin > 8 && u.cin % 32)) return false;
  for (int l = 0; l <= u.levels; ++l) {
    const int h = H >> l, w = W >> l;
    if (h < 1 || w < 1 || w > 128 || 128 % w) return false;
    const int rows_t = h < 128 / w ? h : 128 / w;
    if (rows_t < h ? h % rows_t != 0 : 128 % (h * w) != 0) return false;
  }
  return true;
}

size_t unet_tc_pack_bytes(int cin_stored, int cout) {
  const size_t kb = (9 * (size_t)cin_stored + 31) / 32;  // K blocks of 32 tf32 elements (128 bytes)
  return kb * (size_t)cout * 128;
}

size_t unet_tc_carve(const UnetShape &u, int N, int H, int W, char *base, UnetTcBufs *b) {
  size_t n_dst = 0;
  const std::vector<LayerDesc> L = unet_layers(u, nullptr, &n_dst);
  size_t pack = 0;
  for (const LayerDesc &d : L)
    if (d.kind != 2) pack += align256(unet_tc_pack_bytes(&d == &L[0] ? unet_tc_in_channels(u) : d.cin, d.cout));
  size_t off = 0;
  auto take = [&](size_t bytes) -> char * {
    char *p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  auto takef = [&](size_t floats) { return reinterpret_cast<float *>(take(floats * sizeof(float))); };
  UnetTcBufs t;
  t.fold = takef(n_dst);
  t.B = reinterpret_cast<uint8_t *>(take(pack));
  t.B_lo = reinterpret_cast<uint8_t *>(take(pack));
  t.in = takef((size_t)N * H * W * unet_tc_in_channels(u));
  for (int l = 0; l <= u.levels; ++l) {
    const size_t px = (size_t)N * (H >> l) * (W >> l);
    const size_t c = (size_t)u.base << l;
    t.enc_a[l] = takef(px * c);
    t.enc[l] = takef(px * c);
    if (l > 0) t.pool[l] = takef(px * (c / 2));
    if (l < u.levels) {
      t.up[l] = takef(px * 2 * c);
      t.dec_a[l] = takef(px * c);
      t.dec[l] = takef(px * c);
    }
  }
  if (b) *b = t;
  return off;
}

cudaError_t unet_fold_conv_form(const UnetShape &u, const float *params, float *fold, cudaStream_t st, Tracer *tr) {
  for (const LayerDesc &d : unet_layers(u, nullptr, nullptr)) {
    const size_t work = (d.kind == 2 ? 1 : 9) * (size_t)d.cin * d.cout + d.cout;
    DRC_TRACED(tr, "unet fold", st,
               (unet_fold_kernel<true><<<grid_for(work), 256, 0, st>>>(params, d.kind, d.cin, d.cout, d.bn, d.src,
                                                                       d.dst, fold)));
  }
  return cudaGetLastError();
}

cudaError_t launch_unet_stage_nhwc(const float *in, int N, int cin, long long hw, int cs, float *out,
                                   cudaStream_t st, Tracer *tr) {
  DRC_TRACED(tr, "unet stage input", st,
             (unet_stage_nhwc_kernel<<<grid_for((size_t)N * hw), 256, 0, st>>>(in, N, cin, hw, cs, out)));
  return cudaGetLastError();
}

cudaError_t launch_unet_pool_nhwc(const float *x, int N, int H, int W, int C, float *y, cudaStream_t st, Tracer *tr) {
  const size_t work = (size_t)N * (H / 2) * (W / 2) * (C / 4);
  DRC_TRACED(tr, "unet pool", st,
             (unet_pool_nhwc_kernel<<<grid_for(work), 256, 0, st>>>(reinterpret_cast<const float4 *>(x), N, H, W,
                                                                    C / 4, reinterpret_cast<float4 *>(y))));
  return cudaGetLastError();
}

cudaError_t launch_unet_up_nhwc(const float *x, int N, int h, int w, int C, float *y, cudaStream_t st, Tracer *tr) {
  const size_t work = (size_t)N * (2 * h) * (2 * w) * (C / 4);
  DRC_TRACED(tr, "unet up", st,
             (unet_up_nhwc_kernel<<<grid_for(work), 256, 0, st>>>(reinterpret_cast<const float4 *>(x), N, h, w, C / 4,
                                                                  reinterpret_cast<float4 *>(y))));
  return cudaGetLastError();
}

cudaError_t launch_unet_head_nhwc(const float *d, int N, long long hw, int C, const float *wh, int cout, float *out,
                                  cudaStream_t st, Tracer *tr) {
  const float *bh = wh + (size_t)cout * C;
  DRC_TRACED(tr, "unet head", st,
             (unet_head_nhwc_kernel<<<grid_for((size_t)N * hw), 256, 0, st>>>(d, N, hw, C, wh, bh, cout, out)));
  return cudaGetLastError();
}

}  // namespace drc
