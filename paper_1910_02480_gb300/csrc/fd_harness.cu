// fd_harness.cu -- a test harness, not a hot path.  The autoencoder of
// Sec. 3.3 (stride-2 convolutions with ReLU, stride-2 transposed
// convolutions with ReLU and skip additions, a transposed-convolution head)
// and its mean L1 loss (Sec. 4), evaluated in FP64 on the GPU by direct
// loops, one thread per output element, NCHW.  Its only use is central
// finite differences of the FP32 gradient of drc_backward on the GPU: FP64
// makes the differences of two nearby losses exact to well below the
// gradient's own rounding.  This is the one place device code computes in
// FP64.
#include <cuda_runtime.h>

#include "fd_harness.cuh"

namespace drc {

namespace {

__global__ void fd_input_kernel(const float *in, long long n, int C, long long hw, int encode, double s,
                                double *x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)((i / hw) % C);
  double v = (double)in[i];
  if (encode && c < 3) v = log1p(s * v);
  x[i] = v;
}

// y[n][o][i][j] = b[o] + sum_c sum_uv W[o][c][u][v] x[n][c][2i+u-1][2j+v-1]
__global__ void fd_conv_kernel(const double *x, int N, int Cin, int H, int W, const double *Wt, const double *b,
                               int Cout, int relu, double *y) {
  const int Ho = H / 2, Wo = W / 2;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)N * Cout * Ho * Wo) return;
  const int j = (int)(idx % Wo), i = (int)((idx / Wo) % Ho), o = (int)((idx / ((long long)Wo * Ho)) % Cout);
  const int n = (int)(idx / ((long long)Wo * Ho * Cout));
  double acc = b[o];
  for (int c = 0; c < Cin; ++c)
    for (int u = 0; u < 3; ++u) {
      const int yy = 2 * i + u - 1;
      if (yy < 0 || yy >= H) continue;
      for (int v = 0; v < 3; ++v) {
        const int xx = 2 * j + v - 1;
        if (xx < 0 || xx >= W) continue;
        acc += Wt[((o * Cin + c) * 3 + u) * 3 + v] * x[(((long long)n * Cin + c) * H + yy) * W + xx];
      }
    }
  y[idx] = relu && acc < 0.0 ? 0.0 : acc;
}

// y[n][o][p][q] = b[o] + sum_c sum over (i, u) with 2i + u - 1 = p and (j, v)
// with 2j + v - 1 = q of W[c][o][u][v] x[n][c][i][j]; then ReLU and + skip.
__global__ void fd_convT_kernel(const double *x, int N, int Cin, int h, int w, const double *Wt, const double *b,
                                int Cout, int relu, const double *skip, double *y) {
  const int Ho = 2 * h, Wo = 2 * w;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)N * Cout * Ho * Wo) return;
  const int q = (int)(idx % Wo), p = (int)((idx / Wo) % Ho), o = (int)((idx / ((long long)Wo * Ho)) % Cout);
  const int n = (int)(idx / ((long long)Wo * Ho * Cout));
  double acc = b[o];
  for (int c = 0; c < Cin; ++c)
    for (int u = 0; u < 3; ++u) {
      const int t = p + 1 - u;
      if (t < 0 || (t & 1) || (t >> 1) >= h) continue;
      const int i = t >> 1;
      for (int v = 0; v < 3; ++v) {
        const int s = q + 1 - v;
        if (s < 0 || (s & 1) || (s >> 1) >= w) continue;
        acc += Wt[((c * Cout + o) * 3 + u) * 3 + v] * x[(((long long)n * Cin + c) * h + i) * w + (s >> 1)];
      }
    }
  if (relu && acc < 0.0) acc = 0.0;
  if (skip) acc += skip[idx];
  y[idx] = acc;
}

__global__ void fd_l1_kernel(const double *out, const float *target, long long n, double inv, double *loss) {
  __shared__ double part[256];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += fabs(out[i] - (double)target[i]);
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, part[0] * inv);
}

unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t fd_loss64(const FdLayer *L, int S, const double *w, const float *in, const float *target, int N,
                      int Cin0, int H, int W, bool encode, float exposure, bool out_relu, double *loss,
                      cudaStream_t st) {
  // activations: the input and e_1..e_S, then the decoder's t_{S-1}..t_1 and the output
  size_t total = (size_t)N * Cin0 * H * W;
  for (int s = 1; s <= S; ++s) total += (size_t)N * L[s - 1].Cout * (H >> s) * (W >> s);
  for (int s = S - 1; s >= 1; --s) total += (size_t)N * L[2 * S - 1 - s].Cout * (H >> s) * (W >> s);
  total += (size_t)N * 3 * H * W;
  double *buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, total * sizeof(double));
  if (e != cudaSuccess) return e;
  double *p = buf;
  double *enc[9] = {};
  enc[0] = p;
  p += (size_t)N * Cin0 * H * W;
  const long long n0 = (long long)N * Cin0 * H * W;
  fd_input_kernel<<<blocks_for(n0), 256, 0, st>>>(in, n0, Cin0, (long long)H * W, encode ? 1 : 0, exposure, enc[0]);
  int C = Cin0;
  for (int s = 1; s <= S; ++s) {
    const FdLayer &l = L[s - 1];
    enc[s] = p;
    p += (size_t)N * l.Cout * (H >> s) * (W >> s);
    fd_conv_kernel<<<blocks_for((long long)N * l.Cout * (H >> s) * (W >> s)), 256, 0, st>>>(
        enc[s - 1], N, C, H >> (s - 1), W >> (s - 1), w + l.w_off, w + l.b_off, l.Cout, 1, enc[s]);
    C = l.Cout;
  }
  const double *t = enc[S];
  for (int s = S; s >= 1; --s) {
    const FdLayer &l = L[2 * S - s];
    double *y = p;
    const long long ny = (long long)N * l.Cout * (H >> (s - 1)) * (W >> (s - 1));
    p += ny;
    const bool head = s == 1;
    fd_convT_kernel<<<blocks_for(ny), 256, 0, st>>>(t, N, l.Cin, H >> s, W >> s, w + l.w_off, w + l.b_off, l.Cout,
                                                    head ? (out_relu ? 1 : 0) : 1, head ? nullptr : enc[s - 1], y);
    t = y;
  }
  const long long nout = (long long)N * 3 * H * W;
  if ((e = cudaMemsetAsync(loss, 0, sizeof(double), st)) == cudaSuccess) {
    fd_l1_kernel<<<256, 256, 0, st>>>(t, target, nout, 1.0 / (double)nout, loss);
    e = cudaGetLastError();
  }
  const cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFree(buf);
  return e != cudaSuccess ? e : e2;
}

}  // namespace drc
