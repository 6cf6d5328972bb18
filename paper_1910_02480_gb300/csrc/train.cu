// train.cu -- training-loop kernels (Sec. 4, Implementation).
//
// augment_kernel: the paper augments its training pairs with combinations
// of rotation and flipping of the maps.  Read here as the eight symmetries of
// the square map (the same one for every channel of a map, and for the input
// and target of a pair): code = r + 4 f, a column mirror if f, then r
// counter-clockwise quarter turns, one turn being b[i][j] = a[j][S - 1 - i].
// Output (i, j) reads its source by undoing the turns, (i, j) -> (j, S - 1 -
// i) once per turn, then the mirror, j -> S - 1 - j.  One block per map
// plane: the plane is read into shared memory in rows (coalesced) and written
// out in rows from its permuted position; planes too large for the block's
// shared memory are gathered straight from global memory.
//
// adam_kernel: Adam (Kingma & Ba 2015, Alg. 1), the optimiser the paper
// trains with (PyTorch's, lr = 6e-5): m = b1 m + (1 - b1) g, v = b2 v +
// (1 - b2) g^2, w -= lr (m c1) / (sqrt(v) c2 + eps) with the bias
// corrections c1 = 1 / (1 - b1^t), c2 = 1 / sqrt(1 - b2^t).  Bound by HBM:
// 16 bytes read and 12 written per parameter, four parameters per thread
// through 16-byte accesses where the arrays allow.
#include <cuda_runtime.h>

#include <cstdint>

#include "train.cuh"

namespace drc {

constexpr int AUG_THREADS = 256;
constexpr int AUG_SMEM_MAX = 64 * 65;  // floats: a 64 x 64 plane with one pad column

__device__ __forceinline__ void aug_source(int code, int S, int i, int j, int &si, int &sj) {
  si = i;
  sj = j;
  for (int q = 0; q < (code & 3); ++q) {
    const int t = si;
    si = sj;
    sj = S - 1 - t;
  }
  if (code & 4) sj = S - 1 - sj;
}

__global__ void __launch_bounds__(AUG_THREADS) augment_kernel(const float *in, float *out, int C, int S,
                                                              const int *codes) {
  __shared__ float tile[AUG_SMEM_MAX];
  const int plane = blockIdx.x;  // n * C + c
  const int code = __ldg(codes + plane / C) & 7;
  const size_t base = (size_t)plane * S * S;
  const float *src = in + base;
  float *dst = out + base;
  const int P = S * S;
  if (S * (S + 1) <= AUG_SMEM_MAX) {
    for (int e = threadIdx.x; e < P; e += AUG_THREADS) {
      const int i = e / S, j = e - i * S;
      tile[i * (S + 1) + j] = __ldg(src + e);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < P; e += AUG_THREADS) {
      const int i = e / S, j = e - i * S;
      int si, sj;
      aug_source(code, S, i, j, si, sj);
      dst[e] = tile[si * (S + 1) + sj];
    }
  } else {
    for (int e = threadIdx.x; e < P; e += AUG_THREADS) {
      const int i = e / S, j = e - i * S;
      int si, sj;
      aug_source(code, S, i, j, si, sj);
      dst[e] = __ldg(src + (size_t)si * S + sj);
    }
  }
}

cudaError_t launch_augment(const float *in, float *out, int N, int C, int S, const int *codes, cudaStream_t st,
                           Tracer *tr) {
  const long long planes = (long long)N * C;
  if (planes == 0) return cudaSuccess;
  DRC_TRACED(tr, "augment", st, (augment_kernel<<<(unsigned)planes, AUG_THREADS, 0, st>>>(in, out, C, S, codes)));
  return cudaGetLastError();
}

__device__ __forceinline__ float adam_one(float &w, float g, float &m, float &v, float lr, float b1, float b2,
                                          float eps, float c1, float c2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  w = w - lr * (m * c1) / (sqrtf(v) * c2 + eps);
  return w;
}

__global__ void adam_kernel(float *w, const float *g, float *m, float *v, size_t n, bool vec, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t done = 0;
  if (vec) {
    const size_t n4 = n / 4;
    for (size_t q = i; q < n4; q += stride) {
      float4 W = reinterpret_cast<float4 *>(w)[q], M = reinterpret_cast<float4 *>(m)[q];
      float4 V = reinterpret_cast<float4 *>(v)[q];
      const float4 G = __ldg(reinterpret_cast<const float4 *>(g) + q);
      adam_one(W.x, G.x, M.x, V.x, lr, b1, b2, eps, c1, c2);
      adam_one(W.y, G.y, M.y, V.y, lr, b1, b2, eps, c1, c2);
      adam_one(W.z, G.z, M.z, V.z, lr, b1, b2, eps, c1, c2);
      adam_one(W.w, G.w, M.w, V.w, lr, b1, b2, eps, c1, c2);
      reinterpret_cast<float4 *>(w)[q] = W;
      reinterpret_cast<float4 *>(m)[q] = M;
      reinterpret_cast<float4 *>(v)[q] = V;
    }
    done = n4 * 4;
  }
  for (size_t k = done + i; k < n; k += stride) {
    float W = w[k], M = m[k], V = v[k];
    adam_one(W, __ldg(g + k), M, V, lr, b1, b2, eps, c1, c2);
    w[k] = W;
    m[k] = M;
    v[k] = V;
  }
}

cudaError_t launch_adam(float *w, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st, Tracer *tr) {
  if (n == 0) return cudaSuccess;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const auto aligned = [](const void *p) { return ((uintptr_t)p & 15) == 0; };  // the C ABI asks for it
  const bool vec = aligned(w) && aligned(g) && aligned(m) && aligned(v);
  const size_t work = vec ? (n + 3) / 4 : n;
  size_t blocks = (work + 255) / 256;
  const size_t cap = (size_t)sms * 8;  // grid-stride beyond eight blocks per SM
  if (blocks > cap) blocks = cap;
  DRC_TRACED(tr, "adam", st,
             (adam_kernel<<<(unsigned)blocks, 256, 0, st>>>(w, g, m, v, n, vec, lr, b1, b2, eps, c1, c2)));
  return cudaGetLastError();
}

}  // namespace drc
