// indirect.cu -- the indirect term of Eq. 3 (Sec. 3.2) on the GPU.
//
// At a pixel the indirect radiance is the hemisphere integral of
// f_r cos(theta) R, with R the blend of its k nearest caches' maps by the
// normalised weights of Eq. 4.  The paper estimates it with a few samples,
// alternating between sampling R as an environment map with perfect
// visibility and sampling the BRDF, combined by multiple importance sampling
// (Veach's balance heuristic); the weights serve as map-choice
// probabilities, so the estimate's expectation is the integral of the blend.
//
// Readings (shared with the oracle): a Lambertian BRDF albedo / pi; texel
// (a, b) of a map holds one radiance over polar angles [a, a+1) pi / 2H from
// the cache normal and azimuths [b, b+1) 2 pi / W in the cache frame (up =
// +Z, or +Y when the normal is along Z; t = up x n normalised, b = n x t);
// environment sampling picks a texel with probability proportional to its
// luminance (0.2126 R + 0.7152 G + 0.0722 B) times its solid angle, then a
// direction uniform in solid angle inside it; BRDF sampling is
// cosine-weighted about the pixel normal; sample s takes the environment
// for even s and the BRDF for odd s, and a sample contributes
// f_r cos R / (n_env pdf_env + n_brdf pdf_brdf).  The uniforms are an input,
// u[p][s] = (map choice, three for the direction).
//
// 1. indirect_setup_kernel: one thread per map: its frame and its CDF,
//    summed in row-major order in float32 (the texel choice is taken from
//    these sums, as in the oracle).
// 2. indirect_kernel: one thread per pixel over its S samples; the texel of
//    an environment sample by binary search in the CDF; the result plus the
//    emission and the direct term when given (Eq. 3).
#include <cuda_runtime.h>

#include <cfloat>

#include "indirect.cuh"

namespace drc {

static constexpr int SETUP_THREADS = 128;
static constexpr int IND_THREADS = 256;
static constexpr float kPi = 3.14159265358979f;

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t indirect_scratch_bytes(int n, int H, int W) {
  return align256((size_t)n * H * W * sizeof(float)) + align256((size_t)n * 3 * sizeof(float4));
}

void indirect_carve(IndirectArgs &a, void *base) {
  char *p = static_cast<char *>(base);
  a.cdf = reinterpret_cast<float *>(p);
  p += align256((size_t)a.n * a.H * a.W * sizeof(float));
  a.frame = reinterpret_cast<float4 *>(p);
}

// Frame of a normal: (t, b, n); false for a zero-length normal.
__device__ __forceinline__ bool make_frame(float nx, float ny, float nz, float3 &t, float3 &b, float3 &n) {
  const float len = sqrtf(nx * nx + ny * ny + nz * nz);
  if (!(len > 0.f)) return false;
  n = make_float3(nx / len, ny / len, nz / len);
  float ux = 0.f, uy = 0.f, uz = 1.f;
  if (fabsf(n.z) > 1.f - 1e-6f) {
    uy = 1.f;
    uz = 0.f;
  }
  float cx = uy * n.z - uz * n.y, cy = uz * n.x - ux * n.z, cz = ux * n.y - uy * n.x;
  const float cl = sqrtf(cx * cx + cy * cy + cz * cz);
  t = make_float3(cx / cl, cy / cl, cz / cl);
  b = make_float3(n.y * t.z - n.z * t.y, n.z * t.x - n.x * t.z, n.x * t.y - n.y * t.x);
  return true;
}

__device__ __forceinline__ float lum_of(float r, float g, float b) {
  return __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, r), __fmul_rn(0.7152f, g)), __fmul_rn(0.0722f, b));
}

// One thread per map: its frame and its CDF, summed texel by texel in
// row-major order with separately rounded float32 operations
// (luminance (0.2126 R + 0.7152 G) + 0.0722 B, times the row's solid angle,
// added to the running total).  The texel choice is taken from these sums;
// they are exactly the float32 sums in that order, so the choice is the one
// any float32 evaluation in that order takes.
__global__ void __launch_bounds__(SETUP_THREADS) indirect_setup_kernel(const __grid_constant__ IndirectArgs a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  float3 t, b, n;
  const bool ok = make_frame(__ldg(a.cnrm + 3 * j), __ldg(a.cnrm + 3 * j + 1), __ldg(a.cnrm + 3 * j + 2), t, b, n);
  a.frame[3 * j] = make_float4(t.x, t.y, t.z, 0.f);
  a.frame[3 * j + 1] = make_float4(b.x, b.y, b.z, 0.f);
  a.frame[3 * j + 2] = make_float4(n.x, n.y, n.z, ok ? 1.f : 0.f);
  const size_t plane = (size_t)a.H * a.W;
  const float *R = a.maps + (size_t)j * 3 * plane;
  float *cdf = a.cdf + (size_t)j * plane;
  float acc = 0.f;
  for (int r = 0; r < a.H; ++r) {
    const float om = a.omega[r];
    for (int c = 0; c < a.W; ++c) {
      const size_t e = (size_t)r * a.W + c;
      acc = __fadd_rn(acc, __fmul_rn(lum_of(__ldg(R + e), __ldg(R + plane + e), __ldg(R + 2 * plane + e)), om));
      cdf[e] = acc;
    }
  }
}

// KMAX >= k: the pixel's neighbour list and weights are read once into
// registers (loops over them are unrolled to KMAX with i < k guards), so a
// sample's map choice costs no memory access.
template <int KMAX>
__global__ void __launch_bounds__(IND_THREADS) indirect_kernel(const __grid_constant__ IndirectArgs a) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  float3 tp, bp, np;
  const bool pix_ok =
      make_frame(__ldg(a.gnrm + 3 * p), __ldg(a.gnrm + 3 * p + 1), __ldg(a.gnrm + 3 * p + 2), tp, bp, np);
  const float al0 = __ldg(a.albedo + 3 * p) / kPi, al1 = __ldg(a.albedo + 3 * p + 1) / kPi,
              al2 = __ldg(a.albedo + 3 * p + 2) / kPi;
  const int HW = a.H * a.W;
  const size_t plane = (size_t)HW;
  const float n_env = (float)((a.S + 1) / 2), n_brdf = (float)(a.S / 2);
  const int *nb = a.nbr + p * a.k;
  const float *wb = a.nbr_w + p * a.k;
  int jn[KMAX];
  float wn[KMAX];
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    jn[i] = -1;
    wn[i] = 0.f;
    if (i < a.k) {
      const int ji = __ldg(nb + i);
      jn[i] = ji >= 0 && ji < a.n ? ji : -1;  // no neighbour (an index past n is treated alike)
      wn[i] = __ldg(wb + i);
    }
  }
  for (int s = 0; pix_ok && s < a.S; ++s) {
    const float4 us = __ldg(a.u + p * a.S + s);
    // the map, by the normalised weights (their running float32 sum): the
    // first valid slot whose running sum exceeds u0, else the last valid one
    int j = -1;
    float c = 0.f;
    bool done = false;
#pragma unroll
    for (int i = 0; i < KMAX; ++i) {
      if (!done && jn[i] >= 0) {
        j = jn[i];
        c = __fadd_rn(c, wn[i]);
        done = us.x < c;
      }
    }
    if (j < 0) continue;
    const float4 f2 = __ldg(a.frame + 3 * j + 2);
    if (f2.w == 0.f) continue;
    const float4 f0 = __ldg(a.frame + 3 * j), f1 = __ldg(a.frame + 3 * j + 1);
    const float *cdf = a.cdf + (size_t)j * plane;
    const float total = __ldg(cdf + HW - 1);
    float wx, wy, wz;
    if ((s & 1) == 0) {  // environment: texel by the CDF, direction uniform inside it
      if (!(total > 0.f)) continue;
      const float target = __fmul_rn(us.y, total);
      int lo = 0, hi = HW - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(cdf + mid) > target)
          hi = mid;
        else
          lo = mid + 1;
      }
      const int ta = lo / a.W, tb = lo - ta * a.W;
      const float c0 = a.rowcos[ta], c1 = a.rowcos[ta + 1];
      const float mu = c0 - us.z * (c0 - c1);
      const float sn = sqrtf(fmaxf((1.f - mu) * (1.f + mu), 0.f));
      float sp, cp;
      sincosf(((float)tb + us.w) * (2.f * kPi / (float)a.W), &sp, &cp);
      const float lx = sn * cp, ly = sn * sp;
      wx = lx * f0.x + ly * f1.x + mu * f2.x;
      wy = lx * f0.y + ly * f1.y + mu * f2.y;
      wz = lx * f0.z + ly * f1.z + mu * f2.z;
    } else {  // BRDF: cosine-weighted about the pixel normal
      const float rr = sqrtf(us.y), lz = sqrtf(fmaxf(1.f - us.y, 0.f));
      float sp, cp;
      sincosf(2.f * kPi * us.z, &sp, &cp);
      const float lx = rr * cp, ly = rr * sp;
      wx = lx * tp.x + ly * bp.x + lz * np.x;
      wy = lx * tp.y + ly * bp.y + lz * np.y;
      wz = lx * tp.z + ly * bp.z + lz * np.z;
    }
    const float cosp = wx * np.x + wy * np.y + wz * np.z;
    if (!(cosp > 0.f)) continue;
    // the texel the direction falls in; nothing below the cache's hemisphere
    const float qx = wx * f0.x + wy * f0.y + wz * f0.z;
    const float qy = wx * f1.x + wy * f1.y + wz * f1.z;
    const float qz = wx * f2.x + wy * f2.y + wz * f2.z;
    if (!(qz > 0.f)) continue;
    const float theta = acosf(fminf(qz, 1.f));
    float phi = atan2f(qy, qx);
    if (phi < 0.f) phi += 2.f * kPi;
    const int ta = min(max((int)floorf(theta * (2.f / kPi) * (float)a.H), 0), a.H - 1);
    const int tb = min(max((int)floorf(phi * (1.f / (2.f * kPi)) * (float)a.W), 0), a.W - 1);
    const float *R = a.maps + (size_t)j * 3 * plane + (size_t)ta * a.W + tb;
    const float r0 = __ldg(R), r1 = __ldg(R + plane), r2 = __ldg(R + 2 * plane);
    const float pdf_env = total > 0.f ? lum_of(r0, r1, r2) / total : 0.f;
    const float denom = n_env * pdf_env + n_brdf * cosp / kPi;
    if (!(denom > 0.f)) continue;
    const float g = cosp / denom;
    acc0 += al0 * g * r0;
    acc1 += al1 * g * r1;
    acc2 += al2 * g * r2;
  }
  if (a.emit) {
    acc0 += __ldg(a.emit + 3 * p);
    acc1 += __ldg(a.emit + 3 * p + 1);
    acc2 += __ldg(a.emit + 3 * p + 2);
  }
  if (a.direct) {
    acc0 += __ldg(a.direct + 3 * p);
    acc1 += __ldg(a.direct + 3 * p + 1);
    acc2 += __ldg(a.direct + 3 * p + 2);
  }
  a.out[3 * p] = acc0;
  a.out[3 * p + 1] = acc1;
  a.out[3 * p + 2] = acc2;
}

cudaError_t launch_indirect(const IndirectArgs &a, cudaStream_t st, Tracer *tr) {
  if (a.n > 0)
    DRC_TRACED(tr, "indirect setup", st,
               (indirect_setup_kernel<<<(a.n + SETUP_THREADS - 1) / SETUP_THREADS, SETUP_THREADS, 0, st>>>(a)));
  if (a.P > 0) {
    const unsigned blocks = (unsigned)((a.P + IND_THREADS - 1) / IND_THREADS);
    if (a.k <= 8)
      DRC_TRACED(tr, "indirect estimate", st, (indirect_kernel<8><<<blocks, IND_THREADS, 0, st>>>(a)));
    else if (a.k <= 16)
      DRC_TRACED(tr, "indirect estimate", st, (indirect_kernel<16><<<blocks, IND_THREADS, 0, st>>>(a)));
    else
      DRC_TRACED(tr, "indirect estimate", st, (indirect_kernel<32><<<blocks, IND_THREADS, 0, st>>>(a)));
  }
  return cudaGetLastError();
}

}  // namespace drc
