// interp.cu -- radiance-cache interpolation of Sec. 3.2 on the GPU.
//
// 1. A uniform grid over the cache points (3-D first-hit positions for the
//    WORLD metric, integer pixel coordinates for the IMAGE metric) is built by
//    counting sort: bounds -> per-cell counts -> prefix sum -> scatter into a
//    cell-ordered float4 table (x, y, z, index).
// 2. One thread per pixel searches Chebyshev rings of cells around its own
//    cell, keeping the k best (d^2, index) in registers, and stops once the
//    k-th distance is below the distance to every unsearched cell: the
//    selection is exact (the same set as a brute-force scan).
// 3. Weights w = w_p w_n + w_p + eps (Eq. 4), normalised (Sec. 3.2), blend of
//    the payloads (IRRADIANCE) or of bilinear lat-long lookups of the cached
//    maps in each cache's frame (LOOKUP).
#include <cuda_runtime.h>

#include <cfloat>
#include <climits>

#include "interp.cuh"

namespace drc {

static constexpr int METRIC_IMAGE = 0;
static constexpr int WP_INVERSE = 0;
static constexpr int MODE_IRRADIANCE = 0;

static inline int per_cell(int k) { return k / 2 > 1 ? k / 2 : 1; }

int interp_max_cells(int n, int k) {
  const int pc = per_cell(k);
  return 2 * ((n + pc - 1) / pc) + 8;
}

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t interp_scratch_bytes(int n, int k) {
  const size_t mc = (size_t)interp_max_cells(n, k);
  return align256(sizeof(GridHeader)) + align256(mc * sizeof(int)) + align256((mc + 1) * sizeof(int)) +
         align256((size_t)n * sizeof(int)) + align256((size_t)n * sizeof(float4));
}

InterpScratch interp_carve(void *base, int n, int k) {
  InterpScratch s;
  const size_t mc = (size_t)interp_max_cells(n, k);
  char *p = static_cast<char *>(base);
  s.hdr = reinterpret_cast<GridHeader *>(p);
  p += align256(sizeof(GridHeader));
  s.cell_count = reinterpret_cast<int *>(p);
  p += align256(mc * sizeof(int));
  s.cell_start = reinterpret_cast<int *>(p);
  p += align256((mc + 1) * sizeof(int));
  s.cache_cell = reinterpret_cast<int *>(p);
  p += align256((size_t)n * sizeof(int));
  s.pts = reinterpret_cast<float4 *>(p);
  s.max_cells = (int)mc;
  return s;
}

__device__ __forceinline__ float3 cache_point(const InterpArgs &a, int j) {
  if (a.metric == METRIC_IMAGE) return make_float3((float)a.cpix[2 * j], (float)a.cpix[2 * j + 1], 0.f);
  return make_float3(a.cpos[3 * j], a.cpos[3 * j + 1], a.cpos[3 * j + 2]);
}

__device__ __forceinline__ int cell_of(const GridHeader &g, float3 p, int3 *cc) {
  int c[3];
  const float pv[3] = {p.x, p.y, p.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int v = (int)floorf((pv[d] - g.origin[d]) * g.inv_h);
    v = v < 0 ? 0 : (v >= g.dims[d] ? g.dims[d] - 1 : v);
    c[d] = v;
  }
  if (cc) *cc = make_int3(c[0], c[1], c[2]);
  return (c[2] * g.dims[1] + c[1]) * g.dims[0] + c[0];
}

// Single block: bounds of the cache points, cubic cells sized for about
// k/2 caches each over the occupied axes, counts cleared.
__global__ void grid_bounds_kernel(InterpArgs a, InterpScratch s) {
  __shared__ float slo[3][32], shi[3][32];
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int j = threadIdx.x; j < a.n; j += blockDim.x) {
    const float3 p = cache_point(a, j);
    lo[0] = fminf(lo[0], p.x);
    lo[1] = fminf(lo[1], p.y);
    lo[2] = fminf(lo[2], p.z);
    hi[0] = fmaxf(hi[0], p.x);
    hi[1] = fmaxf(hi[1], p.y);
    hi[2] = fmaxf(hi[2], p.z);
  }
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
    for (int d = 0; d < 3; ++d) {
      slo[d][w] = lo[d];
      shi[d][w] = hi[d];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    float L[3], Hh[3];
    for (int d = 0; d < 3; ++d) {
      L[d] = slo[d][0];
      Hh[d] = shi[d][0];
      for (int q = 1; q < nw; ++q) {
        L[d] = fminf(L[d], slo[d][q]);
        Hh[d] = fmaxf(Hh[d], shi[d][q]);
      }
    }
    float ext[3];
    int active = 0;
    double vol = 1.0;
    for (int d = 0; d < 3; ++d) {
      ext[d] = Hh[d] - L[d];
      if (ext[d] > 0.f) {
        ++active;
        vol *= (double)ext[d];
      }
    }
    const int pc = a.k / 2 > 1 ? a.k / 2 : 1;
    const double target = (double)((a.n + pc - 1) / pc);
    double h = active ? pow(vol / target, 1.0 / active) : 1.0;
    if (!(h > 0.0)) h = 1.0;
    GridHeader g;
    for (;;) {
      long long prod = 1;
      for (int d = 0; d < 3; ++d) {
        int nd = ext[d] > 0.f ? (int)ceil((double)ext[d] / h) : 1;
        if (nd < 1) nd = 1;
        g.dims[d] = nd;
        prod *= nd;
      }
      if (prod <= s.max_cells) {
        g.ncells = (int)prod;
        break;
      }
      h *= 1.125;
    }
    for (int d = 0; d < 3; ++d) g.origin[d] = L[d];
    g.h = (float)h;
    g.inv_h = (float)(1.0 / h);
    g.pad_ = 0;
    *s.hdr = g;
  }
  for (int c = threadIdx.x; c < s.max_cells; c += blockDim.x) s.cell_count[c] = 0;
}

__global__ void grid_count_kernel(InterpArgs a, InterpScratch s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  const GridHeader g = *s.hdr;
  const int c = cell_of(g, cache_point(a, j), nullptr);
  s.cache_cell[j] = c;
  atomicAdd(&s.cell_count[c], 1);
}

// Single block exclusive scan of the cell counts; counts become cursors.
__global__ void grid_scan_kernel(InterpScratch s) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  const int nc = s.hdr->ncells;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nc; base += blockDim.x) {
    const int c = base + threadIdx.x;
    const int v = c < nc ? s.cell_count[c] : 0;
    int x = v;
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (l >= o) x += y;
    }
    if (l == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
      const int nw = blockDim.x >> 5;
      int t = l < nw ? warp_tot[l] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (l >= o) t += y;
      }
      if (l < nw) warp_tot[l] = t;
    }
    __syncthreads();
    const int excl = carry + (w > 0 ? warp_tot[w - 1] : 0) + x - v;
    if (c < nc) {
      s.cell_start[c] = excl;
      s.cell_count[c] = excl;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) s.cell_start[nc] = carry;
}

__global__ void grid_scatter_kernel(InterpArgs a, InterpScratch s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  const int c = s.cache_cell[j];
  const int pos = atomicAdd(&s.cell_count[c], 1);
  const float3 p = cache_point(a, j);
  s.pts[pos] = make_float4(p.x, p.y, p.z, __int_as_float(j));
}

template <int KMAX>
struct TopK {
  float d[KMAX];
  int i[KMAX];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
      d[s] = FLT_MAX;
      i[s] = INT_MAX;
    }
  }
  // insert (dc, ic) keeping ascending (d, i) order
  __device__ __forceinline__ void insert(float dc, int ic) {
#pragma unroll
    for (int s = KMAX - 1; s >= 0; --s) {
      const bool after = d[s] > dc || (d[s] == dc && i[s] > ic);
      if (after) {
        bool prev_after = false;
        if (s > 0) prev_after = d[s - 1] > dc || (d[s - 1] == dc && i[s - 1] > ic);
        if (prev_after) {
          d[s] = d[s - 1];
          i[s] = i[s - 1];
        } else {
          d[s] = dc;
          i[s] = ic;
        }
      }
    }
  }
  __device__ __forceinline__ void kth(int k, float &dk, int &ik) const {
    dk = d[0];
    ik = i[0];
#pragma unroll
    for (int s = 1; s < KMAX; ++s)
      if (s == k - 1) {
        dk = d[s];
        ik = i[s];
      }
  }
};

__device__ __forceinline__ float bilinear_map(const float *R, int H, int W, float ti, float tj) {
  const float fi = floorf(ti), fj = floorf(tj);
  const float ai = ti - fi, aj = tj - fj;
  int i0 = (int)fi, j0 = (int)fj;
  int i1 = i0 + 1, j1 = j0 + 1;
  i0 = i0 < 0 ? 0 : (i0 > H - 1 ? H - 1 : i0);
  i1 = i1 < 0 ? 0 : (i1 > H - 1 ? H - 1 : i1);
  j0 = ((j0 % W) + W) % W;
  j1 = ((j1 % W) + W) % W;
  const float v00 = __ldg(R + i0 * W + j0), v01 = __ldg(R + i0 * W + j1);
  const float v10 = __ldg(R + i1 * W + j0), v11 = __ldg(R + i1 * W + j1);
  return (1.f - ai) * ((1.f - aj) * v00 + aj * v01) + ai * ((1.f - aj) * v10 + aj * v11);
}

template <int KMAX>
__global__ void __launch_bounds__(256, 2) interp_kernel(InterpArgs a, InterpScratch s) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long P = (long long)a.width * a.height;
  if (p >= P) return;
  const GridHeader g = *s.hdr;
  float3 q;
  if (a.metric == METRIC_IMAGE)
    q = make_float3((float)(p % a.width), (float)(p / a.width), 0.f);
  else
    q = make_float3(__ldg(a.gpos + 3 * p), __ldg(a.gpos + 3 * p + 1), __ldg(a.gpos + 3 * p + 2));
  int3 c0;
  cell_of(g, q, &c0);
  TopK<KMAX> top;
  top.init();
  const int k = a.k;
  int found = 0;
  const float margin = 1e-4f * g.h;
  const int maxR = max(g.dims[0], max(g.dims[1], g.dims[2]));
  for (int R = 0; R <= maxR; ++R) {
    const int z0 = max(c0.z - R, 0), z1 = min(c0.z + R, g.dims[2] - 1);
    const int y0 = max(c0.y - R, 0), y1 = min(c0.y + R, g.dims[1] - 1);
    const int x0 = max(c0.x - R, 0), x1 = min(c0.x + R, g.dims[0] - 1);
    for (int cz = z0; cz <= z1; ++cz)
      for (int cy = y0; cy <= y1; ++cy)
        for (int cx = x0; cx <= x1; ++cx) {
          const int cheb = max(abs(cx - c0.x), max(abs(cy - c0.y), abs(cz - c0.z)));
          if (cheb != R) continue;
          const int cell = (cz * g.dims[1] + cy) * g.dims[0] + cx;
          const int e0 = __ldg(s.cell_start + cell), e1 = __ldg(s.cell_start + cell + 1);
          for (int e = e0; e < e1; ++e) {
            const float4 pt = __ldg(s.pts + e);
            const float dx = q.x - pt.x, dy = q.y - pt.y, dz = q.z - pt.z;
            const float d2 = dx * dx + dy * dy + dz * dz;
            const int j = __float_as_int(pt.w);
            ++found;
            float dk;
            int ik;
            top.kth(k, dk, ik);
            if (d2 < dk || (d2 == dk && j < ik)) top.insert(d2, j);
          }
        }
    // stop when every cell is searched, or when the k-th distance is below
    // the distance from q to every unsearched cell
    float bound = FLT_MAX;
    bool all = true;
    const int cc[3] = {c0.x, c0.y, c0.z};
    const float qv[3] = {q.x, q.y, q.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (cc[d] - R > 0) {
        all = false;
        bound = fminf(bound, qv[d] - (g.origin[d] + (float)(cc[d] - R) * g.h));
      }
      if (cc[d] + R < g.dims[d] - 1) {
        all = false;
        bound = fminf(bound, (g.origin[d] + (float)(cc[d] + R + 1) * g.h) - qv[d]);
      }
    }
    if (all) break;
    if (found >= k) {
      float dk;
      int ik;
      top.kth(k, dk, ik);
      const float b = bound - margin;
      if (b > 0.f && dk <= b * b) break;
    }
  }
  const int kk = found < k ? found : k;

  // weights (Eq. 4) and normalisation
  const float pnx = __ldg(a.gnrm + 3 * p), pny = __ldg(a.gnrm + 3 * p + 1), pnz = __ldg(a.gnrm + 3 * p + 2);
  const float pl = sqrtf(pnx * pnx + pny * pny + pnz * pnz);
  float w[KMAX];
  float wsum = 0.f;
#pragma unroll
  for (int t = 0; t < KMAX; ++t) {
    w[t] = 0.f;
    if (t < kk) {
      const int j = top.i[t];
      const float d = sqrtf(top.d[t]);
      const float wp = a.wp_form == WP_INVERSE ? a.r / (d + a.delta_rel * a.r) : fmaxf(0.f, 1.f - d / a.r);
      const float cx = __ldg(a.cnrm + 3 * j), cy = __ldg(a.cnrm + 3 * j + 1), cz = __ldg(a.cnrm + 3 * j + 2);
      const float cl = sqrtf(cx * cx + cy * cy + cz * cz);
      float wn = 0.f;
      if (pl > 0.f && cl > 0.f) wn = fmaxf(0.f, (cx * pnx + cy * pny + cz * pnz) / (cl * pl));
      w[t] = wp * wn + wp + a.eps;
      wsum += w[t];
    }
  }
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  if (a.mode == MODE_IRRADIANCE) {
#pragma unroll
    for (int t = 0; t < KMAX; ++t)
      if (t < kk) {
        const int j = top.i[t];
        const float Wt = w[t] / wsum;
        acc0 += Wt * __ldg(a.payload + 3 * j);
        acc1 += Wt * __ldg(a.payload + 3 * j + 1);
        acc2 += Wt * __ldg(a.payload + 3 * j + 2);
      }
  } else {
    float ox = __ldg(a.gdir + 3 * p), oy = __ldg(a.gdir + 3 * p + 1), oz = __ldg(a.gdir + 3 * p + 2);
    const float ol = sqrtf(ox * ox + oy * oy + oz * oz);
    if (ol > 0.f) {
      ox /= ol;
      oy /= ol;
      oz /= ol;
      const float two_pi = 6.283185307179586f;
      const size_t map_sz = (size_t)a.mapH * a.mapW;
#pragma unroll
      for (int t = 0; t < KMAX; ++t) {
        if (t >= kk) continue;
        const int j = top.i[t];
        float nx = __ldg(a.cnrm + 3 * j), ny = __ldg(a.cnrm + 3 * j + 1), nz = __ldg(a.cnrm + 3 * j + 2);
        const float nl = sqrtf(nx * nx + ny * ny + nz * nz);
        if (!(nl > 0.f)) continue;
        nx /= nl;
        ny /= nl;
        nz /= nl;
        // frame: up = +Z, or +Y when the normal is along Z; t = up x n, b = n x t
        float ux = 0.f, uy = 0.f, uz = 1.f;
        if (fabsf(nz) > 1.f - 1e-6f) {
          uy = 1.f;
          uz = 0.f;
        }
        float tx = uy * nz - uz * ny, ty = uz * nx - ux * nz, tz = ux * ny - uy * nx;
        const float tl = sqrtf(tx * tx + ty * ty + tz * tz);
        tx /= tl;
        ty /= tl;
        tz /= tl;
        const float bx = ny * tz - nz * ty, by = nz * tx - nx * tz, bz = nx * ty - ny * tx;
        const float lx = ox * tx + oy * ty + oz * tz;
        const float ly = ox * bx + oy * by + oz * bz;
        float lz = ox * nx + oy * ny + oz * nz;
        if (!(lz > 0.f)) continue;
        lz = fminf(lz, 1.f);
        const float theta = acosf(lz);
        float phi = atan2f(ly, lx);
        if (phi < 0.f) phi += two_pi;
        const float ti = theta * (2.f / 3.14159265358979f) * (float)a.mapH - 0.5f;
        const float tj = phi * (1.f / two_pi) * (float)a.mapW - 0.5f;
        const float Wt = w[t] / wsum;
        const float *Rj = a.maps + (size_t)j * 3 * map_sz;
        acc0 += Wt * bilinear_map(Rj, a.mapH, a.mapW, ti, tj);
        acc1 += Wt * bilinear_map(Rj + map_sz, a.mapH, a.mapW, ti, tj);
        acc2 += Wt * bilinear_map(Rj + 2 * map_sz, a.mapH, a.mapW, ti, tj);
      }
    }
  }
  a.out[3 * p] = acc0;
  a.out[3 * p + 1] = acc1;
  a.out[3 * p + 2] = acc2;
  if (a.nbr_out) {
#pragma unroll
    for (int t = 0; t < KMAX; ++t)
      if (t < k) a.nbr_out[(size_t)p * k + t] = t < kk ? top.i[t] : -1;
  }
}

cudaError_t launch_interp(const InterpArgs &a, const InterpScratch &s, cudaStream_t st) {
  grid_bounds_kernel<<<1, 1024, 0, st>>>(a, s);
  const int cb = (a.n + 255) / 256;
  grid_count_kernel<<<cb, 256, 0, st>>>(a, s);
  grid_scan_kernel<<<1, 1024, 0, st>>>(s);
  grid_scatter_kernel<<<cb, 256, 0, st>>>(a, s);
  const long long P = (long long)a.width * a.height;
  if (P == 0) return cudaGetLastError();
  const unsigned blocks = (unsigned)((P + 255) / 256);
  if (a.k <= 8)
    interp_kernel<8><<<blocks, 256, 0, st>>>(a, s);
  else if (a.k <= 16)
    interp_kernel<16><<<blocks, 256, 0, st>>>(a, s);
  else
    interp_kernel<32><<<blocks, 256, 0, st>>>(a, s);
  return cudaGetLastError();
}

}  // namespace drc
