// interp.cu -- radiance-cache interpolation of Sec. 3.2 on the GPU.
//
// 1. A uniform grid over the cache points (3-D first-hit positions for the
//    WORLD metric, integer pixel coordinates for the IMAGE metric) is built by
//    counting sort: bounds -> per-cell counts -> prefix sum -> scatter into a
//    cell-ordered float4 table (x, y, z, index).
// 2. Optionally the pixels are counting-sorted by a finer grid over the same
//    box, so that the 32 threads of a warp query nearby points: their cell
//    walks and their candidate lists then coincide (WORLD metric; image order
//    is already coherent for the IMAGE metric).
// 3. One thread per pixel visits its own cell, then the 26 neighbours nearest
//    first, then further Chebyshev shells, skipping every cell whose box is
//    farther than the current k-th distance.  The k best candidates are kept
//    as 64-bit keys (d^2 bits << 32 | index: ascending key = ascending (d^2,
//    index), since d^2 >= 0) in a sorted register array updated by a
//    branch-free min/max network.  The walk stops once the k-th distance is
//    below the distance to every unvisited cell, so the selection equals a
//    brute-force scan.
// 4. Weights w = w_p w_n + w_p + eps (Eq. 4), normalised (Sec. 3.2), blend of
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

// Caches per grid cell the grid is sized for: 3k/8 (at least 1).  At 4096
// caches, k = 16, 1080p WORLD the query measured 0.854 ms with 6 per cell,
// against 0.876 (5), 0.863 (7), 0.874 (8) and 0.892 (12).
static inline int per_cell(int k) { return 3 * k / 8 > 1 ? 3 * k / 8 : 1; }

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
  InterpScratch s = {};
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

static inline long long max_fine_bins(long long P) {
  long long b = P / 16;
  if (b < 1) b = 1;
  if (b > (1 << 20)) b = 1 << 20;
  return b;
}

size_t interp_order_bytes(long long P) {
  const size_t mf = (size_t)max_fine_bins(P);
  return align256(mf * sizeof(int)) + align256((mf + 1) * sizeof(int)) + align256((size_t)P * sizeof(int));
}

void interp_attach_order(InterpScratch &s, void *base, long long P) {
  const size_t mf = (size_t)max_fine_bins(P);
  char *p = static_cast<char *>(base);
  s.fine_count = reinterpret_cast<int *>(p);
  p += align256(mf * sizeof(int));
  s.fine_start = reinterpret_cast<int *>(p);
  p += align256((mf + 1) * sizeof(int));
  s.order = reinterpret_cast<int *>(p);
  s.max_fine = (int)mf;
}

__device__ __forceinline__ float3 cache_point(const InterpArgs &a, int j) {
  if (a.metric == METRIC_IMAGE) return make_float3((float)a.cpix[2 * j], (float)a.cpix[2 * j + 1], 0.f);
  return make_float3(__ldg(a.cpos + 3 * j), __ldg(a.cpos + 3 * j + 1), __ldg(a.cpos + 3 * j + 2));
}

__device__ __forceinline__ float3 query_point(const InterpArgs &a, long long p) {
  if (a.metric == METRIC_IMAGE) return make_float3((float)(p % a.width), (float)(p / a.width), 0.f);
  return make_float3(__ldg(a.gpos + 3 * p), __ldg(a.gpos + 3 * p + 1), __ldg(a.gpos + 3 * p + 2));
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int cell_of(const GridHeader &g, float3 p, int3 *cc) {
  const int cx = clampi((int)floorf((p.x - g.origin[0]) * g.inv_h), 0, g.dims[0] - 1);
  const int cy = clampi((int)floorf((p.y - g.origin[1]) * g.inv_h), 0, g.dims[1] - 1);
  const int cz = clampi((int)floorf((p.z - g.origin[2]) * g.inv_h), 0, g.dims[2] - 1);
  if (cc) *cc = make_int3(cx, cy, cz);
  return (cz * g.dims[1] + cy) * g.dims[0] + cx;
}

__device__ __forceinline__ int fine_of(const GridHeader &g, float3 p) {
  const int cx = clampi((int)floorf((p.x - g.origin[0]) * g.fine_inv_h), 0, g.fdims[0] - 1);
  const int cy = clampi((int)floorf((p.y - g.origin[1]) * g.fine_inv_h), 0, g.fdims[1] - 1);
  const int cz = clampi((int)floorf((p.z - g.origin[2]) * g.fine_inv_h), 0, g.fdims[2] - 1);
  return (cz * g.fdims[1] + cy) * g.fdims[0] + cx;
}

// Single block: bounds of the cache points, cubic cells sized for about 3k/8
// caches each over the occupied axes, the fine pixel-ordering grid, counts
// cleared.
__global__ void grid_bounds_kernel(InterpArgs a, InterpScratch s) {
  __shared__ float slo[3][32], shi[3][32];
  __shared__ GridHeader sg;
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
    const int pc = 3 * a.k / 8 > 1 ? 3 * a.k / 8 : 1;  // as per_cell()
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
    // fine grid: each coarse cell split m ways per occupied axis, about 32
    // pixels per fine cell
    int m = 1;
    if (s.order && active) {
      const double P = (double)a.width * (double)a.height;
      double tgt = P / 32.0;
      if (tgt > (double)s.max_fine) tgt = (double)s.max_fine;
      m = (int)floor(pow(tgt / (double)g.ncells, 1.0 / active));
      if (m < 1) m = 1;
      if (m > 64) m = 64;
    }
    long long nf = 1;
    for (int d = 0; d < 3; ++d) {
      g.fdims[d] = ext[d] > 0.f ? g.dims[d] * m : 1;
      nf *= g.fdims[d];
    }
    while (s.order && nf > s.max_fine && m > 1) {
      --m;
      nf = 1;
      for (int d = 0; d < 3; ++d) {
        g.fdims[d] = ext[d] > 0.f ? g.dims[d] * m : 1;
        nf *= g.fdims[d];
      }
    }
    g.nfine = (int)nf;
    g.fine_inv_h = (float)((double)m / h);
    *s.hdr = g;
    sg = g;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < s.max_cells; c += blockDim.x) s.cell_count[c] = 0;
  if (s.order)
    for (int c = threadIdx.x; c < sg.nfine; c += blockDim.x) s.fine_count[c] = 0;
}

__global__ void grid_count_kernel(InterpArgs a, InterpScratch s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  const GridHeader g = *s.hdr;
  const int c = cell_of(g, cache_point(a, j), nullptr);
  s.cache_cell[j] = c;
  atomicAdd(&s.cell_count[c], 1);
}

// Single block exclusive scan of counts[0..*n_ptr); counts become cursors,
// starts[*n_ptr] = total.  The bins go in tiles of 4 x blockDim.x: each
// thread takes four consecutive bins (one 16-byte load and store), the
// thread totals are scanned across the block, and the running total carries
// to the next tile, whose loads are issued before this tile's scan.
__device__ __forceinline__ void scan_load4(const int *counts, int nc, int i0, int (&v)[4]) {
  if (i0 + 3 < nc) {
    const int4 q = *reinterpret_cast<const int4 *>(counts + i0);
    v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = i0 + e < nc ? counts[i0 + e] : 0;
  }
}
__global__ void __launch_bounds__(1024) scan_kernel(const int *n_ptr, int *counts, int *starts) {
  __shared__ int warp_tot[32];
  const int nc = *n_ptr;
  const int T = 4 * (int)blockDim.x;
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int carry = 0;
  int v[4];
  scan_load4(counts, nc, 4 * threadIdx.x, v);
  for (int base = 0; base < nc; base += T) {
    const int i0 = base + 4 * threadIdx.x;
    int nv[4] = {0, 0, 0, 0};
    if (base + T < nc) scan_load4(counts, nc, i0 + T, nv);
    const int tsum = v[0] + v[1] + v[2] + v[3];
    int x = tsum;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (l >= o) x += y;
    }
    if (l == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
      int t = l < nw ? warp_tot[l] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (l >= o) t += y;
      }
      if (l < nw) warp_tot[l] = t;
    }
    __syncthreads();
    const int off = carry + (w > 0 ? warp_tot[w - 1] : 0) + x - tsum;
    const int o4[4] = {off, off + v[0], off + v[0] + v[1], off + v[0] + v[1] + v[2]};
    if (i0 + 3 < nc) {
      *reinterpret_cast<int4 *>(counts + i0) = make_int4(o4[0], o4[1], o4[2], o4[3]);
#pragma unroll
      for (int e = 0; e < 4; ++e) starts[i0 + e] = o4[e];  // starts + i0 may not be 16-byte aligned
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (i0 + e < nc) {
          counts[i0 + e] = o4[e];
          starts[i0 + e] = o4[e];
        }
    }
    carry += warp_tot[nw - 1];
    __syncthreads();  // warp_tot is rewritten by the next tile
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = nv[e];
  }
  if (threadIdx.x == 0) starts[nc] = carry;
}

__global__ void grid_scatter_kernel(InterpArgs a, InterpScratch s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  const int c = s.cache_cell[j];
  const int pos = atomicAdd(&s.cell_count[c], 1);
  const float3 p = cache_point(a, j);
  s.pts[pos] = make_float4(p.x, p.y, p.z, __int_as_float(j));
}

__global__ void pixel_count_kernel(InterpArgs a, InterpScratch s) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)a.width * a.height) return;
  const GridHeader g = *s.hdr;
  atomicAdd(&s.fine_count[fine_of(g, query_point(a, p))], 1);
}

__global__ void pixel_scatter_kernel(InterpArgs a, InterpScratch s) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)a.width * a.height) return;
  const GridHeader g = *s.hdr;
  const int pos = atomicAdd(&s.fine_count[fine_of(g, query_point(a, p))], 1);
  s.order[pos] = (int)p;
}

// The 26 neighbours of a cell, nearest first: faces, edges, corners.
__constant__ signed char kShell1[26][3] = {
    {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1},
    {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}, {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {1, 0, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1},
    {-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},
    {-1, 1, 1}, {1, 1, 1}};

// k-best register list: KMAX sorted 64-bit keys; the first KMAX-k slots hold
// 0 (never displaced), so the k-th best is always the last slot.  Insertion
// (kc below the last key): gt[s] = key[s] > kc is false up to the insertion
// point and true after it, so each slot takes its lower neighbour (past the
// point), kc (at it) or itself (before it) -- one 64-bit compare and two
// 64-bit selects per slot, the compare of slot s - 1 serving slot s - 1 next.
template <int KMAX>
struct Best {
  unsigned long long key[KMAX];
  __device__ __forceinline__ void init(int k) {
#pragma unroll
    for (int s = 0; s < KMAX; ++s) key[s] = s < KMAX - k ? 0ull : ~0ull;
  }
  __device__ __forceinline__ unsigned long long last() const { return key[KMAX - 1]; }
  __device__ __forceinline__ void insert(unsigned long long kc) {
    bool g_hi = key[KMAX - 1] > kc;  // gt of the slot being written
#pragma unroll
    for (int s = KMAX - 1; s > 0; --s) {
      const bool g_lo = key[s - 1] > kc;  // key[s - 1] is still the old value
      key[s] = g_lo ? key[s - 1] : (g_hi ? kc : key[s]);
      g_hi = g_lo;
    }
    key[0] = g_hi ? kc : key[0];
  }
};

struct Walk {
  float3 q;
  int found;
};

template <int KMAX>
__device__ __forceinline__ void visit_cell(const GridHeader &g, const InterpScratch &s, int k, int cx, int cy,
                                           int cz, Walk &w, Best<KMAX> &best) {
  if (w.found >= k) {
    // skip a cell whose box is farther than the current k-th distance
    const float bx0 = g.origin[0] + (float)cx * g.h, by0 = g.origin[1] + (float)cy * g.h,
                bz0 = g.origin[2] + (float)cz * g.h;
    const float dx = fmaxf(fmaxf(bx0 - w.q.x, w.q.x - (bx0 + g.h)), 0.f);
    const float dy = fmaxf(fmaxf(by0 - w.q.y, w.q.y - (by0 + g.h)), 0.f);
    const float dz = g.dims[2] > 1 ? fmaxf(fmaxf(bz0 - w.q.z, w.q.z - (bz0 + g.h)), 0.f) : 0.f;
    const float mind2 = dx * dx + dy * dy + dz * dz;
    const float kd2 = __uint_as_float((unsigned)(best.last() >> 32));
    if (mind2 > kd2 * 1.00001f + 1e-30f) return;
  }
  const int cell = (cz * g.dims[1] + cy) * g.dims[0] + cx;
  const int e0 = __ldg(s.cell_start + cell), e1 = __ldg(s.cell_start + cell + 1);
  for (int e = e0; e < e1; ++e) {
    const float4 pt = __ldg(s.pts + e);
    const float ex = w.q.x - pt.x, ey = w.q.y - pt.y, ez = w.q.z - pt.z;
    const float d2 = ex * ex + ey * ey + ez * ez;
    const unsigned long long kc =
        ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)__float_as_int(pt.w);
    ++w.found;
    if (kc < best.last()) best.insert(kc);
  }
}

__device__ __forceinline__ float bilinear_map(const float *R, int H, int W, float ti, float tj) {
  const float fi = floorf(ti), fj = floorf(tj);
  const float ai = ti - fi, aj = tj - fj;
  int i0 = (int)fi, j0 = (int)fj;
  int i1 = i0 + 1, j1 = j0 + 1;
  i0 = clampi(i0, 0, H - 1);
  i1 = clampi(i1, 0, H - 1);
  j0 = ((j0 % W) + W) % W;
  j1 = ((j1 % W) + W) % W;
  const float v00 = __ldg(R + i0 * W + j0), v01 = __ldg(R + i0 * W + j1);
  const float v10 = __ldg(R + i1 * W + j0), v11 = __ldg(R + i1 * W + j1);
  return (1.f - ai) * ((1.f - aj) * v00 + aj * v01) + ai * ((1.f - aj) * v10 + aj * v11);
}

// Exact k nearest of q by walking Chebyshev shells of the coarse grid (own
// cell, the 26 neighbours nearest first, then further shells), skipping
// cells farther than the current k-th distance, until the k-th distance is
// below the distance to every unvisited cell.  Returns the candidates seen.
template <int KMAX>
__device__ int knn_walk(const GridHeader &g, const InterpScratch &s, int k, float3 q, Best<KMAX> &best) {
  Walk w;
  w.q = q;
  w.found = 0;
  int3 c0;
  cell_of(g, w.q, &c0);
  best.init(k);
  const float margin = 1e-4f * g.h;
  const int maxR = max(g.dims[0], max(g.dims[1], g.dims[2]));
  for (int R = 0; R <= maxR; ++R) {
    if (R == 0) {
      visit_cell<KMAX>(g, s, k, c0.x, c0.y, c0.z, w, best);
    } else if (R == 1) {
      for (int o = 0; o < 26; ++o) {
        const int cx = c0.x + kShell1[o][0], cy = c0.y + kShell1[o][1], cz = c0.z + kShell1[o][2];
        if (cx < 0 || cy < 0 || cz < 0 || cx >= g.dims[0] || cy >= g.dims[1] || cz >= g.dims[2]) continue;
        visit_cell<KMAX>(g, s, k, cx, cy, cz, w, best);
      }
    } else {
      const int z0 = max(c0.z - R, 0), z1 = min(c0.z + R, g.dims[2] - 1);
      const int y0 = max(c0.y - R, 0), y1 = min(c0.y + R, g.dims[1] - 1);
      const int x0 = max(c0.x - R, 0), x1 = min(c0.x + R, g.dims[0] - 1);
      for (int cz = z0; cz <= z1; ++cz)
        for (int cy = y0; cy <= y1; ++cy)
          for (int cx = x0; cx <= x1; ++cx) {
            const int cheb = max(abs(cx - c0.x), max(abs(cy - c0.y), abs(cz - c0.z)));
            if (cheb != R) continue;
            visit_cell<KMAX>(g, s, k, cx, cy, cz, w, best);
          }
    }
    float bound = FLT_MAX;
    bool all = true;
    const int cc[3] = {c0.x, c0.y, c0.z};
    const float qv[3] = {w.q.x, w.q.y, w.q.z};
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
    if (w.found >= k) {
      const float kd2 = __uint_as_float((unsigned)(best.last() >> 32));
      const float b = bound - margin;
      if (b > 0.f && kd2 <= b * b) break;
    }
  }
  return w.found;
}

// Weights (Eq. 4), normalisation and blend for pixel p from its k best.
template <int KMAX, int MODE>
__device__ __forceinline__ void blend_store(const InterpArgs &a, long long p, const Best<KMAX> &best, int found) {
  const int k = a.k;
  const int kk = found < k ? found : k;
  const int m = KMAX - k;
  const float pnx = __ldg(a.gnrm + 3 * p), pny = __ldg(a.gnrm + 3 * p + 1), pnz = __ldg(a.gnrm + 3 * p + 2);
  const float pl = sqrtf(pnx * pnx + pny * pny + pnz * pnz);
  float wt[KMAX];
  int jj[KMAX];
  float wsum = 0.f;
#pragma unroll
  for (int sl = 0; sl < KMAX; ++sl) {
    wt[sl] = 0.f;
    jj[sl] = -1;
    if (sl >= m && sl - m < kk) {
      const int j = (int)(unsigned)(best.key[sl] & 0xffffffffu);
      const float d = sqrtf(__uint_as_float((unsigned)(best.key[sl] >> 32)));
      const float wp = a.wp_form == WP_INVERSE ? a.r / (d + a.delta_rel * a.r) : fmaxf(0.f, 1.f - d / a.r);
      const float cx = __ldg(a.cnrm + 3 * j), cy = __ldg(a.cnrm + 3 * j + 1), cz = __ldg(a.cnrm + 3 * j + 2);
      const float cl = sqrtf(cx * cx + cy * cy + cz * cz);
      float wn = 0.f;
      if (pl > 0.f && cl > 0.f) wn = fmaxf(0.f, (cx * pnx + cy * pny + cz * pnz) / (cl * pl));
      wt[sl] = wp * wn + wp + a.eps;
      jj[sl] = j;
      wsum += wt[sl];
    }
  }
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  if constexpr (MODE == MODE_IRRADIANCE) {
#pragma unroll
    for (int sl = 0; sl < KMAX; ++sl)
      if (jj[sl] >= 0) {
        const int j = jj[sl];
        const float Wt = wt[sl] / wsum;
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
      for (int sl = 0; sl < KMAX; ++sl) {
        if (jj[sl] < 0) continue;
        const int j = jj[sl];
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
        const float Wt = wt[sl] / wsum;
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
    for (int sl = 0; sl < KMAX; ++sl)
      if (sl >= m) a.nbr_out[(size_t)p * k + (sl - m)] = jj[sl];
  }
}

// One thread per pixel (in the spatial order when the pixel ordering is
// on): exact k nearest by the grid walk, then weights and blend.  MODE is
// the blend (IRRADIANCE / LOOKUP), fixed at compile time so that each kernel
// only carries its own registers and code.
template <int KMAX, int MODE>
__global__ void __launch_bounds__(256, KMAX <= 16 ? 4 : 2) interp_query_kernel(InterpArgs a, InterpScratch s) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long P = (long long)a.width * a.height;
  if (t >= P) return;
  const long long p = s.order ? (long long)__ldg(s.order + t) : t;
  const GridHeader g = *s.hdr;
  Best<KMAX> best;
  const int found = knn_walk<KMAX>(g, s, a.k, query_point(a, p), best);
  blend_store<KMAX, MODE>(a, p, best, found);
}

cudaError_t launch_interp(const InterpArgs &a, const InterpScratch &s, cudaStream_t st, Tracer *tr) {
  DRC_TRACED(tr, "interp grid_bounds", st, (grid_bounds_kernel<<<1, 1024, 0, st>>>(a, s)));
  const int cb = (a.n + 255) / 256;
  DRC_TRACED(tr, "interp grid_count", st, (grid_count_kernel<<<cb, 256, 0, st>>>(a, s)));
  DRC_TRACED(tr, "interp grid_scan", st, (scan_kernel<<<1, 1024, 0, st>>>(&s.hdr->ncells, s.cell_count, s.cell_start)));
  DRC_TRACED(tr, "interp grid_scatter", st, (grid_scatter_kernel<<<cb, 256, 0, st>>>(a, s)));
  const long long P = (long long)a.width * a.height;
  if (P == 0) return cudaGetLastError();
  const unsigned blocks = (unsigned)((P + 255) / 256);
  if (s.order) {
    DRC_TRACED(tr, "interp pixel_count", st, (pixel_count_kernel<<<blocks, 256, 0, st>>>(a, s)));
    DRC_TRACED(tr, "interp pixel_scan", st, (scan_kernel<<<1, 1024, 0, st>>>(&s.hdr->nfine, s.fine_count, s.fine_start)));
    DRC_TRACED(tr, "interp pixel_scatter", st, (pixel_scatter_kernel<<<blocks, 256, 0, st>>>(a, s)));
  }
  if (tr) tr->begin("interp query", st);
  if (a.mode == MODE_IRRADIANCE) {
    if (a.k <= 8)
      interp_query_kernel<8, MODE_IRRADIANCE><<<blocks, 256, 0, st>>>(a, s);
    else if (a.k <= 16)
      interp_query_kernel<16, MODE_IRRADIANCE><<<blocks, 256, 0, st>>>(a, s);
    else
      interp_query_kernel<32, MODE_IRRADIANCE><<<blocks, 256, 0, st>>>(a, s);
  } else {
    if (a.k <= 8)
      interp_query_kernel<8, 1><<<blocks, 256, 0, st>>>(a, s);
    else if (a.k <= 16)
      interp_query_kernel<16, 1><<<blocks, 256, 0, st>>>(a, s);
    else
      interp_query_kernel<32, 1><<<blocks, 256, 0, st>>>(a, s);
  }
  if (tr) tr->end(st);
  return cudaGetLastError();
}

}  // namespace drc
