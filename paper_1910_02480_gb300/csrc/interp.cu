// interp.cu -- radiance-cache interpolation of Sec. 3.2 on the GPU.
//
// 1. A uniform grid over the cache points (3-D first-hit positions for the
//    WORLD metric, integer pixel coordinates for the IMAGE metric) is built by
//    counting sort: bounds -> per-cell counts -> prefix sum -> scatter into a
//    cell-ordered float4 table (x, y, z, index).
// 2. Optionally the pixels are counting-sorted by a finer grid over the same
//    box (serpentine bin order), so that the 32 threads of a warp query
//    nearby points: their candidate sets then coincide (WORLD metric; image
//    order is already coherent for the IMAGE metric).  The sorted copy holds
//    each pixel's position and index.
// 3. WORLD metric with the ordering and no neighbour list: the warp-
//    cooperative query below -- a warp gathers the caches near its 32 points
//    into shared memory once and every lane selects from that buffer.
//    Otherwise one thread per pixel visits its own cell, then the 26 neighbours nearest
//    first, then further Chebyshev shells, skipping every cell whose box is
//    farther than the current k-th distance.  The walk stops once the k-th
//    distance is below the distance to every unvisited cell, so the
//    selection equals a brute-force scan.  WORLD metric without a neighbour
//    list: a first walk keeps the k smallest d^2 as 32-bit keys (two integer
//    min/max per slot per insertion) and notes the cells where keys went in;
//    a second pass collects from those cells every candidate at or below the
//    k-th distance.  Ties there, the IMAGE metric and the neighbour list take
//    the exact walk, whose sorted register array holds 64-bit keys (d^2 bits
//    << 32 | index: ascending key = ascending (d^2, index), since d^2 >= 0).
// 4. Weights w = w_p w_n + w_p + eps (Eq. 4), normalised (Sec. 3.2), blend of
//    the payloads (IRRADIANCE) or of bilinear lat-long lookups of the cached
//    maps in each cache's frame (LOOKUP).
#include <cuda_runtime.h>

#include <cfloat>
#include <climits>
#include <cstdio>
#include <cstdlib>

#include "interp.cuh"

namespace drc {

static constexpr int METRIC_IMAGE = 0;
static constexpr int WP_INVERSE = 0;
static constexpr int MODE_IRRADIANCE = 0;

// Caches per grid cell the grid is sized for.  The per-thread walks: k/2 (at
// least 1).  At 4096 caches, k = 16, 1080p WORLD the per-thread two-walk
// query measured 0.609 ms with 8 per cell, against 0.614 (9) and 0.615 (10);
// 6 per cell suited the single 64-bit walk, whose insertions cost three times
// as much.  The warp-cooperative query gathers whole cells around a warp's
// points, so finer cells gather fewer caches beyond the radius it needs.
static inline int per_cell(int k) { return k / 2 > 1 ? k / 2 : 1; }
// At 1080p, 4096 caches, k = 16: 1 cache per cell 0.363 ms, 2 per cell 0.400.
static constexpr int kCoopPerCell = 1;
// First-gather radius and near distance of the cooperative query, in units of
// the expected distance to the (k+1)-th nearest cache at the caches' mean
// density.  Measured at 1080p, 4096 caches, k = 16 (near 0.8): rho 1.2
// 0.410 ms, 1.4 0.364, 1.6 0.394; near 0.6 / 0.8 / 1.0 (rho 1.4): 0.383,
// 0.364, 0.363.
static constexpr float kCoopRho = 1.4f, kCoopNear = 0.9f;

// Sized for the finer of the two grids, so one scratch serves either query.
int interp_max_cells(int n, int k) {
  const int pc = per_cell(k) < kCoopPerCell ? per_cell(k) : kCoopPerCell;
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

static constexpr long long kScanTile = 16 * 1024;  // bins per scan tile (SCAN_T)
static inline size_t fine_tiles(long long mf) { return (size_t)((mf + kScanTile - 1) / kScanTile); }

size_t interp_order_bytes(long long P, int n) {
  const size_t mf = (size_t)max_fine_bins(P);
  return align256(mf * sizeof(int)) + align256(fine_tiles(mf) * sizeof(int)) + align256((size_t)P * sizeof(float4)) +
         align256((size_t)n * 2 * sizeof(float4));
}

void interp_attach_order(InterpScratch &s, void *base, long long P, int n) {
  const size_t mf = (size_t)max_fine_bins(P);
  char *p = static_cast<char *>(base);
  s.fine_count = reinterpret_cast<int *>(p);
  p += align256(mf * sizeof(int));
  s.fine_tile_sum = reinterpret_cast<int *>(p);
  p += align256(fine_tiles(mf) * sizeof(int));
  s.order = reinterpret_cast<float4 *>(p);
  p += align256((size_t)P * sizeof(float4));
  s.aux = reinterpret_cast<float4 *>(p);
  (void)n;
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

// Fine cell of a point, numbered along a serpentine path (x runs reverse on
// every other row, rows on every other plane), so consecutive bins are
// neighbouring cells and a warp of consecutive sorted pixels stays compact.
__device__ __forceinline__ int fine_of(const GridHeader &g, float3 p) {
  int cx = clampi((int)floorf((p.x - g.origin[0]) * g.fine_inv_h), 0, g.fdims[0] - 1);
  int cy = clampi((int)floorf((p.y - g.origin[1]) * g.fine_inv_h), 0, g.fdims[1] - 1);
  const int cz = clampi((int)floorf((p.z - g.origin[2]) * g.fine_inv_h), 0, g.fdims[2] - 1);
  if (cz & 1) cy = g.fdims[1] - 1 - cy;
  const int row = cz * g.fdims[1] + cy;
  if (row & 1) cx = g.fdims[0] - 1 - cx;
  return row * g.fdims[0] + cx;
}

// Single block: bounds of the cache points, cubic cells sized for about k/2
// caches each over the occupied axes, the fine pixel-ordering grid, counts
// cleared.  The sizing is float arithmetic in the log domain (the cell size
// only moves work between cells: any size gives the same neighbours).
__global__ void grid_bounds_kernel(InterpArgs a, InterpScratch s) {
  __shared__ float slo[3][32], shi[3][32];
  __shared__ GridHeader sg;
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
#pragma unroll 4
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
    float log_vol = 0.f;
    for (int d = 0; d < 3; ++d) {
      ext[d] = Hh[d] - L[d];
      if (ext[d] > 0.f) {
        ++active;
        log_vol += logf(ext[d]);
      }
    }
    const int pc = a.cell_caches > 1 ? a.cell_caches : 1;
    const float target = (float)((a.n + pc - 1) / pc);
    float h = active ? expf((log_vol - logf(target)) / (float)active) : 1.f;
    if (!(h > 0.f) || !(h < FLT_MAX)) h = 1.f;
    GridHeader g;
    // grow h until the cells fit the scratch (a bounded number of times: a
    // non-finite extent ends in one cell, which is still an exact search)
    int tries = 0;
    for (;;) {
      long long prod = 1;
      for (int d = 0; d < 3; ++d) {
        const float q = ext[d] > 0.f ? ceilf(ext[d] / h) : 1.f;
        const int nd = q >= 1.f ? (q <= (float)s.max_cells ? (int)q : s.max_cells + 1) : 1;
        g.dims[d] = nd;
        prod *= nd;
        if (prod > s.max_cells) prod = (long long)s.max_cells + 1;  // no overflow on the next axis
      }
      if (prod <= s.max_cells) {
        g.ncells = (int)prod;
        break;
      }
      if (++tries == 256) {
        g.dims[0] = g.dims[1] = g.dims[2] = 1;
        g.ncells = 1;
        break;
      }
      h *= 1.125f;
    }
    for (int d = 0; d < 3; ++d) g.origin[d] = L[d];
    g.h = h;
    g.inv_h = 1.f / h;
    // fine grid: each coarse cell split m ways per occupied axis, about 32
    // pixels per fine cell (16 and 64 measured slower at 1080p)
    int m = 1;
    if (s.order && active) {
      float tgt = (float)a.width * (float)a.height / 32.f;
      if (tgt > (float)s.max_fine) tgt = (float)s.max_fine;
      const float mf = floorf(expf(logf(tgt / (float)g.ncells) / (float)active));
      m = mf >= 64.f ? 64 : (mf >= 1.f ? (int)mf : 1);
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
    if (s.order && nf > s.max_fine) {
      // more coarse cells than the order scratch has bins (a few pixels,
      // many caches): every pixel in one bin
      g.fdims[0] = g.fdims[1] = g.fdims[2] = 1;
      nf = 1;
      m = 0;
    }
    g.nfine = (int)nf;
    g.fine_inv_h = (float)m / h;
    // expected distance to the (k+1)-th nearest cache at the mean density
    // over the occupied axes (unit-ball volume 2, pi, 4 pi / 3)
    float rk = 0.f;
    if (active) {
      const float per = (float)(a.k + 1) / (float)a.n;  // of the occupied volume
      const float ball = active == 1 ? 2.f : (active == 2 ? 3.14159265f : 4.18879020f);
      rk = expf((logf(per / ball) + log_vol) / (float)active);
      if (!(rk < FLT_MAX)) rk = 0.f;
    }
    g.coop_r0 = a.coop_rho * rk;
    g.coop_near = a.coop_near * rk;
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

// Exclusive scans of bin counts; counts become write cursors.  Each thread
// takes SCAN_V consecutive bins (16-byte loads and stores; the arrays are
// 16-byte aligned), so a 1024-thread block covers a tile of SCAN_T bins.
static constexpr int SCAN_V = 16;
static constexpr int SCAN_THREADS = 1024;
static constexpr int SCAN_T = SCAN_V * SCAN_THREADS;
__device__ __forceinline__ void scan_load(const int *counts, int nc, int i0, int (&v)[SCAN_V]) {
  if (i0 + SCAN_V <= nc) {
#pragma unroll
    for (int q = 0; q < SCAN_V / 4; ++q) {
      const int4 t = *reinterpret_cast<const int4 *>(counts + i0 + 4 * q);
      v[4 * q] = t.x, v[4 * q + 1] = t.y, v[4 * q + 2] = t.z, v[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int e = 0; e < SCAN_V; ++e) v[e] = i0 + e < nc ? counts[i0 + e] : 0;
  }
}

// Block total of the thread values x (every thread gets it).
__device__ __forceinline__ int block_sum(int x, int *warp_tot) {
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (l == 0) warp_tot[w] = x;
  __syncthreads();
  int t = 0;
  for (int i = 0; i < nw; ++i) t += warp_tot[i];
  __syncthreads();
  return t;
}

// One tile starting at base: the thread's bins v (loaded), the total before
// the tile (carry); writes the exclusive offsets to counts and, when given,
// starts.  Returns the tile's total.
__device__ __forceinline__ int scan_tile(int *counts, int *starts, int nc, int base, int carry, int (&v)[SCAN_V],
                                         int *warp_tot) {
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int i0 = base + SCAN_V * threadIdx.x;
  int tsum = 0;
#pragma unroll
  for (int e = 0; e < SCAN_V; ++e) tsum += v[e];
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
  int run = carry + (w > 0 ? warp_tot[w - 1] : 0) + x - tsum;
#pragma unroll
  for (int e = 0; e < SCAN_V; ++e) {  // v becomes the exclusive offsets
    const int c = v[e];
    v[e] = run;
    run += c;
  }
  if (i0 + SCAN_V <= nc) {
#pragma unroll
    for (int q = 0; q < SCAN_V / 4; ++q) {
      const int4 o4 = make_int4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      *reinterpret_cast<int4 *>(counts + i0 + 4 * q) = o4;
      if (starts) *reinterpret_cast<int4 *>(starts + i0 + 4 * q) = o4;
    }
  } else {
#pragma unroll
    for (int e = 0; e < SCAN_V; ++e)
      if (i0 + e < nc) {
        counts[i0 + e] = v[e];
        if (starts) starts[i0 + e] = v[e];
      }
  }
  const int tot = warp_tot[nw - 1];
  __syncthreads();  // warp_tot is rewritten by the next tile
  return tot;
}

// Single block over counts[0..*n_ptr) (the cache grid): tile after tile,
// the next tile's loads issued before this tile's scan; starts[*n_ptr] =
// total.
__global__ void __launch_bounds__(SCAN_THREADS) scan_kernel(const int *n_ptr, int *counts, int *starts) {
  __shared__ int warp_tot[32];
  const int nc = *n_ptr;
  int carry = 0;
  int v[SCAN_V];
  scan_load(counts, nc, SCAN_V * threadIdx.x, v);
  for (int base = 0; base < nc; base += SCAN_T) {
    int nv[SCAN_V];
#pragma unroll
    for (int e = 0; e < SCAN_V; ++e) nv[e] = 0;
    if (base + SCAN_T < nc) scan_load(counts, nc, base + SCAN_T + SCAN_V * threadIdx.x, nv);
    carry += scan_tile(counts, starts, nc, base, carry, v, warp_tot);
#pragma unroll
    for (int e = 0; e < SCAN_V; ++e) v[e] = nv[e];
  }
  if (threadIdx.x == 0) starts[nc] = carry;
}

// Many bins (the pixel order): block b of scan_sum_kernel totals tile b,
// then block b of scan_tiles_kernel scans tile b from the totals before it.
// The grids cover the largest bin count; blocks past *n_ptr do nothing.
__global__ void __launch_bounds__(SCAN_THREADS) scan_sum_kernel(const int *n_ptr, const int *counts, int *tile_sum) {
  __shared__ int warp_tot[32];
  const int nc = *n_ptr, base = blockIdx.x * SCAN_T;
  if (base >= nc) return;  // block-uniform
  int v[SCAN_V];
  scan_load(counts, nc, base + SCAN_V * threadIdx.x, v);
  int t = 0;
#pragma unroll
  for (int e = 0; e < SCAN_V; ++e) t += v[e];
  t = block_sum(t, warp_tot);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = t;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles_kernel(const int *n_ptr, int *counts, const int *tile_sum) {
  __shared__ int warp_tot[32];
  const int nc = *n_ptr, base = blockIdx.x * SCAN_T;
  if (base >= nc) return;  // block-uniform
  int v[SCAN_V];
  scan_load(counts, nc, base + SCAN_V * threadIdx.x, v);
  int carry = 0;
  for (int b = 0; b < (int)blockIdx.x; ++b) carry += __ldg(tile_sum + b);
  scan_tile(counts, nullptr, nc, base, carry, v, warp_tot);
}

__global__ void grid_scatter_kernel(InterpArgs a, InterpScratch s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  const int c = s.cache_cell[j];
  const int pos = atomicAdd(&s.cell_count[c], 1);
  const float3 p = cache_point(a, j);
  s.pts[pos] = make_float4(p.x, p.y, p.z, __int_as_float(j));
  if (s.aux) {
    float nx = __ldg(a.cnrm + 3 * j), ny = __ldg(a.cnrm + 3 * j + 1), nz = __ldg(a.cnrm + 3 * j + 2);
    const float nl = sqrtf(nx * nx + ny * ny + nz * nz);
    if (nl > 0.f) {
      nx /= nl;
      ny /= nl;
      nz /= nl;
    } else {
      nx = ny = nz = 0.f;
    }
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
    if (a.payload) {
      e0 = __ldg(a.payload + 3 * j);
      e1 = __ldg(a.payload + 3 * j + 1);
      e2 = __ldg(a.payload + 3 * j + 2);
    }
    s.aux[2 * pos] = make_float4(nx, ny, nz, e0);
    s.aux[2 * pos + 1] = make_float4(e1, e2, 0.f, 0.f);
  }
}

// Pixel counting sort by fine cell.  Neighbouring pixels mostly share a
// fine cell, so the lanes of a warp that do are grouped (match.any) and one
// of them adds the group's count: one atomic per group instead of per pixel.
// The scatter gives a group consecutive slots in lane order.
__global__ void pixel_count_kernel(InterpArgs a, InterpScratch s) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long P = (long long)a.width * a.height;
  const unsigned live = __ballot_sync(0xffffffffu, p < P);
  if (p >= P) return;
  const GridHeader g = *s.hdr;
  const int f = fine_of(g, query_point(a, p));
  const unsigned peers = __match_any_sync(live, f);
  if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&s.fine_count[f], __popc(peers));
}

__global__ void pixel_scatter_kernel(InterpArgs a, InterpScratch s) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long P = (long long)a.width * a.height;
  const unsigned live = __ballot_sync(0xffffffffu, p < P);
  if (p >= P) return;
  const GridHeader g = *s.hdr;
  const float3 q = query_point(a, p);
  const int f = fine_of(g, q);
  const unsigned peers = __match_any_sync(live, f);
  const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(&s.fine_count[f], __popc(peers));
  base = __shfl_sync(live, base, leader);
  s.order[base + __popc(peers & ((1u << lane) - 1u))] = make_float4(q.x, q.y, q.z, __int_as_float((int)p));
}

// The 26 neighbours of a cell, nearest first: faces, edges, corners.
__constant__ signed char kShell1[26][3] = {
    {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1},
    {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}, {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {1, 0, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1},
    {-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},
    {-1, 1, 1}, {1, 1, 1}};

static constexpr int QUERY_THREADS = 256;

// Selection policies of the walk.  Each takes every candidate the walk
// visits (offer: its d^2, its slot e in the cell-ordered table and its cache
// index bits), and tells the walk its current pruning distance (kd2) and
// whether that distance is a bound yet (bounded).

// Exact k best: KMAX sorted 64-bit keys (d^2 bits << 32 | index, ascending
// = ascending (d^2, index)); the first KMAX-k slots hold 0 (never
// displaced), so the k-th best is always the last slot.  Insertion (kc below
// the last key): gt[s] = key[s] > kc is false up to the insertion point and
// true after it, so each slot takes its lower neighbour (past the point), kc
// (at it) or itself (before it) -- one 64-bit compare and two 64-bit selects
// per slot, the compare of slot s - 1 serving slot s - 1 next.  This gives
// the ordered neighbour list and settles ties at the k-th distance by index.
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
  __device__ __forceinline__ bool bounded(int found, int k) const { return found >= k; }
  __device__ __forceinline__ void enter(unsigned) {}
  __device__ __forceinline__ float kd2() const { return __uint_as_float((unsigned)(last() >> 32)); }
  __device__ __forceinline__ void offer(float d2, int, float idx_bits) {
    const unsigned long long kc = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)__float_as_int(idx_bits);
    if (kc < last()) insert(kc);
  }
};

// The k smallest d^2 alone, as 32-bit keys (the bits of a non-negative float
// order as the float does), same padding.  With no index riding along, slot
// s after inserting kc is min(key[s], max(key[s-1], kc)): two integer
// min/max per slot instead of six 32-bit operations.  The last slot ends as
// the exact k-th smallest d^2, tau.
//
// It also keeps, for the second walk, the cells a key went into (mask: bit
// o < 26 for the o-th neighbour of the first shell, bit 26 for the own cell,
// bit 27 for any farther cell) and whether more than k candidates may lie
// within tau (tie).  Every candidate below tau went in when offered (tau
// only falls), so without a tie the k nearest all lie in mask's cells.  A
// tie shows as a key equal to the current k-th (refused), or as a key that
// pushed out a k-th equal to the one below it (that candidate stays within
// the new k-th distance but out of the list).
static constexpr unsigned kOwnCell = 1u << 26, kFarCells = 1u << 27;
template <int KMAX>
struct KthDist {
  unsigned key[KMAX];
  unsigned cur, mask;
  bool tie;
  __device__ __forceinline__ void init(int k) {
#pragma unroll
    for (int s = 0; s < KMAX; ++s) key[s] = s < KMAX - k ? 0u : ~0u;
    cur = mask = 0u;
    tie = false;
  }
  __device__ __forceinline__ unsigned last() const { return key[KMAX - 1]; }
  __device__ __forceinline__ bool bounded(int found, int k) const { return found >= k; }
  __device__ __forceinline__ void enter(unsigned bit) { cur = bit; }
  __device__ __forceinline__ float kd2() const { return __uint_as_float(last()); }
  __device__ __forceinline__ void offer(float d2, int, float) {
    const unsigned kc = __float_as_uint(d2), kl = last();
    if (kc <= kl) {
      tie |= kc == kl || (key[KMAX - 2] == kl && kl != ~0u);
      if (kc < kl) {
#pragma unroll
        for (int s = KMAX - 1; s > 0; --s) key[s] = min(key[s], max(key[s - 1], kc));
        key[0] = min(key[0], kc);
        mask |= cur;
      }
    }
  }
};

// Second walk, under the k-th distance tau: every candidate with d^2 <= tau
// (bits compared, as in the first walk) is one of the k nearest or tied with
// the k-th.  Their table slots go down the thread's shared-memory column
// (stride QUERY_THREADS, at most cap of them); n counts them all, so n > k
// flags a tie.  tau = ~0u (fewer than k candidates) takes every candidate:
// as a float it is a NaN, which prunes no cell and stops no shell.
struct Collect {
  unsigned tau;
  int n, cap;
  int *col;
  __device__ __forceinline__ bool bounded(int, int) const { return true; }
  __device__ __forceinline__ void enter(unsigned) {}
  __device__ __forceinline__ float kd2() const { return __uint_as_float(tau); }
  __device__ __forceinline__ void offer(float d2, int e, float) {
    if (__float_as_uint(d2) <= tau) {
      if (n < cap) col[n * QUERY_THREADS] = e;
      ++n;
    }
  }
};

struct Walk {
  float3 q;
  int found;
};

__device__ __forceinline__ float cand_d2(float3 q, float4 pt) {
  const float ex = q.x - pt.x, ey = q.y - pt.y, ez = q.z - pt.z;
  return ex * ex + ey * ey + ez * ez;
}

template <class Sel>
__device__ __forceinline__ void visit_range(const InterpScratch &s, int cell, Walk &w, Sel &sel) {
  const int e0 = __ldg(s.cell_start + cell), e1 = __ldg(s.cell_start + cell + 1);
  for (int e = e0; e < e1; ++e) {
    const float4 pt = __ldg(s.pts + e);
    ++w.found;
    sel.offer(cand_d2(w.q, pt), e, pt.w);
  }
}

template <class Sel>
__device__ __forceinline__ void visit_cell(const GridHeader &g, const InterpScratch &s, int k, int cx, int cy,
                                           int cz, Walk &w, Sel &sel) {
  if (sel.bounded(w.found, k)) {
    // skip a cell whose box is farther than the current k-th distance
    const float bx0 = g.origin[0] + (float)cx * g.h, by0 = g.origin[1] + (float)cy * g.h,
                bz0 = g.origin[2] + (float)cz * g.h;
    const float dx = fmaxf(fmaxf(bx0 - w.q.x, w.q.x - (bx0 + g.h)), 0.f);
    const float dy = fmaxf(fmaxf(by0 - w.q.y, w.q.y - (by0 + g.h)), 0.f);
    const float dz = g.dims[2] > 1 ? fmaxf(fmaxf(bz0 - w.q.z, w.q.z - (bz0 + g.h)), 0.f) : 0.f;
    const float mind2 = dx * dx + dy * dy + dz * dz;
    if (mind2 > sel.kd2() * 1.00001f + 1e-30f) return;
  }
  visit_range(s, (cz * g.dims[1] + cy) * g.dims[0] + cx, w, sel);
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

// Walk of Chebyshev shells of the coarse grid around q (own cell, the 26
// neighbours nearest first, then further shells), skipping cells farther
// than the policy's current distance, until that distance is below the
// distance to every unvisited cell: the policy then has seen every
// candidate a brute-force scan would keep.  Returns the candidates seen.
template <class Sel>
__device__ int knn_walk(const GridHeader &g, const InterpScratch &s, int k, float3 q, Sel &sel) {
  Walk w;
  w.q = q;
  w.found = 0;
  int3 c0;
  cell_of(g, w.q, &c0);
  const float margin = 1e-4f * g.h;
  const int maxR = max(g.dims[0], max(g.dims[1], g.dims[2]));
  for (int R = 0; R <= maxR; ++R) {
    if (R == 0) {
      sel.enter(kOwnCell);
      visit_cell(g, s, k, c0.x, c0.y, c0.z, w, sel);
    } else if (R == 1) {
      for (int o = 0; o < 26; ++o) {
        const int cx = c0.x + kShell1[o][0], cy = c0.y + kShell1[o][1], cz = c0.z + kShell1[o][2];
        if (cx < 0 || cy < 0 || cz < 0 || cx >= g.dims[0] || cy >= g.dims[1] || cz >= g.dims[2]) continue;
        sel.enter(1u << o);
        visit_cell(g, s, k, cx, cy, cz, w, sel);
      }
    } else {
      sel.enter(kFarCells);
      const int z0 = max(c0.z - R, 0), z1 = min(c0.z + R, g.dims[2] - 1);
      const int y0 = max(c0.y - R, 0), y1 = min(c0.y + R, g.dims[1] - 1);
      const int x0 = max(c0.x - R, 0), x1 = min(c0.x + R, g.dims[0] - 1);
      for (int cz = z0; cz <= z1; ++cz)
        for (int cy = y0; cy <= y1; ++cy)
          for (int cx = x0; cx <= x1; ++cx) {
            const int cheb = max(abs(cx - c0.x), max(abs(cy - c0.y), abs(cz - c0.z)));
            if (cheb != R) continue;
            visit_cell(g, s, k, cx, cy, cz, w, sel);
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
    if (sel.bounded(w.found, k)) {
      const float kd2 = sel.kd2();
      const float b = bound - margin;
      if (b > 0.f && kd2 <= b * b) break;
    }
  }
  return w.found;
}

// Per-pixel data of the blend: the unit-length test of the surface normal
// and, for LOOKUP, the unit direction the maps are read in.
struct PixelShade {
  float nx, ny, nz, nl;
  float ox, oy, oz;
  bool dir_ok;
};

template <int MODE>
__device__ __forceinline__ PixelShade pixel_shade(const InterpArgs &a, long long p) {
  PixelShade px;
  px.nx = __ldg(a.gnrm + 3 * p), px.ny = __ldg(a.gnrm + 3 * p + 1), px.nz = __ldg(a.gnrm + 3 * p + 2);
  px.nl = sqrtf(px.nx * px.nx + px.ny * px.ny + px.nz * px.nz);
  px.ox = px.oy = px.oz = 0.f;
  px.dir_ok = false;
  if constexpr (MODE != MODE_IRRADIANCE) {
    const float ox = __ldg(a.gdir + 3 * p), oy = __ldg(a.gdir + 3 * p + 1), oz = __ldg(a.gdir + 3 * p + 2);
    const float ol = sqrtf(ox * ox + oy * oy + oz * oz);
    if (ol > 0.f) {
      px.ox = ox / ol;
      px.oy = oy / ol;
      px.oz = oz / ol;
      px.dir_ok = true;
    }
  }
  return px;
}

// Eq. 4: w = w_p w_n + w_p + eps for cache j at squared distance d2, with
// w_p = r / (d + delta) (INVERSE) or max(0, 1 - d / r) (LINEAR) and w_n the
// clamped cosine between the normals (0 for a zero-length normal).
__device__ __forceinline__ float nbr_weight(const InterpArgs &a, const PixelShade &px, int j, float d2) {
  const float d = sqrtf(d2);
  const float wp = a.wp_form == WP_INVERSE ? a.r / (d + a.delta_rel * a.r) : fmaxf(0.f, 1.f - d / a.r);
  const float cx = __ldg(a.cnrm + 3 * j), cy = __ldg(a.cnrm + 3 * j + 1), cz = __ldg(a.cnrm + 3 * j + 2);
  const float cl = sqrtf(cx * cx + cy * cy + cz * cz);
  float wn = 0.f;
  if (px.nl > 0.f && cl > 0.f) wn = fmaxf(0.f, (cx * px.nx + cy * px.ny + cz * px.nz) / (cl * px.nl));
  return wp * wn + wp + a.eps;
}

// What cache j contributes to the blend: its irradiance payload, or (LOOKUP)
// a bilinear lat-long read of its map in the pixel's direction expressed in
// the cache's frame (up = +Z, or +Y when the normal is along Z; t = up x n,
// b = n x t).  False where the cache adds nothing: a zero normal, or the
// direction below the cache's horizon.
template <int MODE>
__device__ __forceinline__ bool nbr_value(const InterpArgs &a, const PixelShade &px, int j, float3 &v) {
  if constexpr (MODE == MODE_IRRADIANCE) {
    v = make_float3(__ldg(a.payload + 3 * j), __ldg(a.payload + 3 * j + 1), __ldg(a.payload + 3 * j + 2));
    return true;
  } else {
    if (!px.dir_ok) return false;
    const float two_pi = 6.283185307179586f;
    const size_t map_sz = (size_t)a.mapH * a.mapW;
    float nx = __ldg(a.cnrm + 3 * j), ny = __ldg(a.cnrm + 3 * j + 1), nz = __ldg(a.cnrm + 3 * j + 2);
    const float nl = sqrtf(nx * nx + ny * ny + nz * nz);
    if (!(nl > 0.f)) return false;
    nx /= nl;
    ny /= nl;
    nz /= nl;
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
    const float lx = px.ox * tx + px.oy * ty + px.oz * tz;
    const float ly = px.ox * bx + px.oy * by + px.oz * bz;
    float lz = px.ox * nx + px.oy * ny + px.oz * nz;
    if (!(lz > 0.f)) return false;
    lz = fminf(lz, 1.f);
    const float theta = acosf(lz);
    float phi = atan2f(ly, lx);
    if (phi < 0.f) phi += two_pi;
    const float ti = theta * (2.f / 3.14159265358979f) * (float)a.mapH - 0.5f;
    const float tj = phi * (1.f / two_pi) * (float)a.mapW - 0.5f;
    const float *Rj = a.maps + (size_t)j * 3 * map_sz;
    v = make_float3(bilinear_map(Rj, a.mapH, a.mapW, ti, tj), bilinear_map(Rj + map_sz, a.mapH, a.mapW, ti, tj),
                    bilinear_map(Rj + 2 * map_sz, a.mapH, a.mapW, ti, tj));
    return true;
  }
}

// Normalisation (Sec. 3.2) and blend for pixel p from its k best in (d^2,
// index) order; the optional neighbour list in that order.
template <int KMAX, int MODE>
__device__ __forceinline__ void blend_store(const InterpArgs &a, long long p, const Best<KMAX> &best, int found) {
  const int k = a.k;
  const int kk = found < k ? found : k;
  const int m = KMAX - k;
  const PixelShade px = pixel_shade<MODE>(a, p);
  float wt[KMAX];
  int jj[KMAX];
  float wsum = 0.f;
#pragma unroll
  for (int sl = 0; sl < KMAX; ++sl) {
    wt[sl] = 0.f;
    jj[sl] = -1;
    if (sl >= m && sl - m < kk) {
      const int j = (int)(unsigned)(best.key[sl] & 0xffffffffu);
      wt[sl] = nbr_weight(a, px, j, __uint_as_float((unsigned)(best.key[sl] >> 32)));
      jj[sl] = j;
      wsum += wt[sl];
    }
  }
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
#pragma unroll
  for (int sl = 0; sl < KMAX; ++sl) {
    float3 v;
    if (jj[sl] >= 0 && nbr_value<MODE>(a, px, jj[sl], v)) {
      const float Wt = wt[sl] / wsum;
      acc0 += Wt * v.x;
      acc1 += Wt * v.y;
      acc2 += Wt * v.z;
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
  if (a.nbr_w) {
#pragma unroll
    for (int sl = 0; sl < KMAX; ++sl)
      if (sl >= m) a.nbr_w[(size_t)p * k + (sl - m)] = jj[sl] >= 0 ? wt[sl] / wsum : 0.f;
  }
}

// The same blend from the collected table slots (cnt of them, in visit
// order): sum of w v over the sum of w.
template <int MODE>
__device__ __forceinline__ void blend_list(const InterpArgs &a, const InterpScratch &s, long long p, float3 q,
                                           const int *col, int cnt) {
  const PixelShade px = pixel_shade<MODE>(a, p);
  float wsum = 0.f, acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  for (int i = 0; i < cnt; ++i) {
    const float4 pt = __ldg(s.pts + col[i * QUERY_THREADS]);
    const int j = __float_as_int(pt.w);
    const float w = nbr_weight(a, px, j, cand_d2(q, pt));
    wsum += w;
    float3 v;
    if (nbr_value<MODE>(a, px, j, v)) {
      acc0 += w * v.x;
      acc1 += w * v.y;
      acc2 += w * v.z;
    }
  }
  const bool any = cnt > 0;
  a.out[3 * p] = any ? acc0 / wsum : 0.f;
  a.out[3 * p + 1] = any ? acc1 / wsum : 0.f;
  a.out[3 * p + 2] = any ? acc2 / wsum : 0.f;
}

// One thread per pixel (in the spatial order when the pixel ordering is
// on).  MODE is the blend (IRRADIANCE / LOOKUP), fixed at compile time so
// that each kernel only carries its own registers and code.
//
// FAST (WORLD metric, no neighbour list asked for): the first walk finds the
// k-th smallest d^2 with 32-bit keys, the second collects every candidate
// at or below it from the cells where keys went in (or from a whole second
// walk, when one went in beyond the first shell), and the blend reads them
// back.  A pixel with a possible tie at the k-th distance (which the (d^2,
// index) order settles), or with a count other than min(k, candidates),
// takes the exact 64-bit walk.  The other form
// always takes that walk: integer IMAGE distances tie often, and the
// neighbour list is given in (d^2, index) order.
template <int KMAX, int MODE, bool FAST>
// Blocks per SM: 6 for the IRRADIANCE two-walk form at k <= 16 (40
// registers and some spill traffic, yet at 1080p, k = 16: 0.609 ms, against
// 0.626 with 5, 0.632 with 4 and 0.675 with 7), else 4 (64 registers) or 2.
__global__ void __launch_bounds__(QUERY_THREADS, KMAX <= 16 ? (FAST && MODE == MODE_IRRADIANCE ? 6 : 4) : 2)
    interp_query_kernel(InterpArgs a, InterpScratch s) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long P = (long long)a.width * a.height;
  if (t >= P) return;
  const long long p = s.order ? (long long)__float_as_int(__ldg(s.order + t).w) : t;
  const GridHeader g = *s.hdr;
  const float3 q = query_point(a, p);
  if constexpr (FAST) {
    __shared__ int column[KMAX * QUERY_THREADS];
    int *col = column + threadIdx.x;
    KthDist<KMAX> kth;
    kth.init(a.k);
    const int found = knn_walk(g, s, a.k, q, kth);
    Collect c{kth.last(), 0, KMAX, col};
    if (kth.mask & kFarCells) {
      knn_walk(g, s, a.k, q, c);
    } else {
      // only the cells of the first shell a key went into
      Walk w;
      w.q = q;
      w.found = 0;
      int3 c0;
      const int cell0 = cell_of(g, q, &c0);
      for (unsigned m = kth.mask; m; m &= m - 1) {
        const int o = __ffs(m) - 1;
        const int cell = o == 26 ? cell0
                                 : cell0 + kShell1[o][0] + g.dims[0] * (kShell1[o][1] + g.dims[1] * kShell1[o][2]);
        visit_range(s, cell, w, c);
      }
    }
    if (!kth.tie && c.n == min(found, a.k)) {
      blend_list<MODE>(a, s, p, q, col, c.n);
      return;
    }
  }
  Best<KMAX> best;
  best.init(a.k);
  const int found = knn_walk(g, s, a.k, q, best);
  blend_store<KMAX, MODE>(a, p, best, found);
}

// ---------------------------------------------------------------------------
// Warp-cooperative query: WORLD metric, pixels in spatial order, no neighbour
// list.  The 32 pixels of a warp are neighbours in the fine order, so they
// share most of their candidates.  The warp gathers once, into its own
// shared-memory buffer, every cache of the grid cells whose box lies within
// a radius rho of the box around its 32 points; each lane then scans the
// buffer (broadcast reads) for its k + 1 smallest keys
//   key = (bits of d^2 with the low 8 bits cleared) | buffer index,
// two integer min/max per slot per insertion.  The buffer holds every cache
// within rho of each of the warp's points, so a lane whose (k+1)-th distance
// is below rho (less a rounding margin) has its exact k + 1 nearest.  Lanes
// further out make the warp gather a second time, out to the largest radius
// they need, which settles them: their (k+1)-th distance can only fall.  A
// lane whose k-th and (k+1)-th keys agree above the index bits (a tie, or a
// near-tie within 2^-15 relative, at the cut), or a warp whose buffer would
// overflow, takes the exact per-thread (d^2, index) walk instead, so the
// selection is the exact one.  Gathered caches within the near distance of
// the box go to the front of the buffer and the rest to the back, so the
// scan meets close candidates first and later ones rarely insert.
static constexpr int COOP_CAP = 256;  // caches per warp buffer (8-bit index in the key)
static constexpr int COOP_WARPS = QUERY_THREADS / 32;
static constexpr unsigned kIdxBits = 0xffu;

// v as a cell coordinate in [0, dims - 1]; huge, infinite or NaN v are safe.
__device__ __forceinline__ int cell_coord(float v, int dims) {
  return (int)fminf(fmaxf(floorf(v), 0.f), (float)(dims - 1));
}

struct RowSet {
  int y0, y1, z0, z1;
};

// The rows (cy, cz) of cells that can lie within rho of the box [lo, hi].
__device__ __forceinline__ RowSet row_set(const GridHeader &g, const float (&lo)[3], const float (&hi)[3],
                                          float rho) {
  RowSet r;
  r.y0 = cell_coord((lo[1] - rho - g.origin[1]) * g.inv_h, g.dims[1]);
  r.y1 = cell_coord((hi[1] + rho - g.origin[1]) * g.inv_h, g.dims[1]);
  r.z0 = cell_coord((lo[2] - rho - g.origin[2]) * g.inv_h, g.dims[2]);
  r.z1 = cell_coord((hi[2] + rho - g.origin[2]) * g.inv_h, g.dims[2]);
  return r;
}

// Cells [x0, x1] of row (cy, cz) whose box lies within rho of the box
// [lo, hi] (x0 > x1: none; rho < 0: none).  A pure function of its
// arguments, monotone in rho, so the cells of a smaller radius are found
// again, and only they, when a larger gather leaves them out.
__device__ __forceinline__ void row_cells(const GridHeader &g, const float (&lo)[3], const float (&hi)[3],
                                          float rho, const RowSet &rs, int cy, int cz, int &x0, int &x1) {
  x0 = 1;
  x1 = 0;
  if (!(rho >= 0.f) || cy < rs.y0 || cy > rs.y1 || cz < rs.z0 || cz > rs.z1) return;
  const float by = g.origin[1] + (float)cy * g.h, bz = g.origin[2] + (float)cz * g.h;
  const float dy = fmaxf(fmaxf(by - hi[1], lo[1] - (by + g.h)), 0.f);
  const float dz = fmaxf(fmaxf(bz - hi[2], lo[2] - (bz + g.h)), 0.f);
  const float rem = rho * rho - (dy * dy + dz * dz);
  if (rem < 0.f) return;
  const float w = sqrtf(rem);
  x0 = cell_coord((lo[0] - w - g.origin[0]) * g.inv_h, g.dims[0]);
  x1 = cell_coord((hi[0] + w - g.origin[0]) * g.inv_h, g.dims[0]);
}

__device__ __forceinline__ float box_d2(const float (&lo)[3], const float (&hi)[3], float4 pt) {
  const float dx = fmaxf(fmaxf(lo[0] - pt.x, pt.x - hi[0]), 0.f);
  const float dy = fmaxf(fmaxf(lo[1] - pt.y, pt.y - hi[1]), 0.f);
  const float dz = fmaxf(fmaxf(lo[2] - pt.z, pt.z - hi[2]), 0.f);
  return dx * dx + dy * dy + dz * dz;
}

// Warp-wide: appends to the warp's buffer the caches within rho_out of the
// box [lo, hi] (box distance, squared, against rho_out^2) that an earlier
// call with rho_in did not take (rho_in < 0: none) -- those within the near
// distance upwards from nf, the others downwards from COOP_CAP - 1 - nb.  An
// earlier call took the caches within rho_in of the box from the cells
// within rho_in of it; this call reads the cells within rho_out and leaves
// out exactly those, so the two calls together hold each cache once.  One
// lane per row of cells: a row's selected cells are consecutive, so one
// contiguous range of the cell-ordered table, with the earlier call's cells
// a contiguous sub-range.  A buffer entry is (x, y, z, table slot bits).
// False (buffer unusable) when it would overflow.
__device__ bool coop_gather(const GridHeader &g, const InterpScratch &s, const float (&lo)[3],
                            const float (&hi)[3], float rho_in, float rho_out, float near2, float4 *buf, int &nf,
                            int &nb) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const RowSet ro = row_set(g, lo, hi, rho_out);
  const RowSet ri = row_set(g, lo, hi, rho_in);
  const float in2 = rho_in >= 0.f ? rho_in * rho_in : -1.f, out2 = rho_out * rho_out;
  const int ny = ro.y1 - ro.y0 + 1, nrows = ny * (ro.z1 - ro.z0 + 1);
  for (int r0 = 0; r0 < nrows; r0 += 32) {
    const int r = r0 + lane;
    int e = 0, e1 = 0, i0 = 0, i1 = 0;  // table range [e, e1), the earlier call's cells [i0, i1)
    if (r < nrows) {
      const int cy = ro.y0 + r % ny, cz = ro.z0 + r / ny;
      int ox0, ox1, ix0, ix1;
      row_cells(g, lo, hi, rho_out, ro, cy, cz, ox0, ox1);
      row_cells(g, lo, hi, rho_in, ri, cy, cz, ix0, ix1);
      if (ox0 <= ox1) {
        const int base = (cz * g.dims[1] + cy) * g.dims[0];
        e = __ldg(s.cell_start + base + ox0);
        e1 = __ldg(s.cell_start + base + ox1 + 1);
        if (ix0 <= ix1) {
          i0 = __ldg(s.cell_start + base + ix0);
          i1 = __ldg(s.cell_start + base + ix1 + 1);
        }
      }
    }
    for (;;) {
      const bool has = e < e1;
      if (!__any_sync(0xffffffffu, has)) break;
      float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);
      bool take = false, nr = false;
      if (has) {
        pt = __ldg(s.pts + e);
        const float bd2 = box_d2(lo, hi, pt);
        take = bd2 <= out2 && !(e >= i0 && e < i1 && bd2 <= in2);
        nr = bd2 <= near2;
        pt.w = __int_as_float(e);
        ++e;
      }
      const unsigned mf = __ballot_sync(0xffffffffu, take && nr), mb = __ballot_sync(0xffffffffu, take && !nr);
      if (nf + nb + __popc(mf) + __popc(mb) > COOP_CAP) return false;
      if (take) buf[nr ? nf + __popc(mf & lt) : COOP_CAP - 1 - nb - __popc(mb & lt)] = pt;
      nf += __popc(mf);
      nb += __popc(mb);
    }
  }
  return true;
}

// The lane's k + 1 smallest keys over buffer entries [i0, i1), four
// candidates' keys at a time (independent arithmetic), then their insertions.
template <int KC>
__device__ __forceinline__ void coop_insert(unsigned (&key)[KC], unsigned kc) {
  if (kc < key[KC - 1]) {
#pragma unroll
    for (int sl = KC - 1; sl > 0; --sl) key[sl] = min(key[sl], max(key[sl - 1], kc));
    key[0] = min(key[0], kc);
  }
}
__device__ __forceinline__ unsigned coop_key(const float4 *buf, int i, float3 q) {
  return (__float_as_uint(cand_d2(q, buf[i])) & ~kIdxBits) | (unsigned)i;
}
template <int KC>
__device__ __forceinline__ void coop_scan(const float4 *buf, int i0, int i1, float3 q, unsigned (&key)[KC]) {
  int i = i0;
  for (; i + 4 <= i1; i += 4) {
    const unsigned k0 = coop_key(buf, i, q), k1 = coop_key(buf, i + 1, q), k2 = coop_key(buf, i + 2, q),
                   k3 = coop_key(buf, i + 3, q);
    coop_insert<KC>(key, k0);
    coop_insert<KC>(key, k1);
    coop_insert<KC>(key, k2);
    coop_insert<KC>(key, k3);
  }
  for (; i < i1; ++i) coop_insert<KC>(key, coop_key(buf, i, q));
}

// An upper bound on the (k+1)-th squared distance from its key (the cleared
// low bits set), infinite while the list is not full.
__device__ __forceinline__ float kth_bound2(unsigned klast) {
  return klast == ~0u ? __int_as_float(0x7f800000) : __uint_as_float(klast | kIdxBits);
}

// Whether the lane's list is exact after gathering out to rho.
__device__ __forceinline__ bool coop_covered(unsigned klast, float rho, float rho_all, float margin) {
  if (rho >= rho_all) return true;
  const float c = rho - margin;
  return c > 0.f && kth_bound2(klast) <= c * c;
}

// Normalisation (Sec. 3.2) and blend from the k nearest keys, in ascending
// key order: w = w_p w_n + w_p + eps (Eq. 4) with the cache's unit normal
// and payload from the cell-ordered table (IRRADIANCE), or the map lookup of
// the generic path (LOOKUP); one reciprocal of the weight sum per pixel.
template <int KMAX, int MODE>
__device__ __forceinline__ void coop_blend(const InterpArgs &a, const InterpScratch &s, long long p, float3 q,
                                           const float4 *buf, const unsigned (&key)[KMAX + 1]) {
  const int m = KMAX - a.k;  // slot of the nearest (the (k+1)-th is slot KMAX)
  const PixelShade px = pixel_shade<MODE>(a, p);
  const float inl = px.nl > 0.f ? 1.f / px.nl : 0.f;
  const float pnx = px.nx * inl, pny = px.ny * inl, pnz = px.nz * inl;
  const bool inverse = a.wp_form == WP_INVERSE;
  const float delta = a.delta_rel * a.r, inv_r = 1.f / a.r;
  float wsum = 0.f, acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
#pragma unroll
  for (int sl = 0; sl < KMAX; ++sl) {
    if (sl >= m && key[sl] != ~0u) {
      const float4 pt = buf[key[sl] & kIdxBits];
      const int e = __float_as_int(pt.w);
      const float4 x0 = __ldg(s.aux + 2 * e);
      const float d = sqrtf(cand_d2(q, pt));
      const float wp = inverse ? a.r * __frcp_rn(d + delta) : fmaxf(0.f, 1.f - d * inv_r);
      const float wn = fmaxf(0.f, x0.x * pnx + x0.y * pny + x0.z * pnz);
      const float w = wp * wn + wp + a.eps;
      wsum += w;
      if constexpr (MODE == MODE_IRRADIANCE) {
        const float4 x1 = __ldg(s.aux + 2 * e + 1);
        acc0 += w * x0.w;
        acc1 += w * x1.x;
        acc2 += w * x1.y;
      } else {
        float3 v;
        if (nbr_value<MODE>(a, px, __float_as_int(__ldg(s.pts + e).w), v)) {
          acc0 += w * v.x;
          acc1 += w * v.y;
          acc2 += w * v.z;
        }
      }
    }
  }
  const float iw = __frcp_rn(wsum);
  a.out[3 * p] = acc0 * iw;
  a.out[3 * p + 1] = acc1 * iw;
  a.out[3 * p + 2] = acc2 * iw;
}

template <int KMAX, int MODE>
__global__ void __launch_bounds__(QUERY_THREADS, KMAX <= 16 ? 4 : 2) interp_coop_kernel(InterpArgs a, InterpScratch s) {
  constexpr int KC = KMAX + 1;
  __shared__ float4 sbuf[COOP_WARPS * COOP_CAP];
  float4 *buf = sbuf + (threadIdx.x >> 5) * COOP_CAP;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long P = (long long)a.width * a.height;
  const bool live = t < P;
  if (!__any_sync(0xffffffffu, live)) return;  // warp-uniform
  const GridHeader g = *s.hdr;
  const int k = a.k;
  const float4 o = live ? __ldg(s.order + t) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float3 q = make_float3(o.x, o.y, o.z);
  const long long p = live ? (long long)__float_as_int(o.w) : 0;
  float lo[3] = {live ? q.x : FLT_MAX, live ? q.y : FLT_MAX, live ? q.z : FLT_MAX};
  float hi[3] = {live ? q.x : -FLT_MAX, live ? q.y : -FLT_MAX, live ? q.z : -FLT_MAX};
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], sh));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], sh));
    }
  const float margin = 1e-3f * g.h;
  // gathering as far as the grid reaches from the box takes every cache
  float far2 = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float e = fmaxf(fmaxf(g.origin[d] + (float)g.dims[d] * g.h - lo[d], hi[d] - g.origin[d]), 0.f);
    far2 += e * e;
  }
  const float rho_all = sqrtf(far2) + 2.f * margin;
  const float near2 = g.coop_near * g.coop_near;
  unsigned key[KC];
#pragma unroll
  for (int sl = 0; sl < KC; ++sl) key[sl] = sl < KC - (k + 1) ? 0u : ~0u;
  int nf = 0, nb = 0;
  const float rho = fminf(g.coop_r0, rho_all);
  const bool ok = coop_gather(g, s, lo, hi, -1.f, rho, near2, buf, nf, nb);
  __syncwarp();
  bool covered = false;
  if (ok) {
    if (live) {
      coop_scan<KC>(buf, 0, nf, q, key);
      coop_scan<KC>(buf, COOP_CAP - nb, COOP_CAP, q, key);
    }
    covered = coop_covered(key[KC - 1], rho, rho_all, margin);
    const bool need = live && !covered;
    if (__any_sync(0xffffffffu, need)) {
      // the largest radius a lane still needs, then the caches out to it
      float rn = 0.f;
      if (need) rn = key[KC - 1] == ~0u ? rho_all : sqrtf(kth_bound2(key[KC - 1])) + 2.f * margin;
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) rn = fmaxf(rn, __shfl_xor_sync(0xffffffffu, rn, sh));
      const float rho1 = fminf(rn, rho_all);
      const int nf0 = nf, nb0 = nb;
      const bool ok2 = coop_gather(g, s, lo, hi, rho, rho1, near2, buf, nf, nb);
      __syncwarp();
      if (ok2 && need) {
        coop_scan<KC>(buf, nf0, nf, q, key);
        coop_scan<KC>(buf, COOP_CAP - nb, COOP_CAP - nb0, q, key);
        covered = coop_covered(key[KC - 1], rho1, rho_all, margin);
      }
    }
  }
  // a tie or near-tie at the cut: the exact walk orders it by (d^2, index)
  const bool tie = key[KC - 1] != ~0u && ((key[KC - 2] ^ key[KC - 1]) & ~kIdxBits) == 0u;
  if (!live) return;
  if (ok && covered && !tie) {
    coop_blend<KMAX, MODE>(a, s, p, q, buf, key);
    return;
  }
  Best<KMAX> best;
  best.init(k);
  const int found = knn_walk(g, s, k, q, best);
  blend_store<KMAX, MODE>(a, p, best, found);
}

// The cooperative query needs the pixel order (coherent warps); without it
// (no order scratch) the WORLD metric takes the per-thread two-walk query.
static inline bool use_coop(const InterpArgs &a, const InterpScratch &s) {
  return a.metric != METRIC_IMAGE && a.nbr_out == nullptr && s.order != nullptr;
}

template <int KMAX, int MODE>
static void launch_query(const InterpArgs &a, const InterpScratch &s, unsigned blocks, cudaStream_t st) {
  if (use_coop(a, s))
    interp_coop_kernel<KMAX, MODE><<<blocks, QUERY_THREADS, 0, st>>>(a, s);
  else if (a.metric != METRIC_IMAGE && a.nbr_out == nullptr)
    interp_query_kernel<KMAX, MODE, true><<<blocks, QUERY_THREADS, 0, st>>>(a, s);
  else
    interp_query_kernel<KMAX, MODE, false><<<blocks, QUERY_THREADS, 0, st>>>(a, s);
}

cudaError_t launch_interp(const InterpArgs &a_in, const InterpScratch &s, cudaStream_t st, Tracer *tr) {
  InterpArgs a = a_in;
  a.cell_caches = use_coop(a, s) ? kCoopPerCell : per_cell(a.k);
  a.coop_rho = kCoopRho;
  a.coop_near = kCoopNear;
  // Tuning knob for measurements: DRC_INTERP_COOP="caches_per_cell,rho,near"
  // overrides the cooperative query's grid and radii (same results).
  if (use_coop(a, s)) {
    if (const char *e = std::getenv("DRC_INTERP_COOP")) {
      int pc = 0;
      float rho = 0.f, nr = 0.f;
      if (sscanf(e, "%d,%f,%f", &pc, &rho, &nr) == 3 && pc >= 1 && rho > 0.f && nr >= 0.f) {
        a.cell_caches = pc < kCoopPerCell ? pc : kCoopPerCell;  // the scratch is sized for kCoopPerCell
        a.coop_rho = rho;
        a.coop_near = nr;
      }
    }
  }
  DRC_TRACED(tr, "interp grid_bounds", st, (grid_bounds_kernel<<<1, 1024, 0, st>>>(a, s)));
  const int cb = (a.n + 255) / 256;
  DRC_TRACED(tr, "interp grid_count", st, (grid_count_kernel<<<cb, 256, 0, st>>>(a, s)));
  DRC_TRACED(tr, "interp grid_scan", st, (scan_kernel<<<1, SCAN_THREADS, 0, st>>>(&s.hdr->ncells, s.cell_count, s.cell_start)));
  DRC_TRACED(tr, "interp grid_scatter", st, (grid_scatter_kernel<<<cb, 256, 0, st>>>(a, s)));
  const long long P = (long long)a.width * a.height;
  if (P == 0) return cudaGetLastError();
  const unsigned blocks = (unsigned)((P + 255) / 256);
  if (s.order) {
    DRC_TRACED(tr, "interp pixel_count", st, (pixel_count_kernel<<<blocks, 256, 0, st>>>(a, s)));
    const unsigned tiles = (unsigned)fine_tiles(s.max_fine);
    DRC_TRACED(tr, "interp pixel_scan", st,
               (scan_sum_kernel<<<tiles, SCAN_THREADS, 0, st>>>(&s.hdr->nfine, s.fine_count, s.fine_tile_sum)));
    DRC_TRACED(tr, "interp pixel_scan", st,
               (scan_tiles_kernel<<<tiles, SCAN_THREADS, 0, st>>>(&s.hdr->nfine, s.fine_count, s.fine_tile_sum)));
    DRC_TRACED(tr, "interp pixel_scatter", st, (pixel_scatter_kernel<<<blocks, 256, 0, st>>>(a, s)));
  }
  const unsigned qblocks = (unsigned)((P + QUERY_THREADS - 1) / QUERY_THREADS);
  if (tr) tr->begin("interp query", st);
  if (a.mode == MODE_IRRADIANCE) {
    if (a.k <= 8)
      launch_query<8, MODE_IRRADIANCE>(a, s, qblocks, st);
    else if (a.k <= 16)
      launch_query<16, MODE_IRRADIANCE>(a, s, qblocks, st);
    else
      launch_query<32, MODE_IRRADIANCE>(a, s, qblocks, st);
  } else {
    if (a.k <= 8)
      launch_query<8, 1>(a, s, qblocks, st);
    else if (a.k <= 16)
      launch_query<16, 1>(a, s, qblocks, st);
    else
      launch_query<32, 1>(a, s, qblocks, st);
  }
  if (tr) tr->end(st);
  return cudaGetLastError();
}

}  // namespace drc
