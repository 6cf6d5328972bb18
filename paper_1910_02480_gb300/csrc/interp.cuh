// interp.cuh -- radiance-cache interpolation (Sec. 3.2): uniform grid over the
// caches, exact k-nearest selection per pixel, the weight w = w_p w_n + w_p +
// eps, normalisation and the blend of payloads or map lookups.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "trace.cuh"

namespace drc {

struct GridHeader {
  float origin[3];
  float h, inv_h;      // coarse cells (InterpArgs::cell_caches caches each)
  int dims[3];
  int ncells;
  float fine_inv_h;    // fine cells for ordering the pixels (about 32 pixels each)
  int fdims[3];
  int nfine;
  // warp-cooperative query: the radius of the first gather around a warp's
  // points and the distance within which a gathered cache is scanned first
  float coop_r0, coop_near;
};

// Device scratch used by one interpolation call.
struct InterpScratch {
  GridHeader *hdr;
  int *cell_count;   // [max_cells] counts, then write cursors
  int *cell_start;   // [max_cells + 1]
  int *cache_cell;   // [n]
  float4 *pts;       // [n] (x, y, z, index bits) in cell order
  int max_cells;
  // optional pixel ordering (nullptr: pixels are processed in index order)
  int *fine_count;     // [max_fine] counts, then cursors
  int *fine_tile_sum;  // [max_fine / 16384, rounded up] per-tile totals of the counts
  float4 *order;       // [P] (x, y, z, pixel index bits) sorted by fine cell
  int max_fine;
  // with the ordering: per cache, in the cell order of pts, the unit normal
  // (0 for a zero-length one) and the payload: aux[2 e] = (nx, ny, nz, E0),
  // aux[2 e + 1] = (E1, E2, 0, 0); read by the warp-cooperative blend
  float4 *aux;
};

// Grid scratch for n caches (no pixel ordering).
size_t interp_scratch_bytes(int n, int k);
int interp_max_cells(int n, int k);
InterpScratch interp_carve(void *base, int n, int k);
// Extra scratch that orders P pixels spatially before the search (same
// results, better warp coherence); attach to a carved InterpScratch.
size_t interp_order_bytes(long long P, int n);
void interp_attach_order(InterpScratch &s, void *base, long long P, int n);

struct InterpArgs {
  int n, mapH, mapW;
  const float *maps, *payload, *cpos, *cnrm;
  const int *cpix;
  int width, height;
  const float *gpos, *gnrm, *gdir;
  int k, metric, wp_form, mode;
  float r, eps, delta_rel;
  float *out;
  int *nbr_out;
  float *nbr_w;      // with nbr_out: the normalised weights
  // set by launch_interp: caches per grid cell the grid is sized for, and
  // the cooperative query's first-gather radius and near distance, in units
  // of the expected distance to the (k+1)-th nearest cache
  int cell_caches;
  float coop_rho, coop_near;
};

// tr: nullable launch tracer (counts and optionally times each kernel).
cudaError_t launch_interp(const InterpArgs &a, const InterpScratch &s, cudaStream_t st, Tracer *tr = nullptr);

}  // namespace drc
