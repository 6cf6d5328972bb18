// interp.cuh -- radiance-cache interpolation (Sec. 3.2): uniform grid over the
// caches, exact k-nearest selection per pixel, the weight w = w_p w_n + w_p +
// eps, normalisation and the blend of payloads or map lookups.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace drc {

struct GridHeader {
  float origin[3];
  float h, inv_h;
  int dims[3];
  int ncells;
  int pad_;
};

// Device scratch used by one interpolation call, carved from one buffer.
struct InterpScratch {
  GridHeader *hdr;
  int *cell_count;   // [max_cells] counts, then write cursors
  int *cell_start;   // [max_cells + 1]
  int *cache_cell;   // [n]
  float4 *pts;       // [n] (x, y, z, index bits) in cell order
  int max_cells;
};

// Bytes of scratch for n caches and the cell budget chosen for them.
size_t interp_scratch_bytes(int n, int k);
int interp_max_cells(int n, int k);
InterpScratch interp_carve(void *base, int n, int k);

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
};

cudaError_t launch_interp(const InterpArgs &a, const InterpScratch &s, cudaStream_t st);

}  // namespace drc
