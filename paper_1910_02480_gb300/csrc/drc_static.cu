// drc_static.cu -- drc_interpolate_static: the interpolation of drc_interpolate
// for callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application that owns the whole
// device-memory budget and gives plugins none of their own, or a frame loop in
// which cudaMalloc's implicit device synchronisation is not allowed.  This
// entry point needs no context and allocates nothing: the cache grid it builds
// lives in the file-scope device array below (kStaticScratchBytes, held by
// every GPU that loads the library until the process exits).  Inputs and the
// output are still the caller's.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "drc.h"
#include "interp.cuh"

using namespace drc;

namespace {

constexpr size_t kStaticScratchBytes = 3u << 20;  // 3 MiB
constexpr int kStaticMaxCaches = 65536;            // fits kStaticScratchBytes for every k

// The grid scratch.  In host code this name is only a stand-in: its device
// address comes from cudaGetSymbolAddress, looked up on every call with the
// caller's device current.  The lookup is a host-side table read, and it is
// not cached: after cudaDeviceReset, or under another context on the same
// device, the module is loaded again and the array may move.
static __device__ __align__(256) unsigned char g_interp_scratch[kStaticScratchBytes];

bool device_ptr_ok(const void *p, int device) {
  if (!p || (reinterpret_cast<uintptr_t>(p) & 15u)) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice) return at.device == device;
  return at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" drc_status drc_interpolate_static(const drc_caches *caches, const drc_gbuffer *gbuf,
                                              const drc_interp_params *prm, float *out_rgb, void *stream) {
  if (!caches || !gbuf || !prm) return DRC_ERR_INVALID_ARG;
  if (caches->n < 1 || caches->n > kStaticMaxCaches) return DRC_ERR_INVALID_ARG;
  if (prm->k < 1 || prm->k > 32) return DRC_ERR_INVALID_ARG;
  if (prm->metric != DRC_METRIC_IMAGE && prm->metric != DRC_METRIC_WORLD) return DRC_ERR_INVALID_ARG;
  if (prm->wp_form != DRC_WP_INVERSE && prm->wp_form != DRC_WP_LINEAR) return DRC_ERR_INVALID_ARG;
  if (prm->mode != DRC_INTERP_IRRADIANCE && prm->mode != DRC_INTERP_LOOKUP) return DRC_ERR_INVALID_ARG;
  if (!(prm->r > 0.f) || !(prm->eps >= 0.f) || !(prm->delta_rel > 0.f)) return DRC_ERR_INVALID_ARG;
  if (gbuf->width < 0 || gbuf->height < 0) return DRC_ERR_INVALID_ARG;
  const long long P = (long long)gbuf->width * gbuf->height;
  if (P >= (1ll << 31) / 3) return DRC_ERR_INVALID_ARG;
  if (interp_scratch_bytes(caches->n, prm->k) > kStaticScratchBytes) return DRC_ERR_INVALID_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return DRC_ERR_CUDA;
  }
  const bool world = prm->metric == DRC_METRIC_WORLD;
  const bool lookup = prm->mode == DRC_INTERP_LOOKUP;
  if (!device_ptr_ok(world ? (const void *)caches->pos : (const void *)caches->pix, dev)) return DRC_ERR_INVALID_ARG;
  if (!device_ptr_ok(caches->nrm, dev)) return DRC_ERR_INVALID_ARG;
  if (lookup) {
    if (caches->H < 1 || caches->W < 1 || !device_ptr_ok(caches->maps, dev)) return DRC_ERR_INVALID_ARG;
  } else if (!device_ptr_ok(caches->payload, dev)) {
    return DRC_ERR_INVALID_ARG;
  }
  if (P > 0) {
    if (!device_ptr_ok(out_rgb, dev) || !device_ptr_ok(gbuf->nrm, dev)) return DRC_ERR_INVALID_ARG;
    if (world && !device_ptr_ok(gbuf->pos, dev)) return DRC_ERR_INVALID_ARG;
    if (lookup && !device_ptr_ok(gbuf->dir, dev)) return DRC_ERR_INVALID_ARG;
    if (prm->nbr_out && !device_ptr_ok(prm->nbr_out, dev)) return DRC_ERR_INVALID_ARG;
    if (prm->nbr_w && (!prm->nbr_out || !device_ptr_ok(prm->nbr_w, dev))) return DRC_ERR_INVALID_ARG;
  }

  // The array's address in the current context.  The first call in a
  // context may load the library's module, so make it before any stream
  // capture.
  void *scratch = nullptr;
  if (cudaGetSymbolAddress(&scratch, g_interp_scratch) != cudaSuccess || !scratch) {
    cudaGetLastError();
    return DRC_ERR_CUDA;
  }

  InterpArgs a;
  memset(&a, 0, sizeof a);
  a.n = caches->n;
  a.mapH = caches->H;
  a.mapW = caches->W;
  a.maps = caches->maps;
  a.payload = caches->payload;
  a.cpos = caches->pos;
  a.cnrm = caches->nrm;
  a.cpix = caches->pix;
  a.width = gbuf->width;
  a.height = gbuf->height;
  a.gpos = gbuf->pos;
  a.gnrm = gbuf->nrm;
  a.gdir = gbuf->dir;
  a.k = prm->k;
  a.metric = prm->metric;
  a.wp_form = prm->wp_form;
  a.mode = prm->mode;
  a.r = prm->r;
  a.eps = prm->eps;
  a.delta_rel = prm->delta_rel;
  a.out = out_rgb;
  a.nbr_out = prm->nbr_out;
  a.nbr_w = prm->nbr_w;
  // The grid kernels rewrite every part of the scratch they read (the cell
  // counts are cleared first), so nothing is left over from an earlier call.
  const InterpScratch sc = interp_carve(scratch, caches->n, prm->k);
  if (launch_interp(a, sc, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return DRC_ERR_CUDA;
  }
  return DRC_OK;
}
