// mapgen.cu -- the denoiser's input maps traced on the GPU (Sec. 3.1-3.3).
//
// The paper traces, at each cache point (a first non-specular intersection),
// a hemispherical map of the indirect light arriving there: radiance, the
// distance to what is seen and that surface's normal (Sec. 3.3's seven
// channels), with the direct light left out of the radiance (Sec. 3.2: it
// is added back by a separate pass).  The scene here is an analytic interior
// (the paper's scenes are not available): the unit box [0,1]^3 of six
// diffuse walls (albedo and emission each, in the order -x, +x, -y, +y, -z,
// +z), an emitting rectangle on the ceiling z = 1, and diffuse spheres seen
// from outside.
//
// One thread per texel (a, b) of cache j: one ray from the cache point along
// the texel's centre direction -- polar angle (a + 1/2) pi / 2H from the
// cache normal, azimuth (b + 1/2) 2 pi / W in the cache frame (up = +Z, or
// +Y when the normal is along Z; t = up x n normalised, b = n x t).  The
// first hit gives the distance and the normal facing the ray; the radiance
// is that of a path of D bounces from the first hit, each a cosine-weighted
// direction about the current normal (a frame of the same rule), adding the
// throughput times the next hit's emission and multiplying the throughput by
// that hit's albedo (the Lambertian one-sample estimate), so the first hit's
// own emission is left out.  The uniforms u[j][a][b][k] = (u0, u1) of
// bounce k are an input.  A ray that leaves the box (not possible from
// inside) or a cache with a zero normal writes zeros.
#include <cuda_runtime.h>

#include "mapgen.cuh"

namespace drc {

static constexpr int GEN_THREADS = 256;
static constexpr float kPiF = 3.14159265358979f;

__device__ __forceinline__ bool gen_frame(float nx, float ny, float nz, float3 &t, float3 &b, float3 &n) {
  const float len = sqrtf(nx * nx + ny * ny + nz * nz);
  if (!(len > 0.f)) return false;
  n = make_float3(nx / len, ny / len, nz / len);
  float ux = 0.f, uy = 0.f, uz = 1.f;
  if (fabsf(n.z) > 1.f - 1e-6f) {
    uy = 1.f;
    uz = 0.f;
  }
  const float cx = uy * n.z - uz * n.y, cy = uz * n.x - ux * n.z, cz = ux * n.y - uy * n.x;
  const float cl = sqrtf(cx * cx + cy * cy + cz * cz);
  t = make_float3(cx / cl, cy / cl, cz / cl);
  b = make_float3(n.y * t.z - n.z * t.y, n.z * t.x - n.x * t.z, n.x * t.y - n.y * t.x);
  return true;
}

struct Hit {
  float t;
  float3 n, alb, em;
};

// Nearest hit of o + t d (t > 0): the wall ahead on each axis, and every
// sphere with the origin outside it.
__device__ __forceinline__ bool gen_hit(const drc_scene &sc, float3 o, float3 d, Hit &h) {
  float best = __int_as_float(0x7f800000);
  int which = -1;  // 0..5 wall, 6 + s sphere s
  const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (dd[i] > 0.f) {
      const float t = (1.f - oo[i]) / dd[i];
      if (t > 1e-12f && t < best) {
        best = t;
        which = 2 * i + 1;
      }
    } else if (dd[i] < 0.f) {
      const float t = -oo[i] / dd[i];
      if (t > 1e-12f && t < best) {
        best = t;
        which = 2 * i;
      }
    }
  }
  // Spheres: with oc = o - centre and B = oc . d, the ray meets the sphere at
  // t = -B - sqrt(r^2 - |oc - B d|^2): the discriminant written through the
  // ray's closest approach, |oc - B d|, rather than as B^2 - (|oc|^2 - r^2),
  // which in float32 cancels badly for grazing rays.
  for (int s = 0; s < sc.nsph; ++s) {
    const float *sp = sc.sph[s];
    const float ox = o.x - sp[0], oy = o.y - sp[1], oz = o.z - sp[2];
    const float B = ox * d.x + oy * d.y + oz * d.z;
    const float C = ox * ox + oy * oy + oz * oz - sp[3] * sp[3];
    const float px = ox - B * d.x, py = oy - B * d.y, pz = oz - B * d.z;
    const float disc = sp[3] * sp[3] - (px * px + py * py + pz * pz);
    if (C <= 0.f || disc < 0.f) continue;  // seen from outside only
    const float t = -B - sqrtf(disc);
    if (t > 1e-12f && t < best) {
      best = t;
      which = 6 + s;
    }
  }
  if (which < 0) return false;
  h.t = best;
  const float hx = o.x + best * d.x, hy = o.y + best * d.y, hz = o.z + best * d.z;
  if (which < 6) {
    const int axis = which >> 1;
    const float sgn = (which & 1) ? -1.f : 1.f;  // inward
    h.n = make_float3(axis == 0 ? sgn : 0.f, axis == 1 ? sgn : 0.f, axis == 2 ? sgn : 0.f);
    h.alb = make_float3(sc.wall_alb[which][0], sc.wall_alb[which][1], sc.wall_alb[which][2]);
    h.em = make_float3(sc.wall_em[which][0], sc.wall_em[which][1], sc.wall_em[which][2]);
    if (which == 5 && sc.has_light && hx >= sc.light[0] && hx <= sc.light[1] && hy >= sc.light[2] &&
        hy <= sc.light[3]) {
      h.em.x += sc.light[4];
      h.em.y += sc.light[5];
      h.em.z += sc.light[6];
    }
  } else {
    const float *sp = sc.sph[which - 6];
    // hit - centre = oc + t d (no cancellation against the centre)
    h.n = make_float3((o.x - sp[0] + best * d.x) / sp[3], (o.y - sp[1] + best * d.y) / sp[3],
                      (o.z - sp[2] + best * d.z) / sp[3]);
    h.alb = make_float3(sp[4], sp[5], sp[6]);
    h.em = make_float3(0.f, 0.f, 0.f);
  }
  return true;
}

__global__ void __launch_bounds__(GEN_THREADS) gen_maps_kernel(const __grid_constant__ MapGenArgs a) {
  const long long HW = (long long)a.H * a.W;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)a.n * HW) return;
  const int j = (int)(tid / HW);
  const long long e = tid - (long long)j * HW;
  const int ar = (int)(e / a.W), bc = (int)(e - (long long)ar * a.W);
  float *out = a.maps + (size_t)j * 7 * HW + e;
  float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float3 ft, fb, fn;
  if (gen_frame(__ldg(a.nrm + 3 * j), __ldg(a.nrm + 3 * j + 1), __ldg(a.nrm + 3 * j + 2), ft, fb, fn)) {
    const float3 x = make_float3(__ldg(a.pos + 3 * j), __ldg(a.pos + 3 * j + 1), __ldg(a.pos + 3 * j + 2));
    float st, ct, sp, cp;
    sincosf(((float)ar + 0.5f) * (0.5f * kPiF / (float)a.H), &st, &ct);
    sincosf(((float)bc + 0.5f) * (2.f * kPiF / (float)a.W), &sp, &cp);
    const float lx = st * cp, ly = st * sp;
    const float3 d = make_float3(lx * ft.x + ly * fb.x + ct * fn.x, lx * ft.y + ly * fb.y + ct * fn.y,
                                 lx * ft.z + ly * fb.z + ct * fn.z);
    Hit h;
    if (gen_hit(a.scene, x, d, h)) {
      v[3] = h.t;
      v[4] = h.n.x;
      v[5] = h.n.y;
      v[6] = h.n.z;
      // the path from the first hit, its own emission left out
      float3 thr = h.alb, L = make_float3(0.f, 0.f, 0.f);
      float3 o = make_float3(x.x + h.t * d.x, x.y + h.t * d.y, x.z + h.t * d.z);
      float3 nc = h.n;
      const float2 *u = a.u + tid * a.D;
      for (int k = 0; k < a.D; ++k) {
        const float2 uk = __ldg(u + k);
        float3 tt, bb, n2;
        gen_frame(nc.x, nc.y, nc.z, tt, bb, n2);
        const float rr = sqrtf(uk.x), lz = sqrtf(fmaxf(1.f - uk.x, 0.f));
        float s2, c2;
        sincosf(2.f * kPiF * uk.y, &s2, &c2);
        const float px = rr * c2, py = rr * s2;
        const float3 dn = make_float3(px * tt.x + py * bb.x + lz * nc.x, px * tt.y + py * bb.y + lz * nc.y,
                                      px * tt.z + py * bb.z + lz * nc.z);
        Hit h2;
        if (!gen_hit(a.scene, o, dn, h2)) break;
        L.x += thr.x * h2.em.x;
        L.y += thr.y * h2.em.y;
        L.z += thr.z * h2.em.z;
        thr.x *= h2.alb.x;
        thr.y *= h2.alb.y;
        thr.z *= h2.alb.z;
        o = make_float3(o.x + h2.t * dn.x, o.y + h2.t * dn.y, o.z + h2.t * dn.z);
        nc = h2.n;
      }
      v[0] = L.x;
      v[1] = L.y;
      v[2] = L.z;
    }
  }
#pragma unroll
  for (int c = 0; c < 7; ++c) out[c * HW] = v[c];
}

cudaError_t launch_gen_maps(const MapGenArgs &a, cudaStream_t st, Tracer *tr) {
  const long long total = (long long)a.n * a.H * a.W;
  if (total == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((total + GEN_THREADS - 1) / GEN_THREADS);
  DRC_TRACED(tr, "gen maps", st, (gen_maps_kernel<<<blocks, GEN_THREADS, 0, st>>>(a)));
  return cudaGetLastError();
}

}  // namespace drc
