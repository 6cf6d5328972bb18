/*
 * drc.h -- C ABI of the Deep Radiance Caching hot path on one GB300 (sm_103a).
 *
 * Method: Jiang & Kainz, "Deep Radiance Caching: Convolutional Autoencoders
 * Deeper in Ray Tracing" (arXiv 1910.02480).  Two operations:
 *   - denoise:      a convolutional autoencoder maps noisy low-sample
 *                   hemispherical radiance maps (radiance RGB, distance,
 *                   normal) to denoised radiance maps (Sec. 3.3);
 *   - interpolate:  every first-hit pixel blends the k nearest cached maps
 *                   with the weight w = w_p * w_n + w_p + eps, normalised
 *                   (Sec. 3.2, Eqs. 4-6);
 *   plus the gradient of an L1 loss through the autoencoder for training
 *   (Sec. 3.3 loss, Sec. 4 training).
 *
 * Conventions for every call:
 *   - Tensor pointers are caller-owned DEVICE memory on the context's device,
 *     contiguous, 16-byte aligned, not overlapping unless stated.
 *   - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *     stream) and is asynchronous.  Argument errors are detected on the host
 *     and returned before anything is enqueued.
 *   - Errors raised on the device (a bounded wait that ran out) are latched in
 *     a per-context status word and returned by drc_get_status().
 *   - A context is used by one host thread at a time.  No C++ exception
 *     crosses this interface.
 */
#ifndef DRC_H_
#define DRC_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DRC_OK = 0,
  DRC_ERR_INVALID_ARG = 1, /* bad pointer, shape, flag or configuration */
  DRC_ERR_UNSUPPORTED = 2, /* valid request this build does not implement */
  DRC_ERR_OOM = 3,         /* device allocation failed */
  DRC_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  DRC_ERR_TIMEOUT = 5,     /* a device-side wait ran out (latched) */
  DRC_ERR_INTERNAL = 6
} drc_status;

typedef enum {
  DRC_PREC_FP32 = 0, /* fp32 operands split into two tf32 parts (3 products) */
  DRC_PREC_BF16 = 1,
  DRC_PREC_FP8_E4M3 = 2
} drc_precision;

/* Network description.  The autoencoder of Sec. 3.3 in the form used here:
 * encoder stage s (s = 1..S): e_s = ReLU(conv3x3, stride 2, pad 1 (e_{s-1}) + b);
 * decoder stage s (s = S..2): t_{s-1} = ReLU(convT3x3, stride 2, pad 1,
 * output pad 1 (t_s) + b) + e_{s-1}  (t_S = e_S, skip added after the ReLU);
 * head: out = convT3x3 s2 (t_1) + b, followed by ReLU when out_relu. */
typedef struct {
  int in_channels;  /* must be 7: [0..2] radiance (log), [3] distance, [4..6] normal */
  int out_channels; /* must be 3 */
  int num_stages;   /* S, 1..6 */
  int widths[8];    /* encoder widths c_1..c_S; multiples of 16, <= 1024 */
  int out_relu;     /* 0: linear head (default); 1: ReLU head (the paper's) */
  drc_precision precision;
  float exposure;    /* s in the log encode log1p(s L) / decode expm1(y)/s; > 0 */
  int max_maps;      /* workspace sizing hint: largest N per call (grown on demand) */
  int max_hw;        /* workspace sizing hint: largest H*W per map */
  int wait_timeout_ms; /* bound on every device-side wait; 0 = 2000 ms */
} drc_config;

typedef struct drc_ctx drc_ctx;

/* Packed weights: layers conv_1..conv_S then convT_S..convT_1, each as W
 * followed by b, float32.  conv W is [Cout][Cin][3][3], convT W is
 * [Cin][Cout][3][3] (the PyTorch Conv2d / ConvTranspose2d layouts).
 * n_floats must equal sum over layers of 9*Cin*Cout + Cout. */
size_t drc_weight_count(const drc_config *cfg);

/* Create a context on the current CUDA device.  `weights_host` (host memory,
 * n_floats floats, read during the call) may be NULL, in which case weights
 * must be set with drc_set_weights before the first denoise.  On success
 * *out owns all device memory it allocates; release it with drc_destroy. */
drc_status drc_create(const drc_config *cfg, const float *weights_host,
                      size_t n_floats, drc_ctx **out);

/* Replace the weights: `weights` holds drc_weight_count() floats in host
 * memory (weights_on_device = 0; copied before return) or device memory
 * (weights_on_device = 1; read on `stream`).  Re-packs the tensor-core
 * operand tiles on `stream`.  Setting weights from device memory does not
 * synchronise: until the next drc_denoise, drc_frame_host or plan capture
 * (which synchronises `stream` once to copy the output head's weights to the
 * host, where its kernel takes them as launch parameters), the head reads
 * its weights from device memory, as drc_backward does after such an
 * update. */
drc_status drc_set_weights(drc_ctx *ctx, const float *weights,
                           int weights_on_device, void *stream);

drc_status drc_destroy(drc_ctx *ctx);

/* drc_denoise flags */
#define DRC_F_ENCODE_INPUT 0x1u  /* apply log1p(s L) to input channels 0..2 */
#define DRC_F_DECODE_OUTPUT 0x2u /* write expm1(y)/s instead of log-space y */
#define DRC_F_DEBUG_STALL 0x100u /* test only: the first device wait never
                                    completes; the call's kernels give up after
                                    the context's wait timeout and latch
                                    DRC_ERR_TIMEOUT (output undefined) */

/* Denoise N maps (Sec. 3.3).
 *   in:      device [N][7][H][W] float32 (NCHW), log radiance unless
 *            DRC_F_ENCODE_INPUT;
 *   out:     device [N][3][H][W] float32, log radiance unless
 *            DRC_F_DECODE_OUTPUT;
 *   payload: nullable; device [N][3] float32, overwritten with E/pi of the
 *            decoded map (linear radiance expm1(y)/s): the irradiance a
 *            white diffuse surface receives from the map, divided by pi
 *            (Eq. 2 with a Lambertian BRDF).  Lat-long layout: row i spans
 *            polar angle [i, i+1] * pi/(2H) from the normal, column j
 *            azimuth [j, j+1] * 2 pi / W.
 * H and W must be multiples of 2^S and at least 2^S; N >= 0 (0 is a no-op). */
drc_status drc_denoise(drc_ctx *ctx, const float *in, float *out,
                       float *payload, int N, int H, int W, unsigned flags,
                       void *stream);

/* Caches for interpolation (Sec. 3.2). */
typedef struct {
  int n;              /* number of caches, >= 1 */
  int H, W;           /* map size (LOOKUP only) */
  const float *maps;  /* LOOKUP: device [n][3][H][W] linear radiance, else NULL */
  const float *payload; /* IRRADIANCE: device [n][3], else may be NULL */
  const float *pos;   /* device [n][3] first-hit position (WORLD metric) */
  const float *nrm;   /* device [n][3] surface normal (any length; 0 = none) */
  const int *pix;     /* device [n][2] (x, y) integer pixel (IMAGE metric) */
} drc_caches;

typedef struct {
  int width, height;  /* pixel p = y * width + x */
  const float *pos;   /* device [P][3] first-hit position (WORLD metric) */
  const float *nrm;   /* device [P][3] surface normal */
  const float *dir;   /* LOOKUP: device [P][3] world direction (normalised by
                         the callee), else NULL */
} drc_gbuffer;

#define DRC_METRIC_IMAGE 0  /* distance in pixels on the image plane (the paper's) */
#define DRC_METRIC_WORLD 1  /* distance between first-hit positions */
#define DRC_WP_INVERSE 0    /* w_p = r / (d + delta_rel * r) */
#define DRC_WP_LINEAR 1     /* w_p = max(0, 1 - d / r) */
#define DRC_INTERP_IRRADIANCE 0 /* out = sum_j W_j payload_j */
#define DRC_INTERP_LOOKUP 1     /* out = sum_j W_j R_j(dir in cache j's frame) */

typedef struct {
  int k;          /* neighbours, 1..32 */
  int metric;     /* DRC_METRIC_* */
  int wp_form;    /* DRC_WP_* */
  int mode;       /* DRC_INTERP_* */
  float r;        /* grid spacing (pixels or world units), > 0 */
  float eps;      /* the small term of Eq. 4, >= 0 (1e-6 typical) */
  float delta_rel;/* INVERSE softening, delta = delta_rel * r, > 0 */
  int *nbr_out;   /* nullable; device [P][k] int32, the chosen cache indices
                     in (d^2, index) order (-1 past the number of caches) */
  float *nbr_w;   /* nullable (needs nbr_out); device [P][k] float32, the
                     normalised weights W_j of those caches (0 past the number
                     of caches): the map-choice probabilities drc_indirect
                     samples with */
} drc_interp_params;

/* Interpolate cached values at every pixel (Sec. 3.2).  For each pixel: the
 * k caches nearest by (d^2, index) order; w_p as selected; w_n =
 * max(0, n_j . n_p) for unit normals (0 for a zero-length normal);
 * w = w_p w_n + w_p + eps; W_j = w_j / sum w; out = sum W_j value_j.
 * LOOKUP: value_j = bilinear lookup of map j at the pixel direction in cache
 * j's frame (normal = map Z; up = +Z, or +Y when the normal is along Z;
 * t = normalize(up x n), b = n x t), 0 when the direction is not above the
 * cache's horizon.
 * out_rgb: device [P][3] float32.  The context keeps a grid over the caches
 * in its own device memory (grown on demand). */
drc_status drc_interpolate(drc_ctx *ctx, const drc_caches *caches,
                           const drc_gbuffer *gbuf,
                           const drc_interp_params *params, float *out_rgb,
                           void *stream);

/* drc_interpolate without a context and without allocating.  The paper has
 * no counterpart: this serves callers that cannot call cudaMalloc -- a host
 * application that owns the device-memory budget and gives plugins none of
 * their own, or a frame loop in which cudaMalloc's implicit device
 * synchronisation is not allowed.
 *   Same arguments and result as drc_interpolate.  The cache grid lives in a
 *   3 MiB static device array of the library (held on every GPU that loads
 *   the library until the process exits); n may be at most 65536 caches (any
 *   k); larger n returns DRC_ERR_INVALID_ARG before anything is enqueued.
 *   Argument errors return DRC_ERR_INVALID_ARG, a failed CUDA call
 *   DRC_ERR_CUDA.  Allocates no device memory (no cudaMalloc, cudaFree or
 *   allocating library routine).
 *   Every call looks up the array's device address in the current context
 *   (cudaGetSymbolAddress, a host-side lookup).  The first call in a context
 *   may load the library's module: make it before any stream capture.
 *   For the WORLD metric this path does not reorder the pixels spatially
 *   (that ordering needs a scratch array as large as the G-buffer): the
 *   result is the same, but an incoherent G-buffer is searched more slowly
 *   than by drc_interpolate.
 *   Every call shares the one array: calls that overlap on the GPU (different
 *   streams, different host threads) race and their results are undefined;
 *   calls ordered on one stream are safe, since each call rewrites all the
 *   scratch it reads. */
drc_status drc_interpolate_static(const drc_caches *caches, const drc_gbuffer *gbuf,
                                  const drc_interp_params *params, float *out_rgb,
                                  void *stream);

/* The indirect term of Eq. 3 at every pixel, by multiple importance
 * sampling (Sec. 3.2): R, the blend of the pixel's k caches' maps by their
 * normalised weights, is sampled as an environment map with perfect
 * visibility for even samples s and the BRDF (Lambertian, f_r = albedo / pi,
 * cosine-weighted about the pixel normal) for odd s; each sample first
 * draws one of the k maps with probability W_j, and contributes
 * f_r cos R / (n_env pdf_env + n_brdf pdf_brdf) (balance heuristic, sample
 * counts n_env = ceil(S/2), n_brdf = floor(S/2)).  Environment sampling
 * takes a texel with probability proportional to its luminance
 * (0.2126 R + 0.7152 G + 0.0722 B) times its solid angle, then a direction
 * uniform in solid angle inside it.  Texel (a, b) of a map covers polar
 * angles [a, a+1) pi/2H from the cache normal and azimuths [b, b+1) 2 pi/W in
 * the cache frame of drc_interpolate's LOOKUP mode.
 *   out = emit + direct + the estimate (Eq. 3: L_e, the direct-light integral
 *   of the renderer's own pass, and the indirect integral over R).
 * caches: n, H (<= 256), W, maps (device [n][3][H][W] LINEAR radiance, e.g.
 * drc_denoise with DRC_F_DECODE_OUTPUT) and nrm (device [n][3]).  gbuf:
 * width, height, nrm (device [P][3]).  out_rgb: device [P][3].  Uniforms and
 * neighbours are inputs, so a call is deterministic.  The context keeps the
 * maps' CDFs and frames in its own device memory (grown on demand).
 * INVALID_ARG for k outside 1..32, S outside 1..4096, H > 256, host or
 * unaligned pointers; asynchronous on `stream`. */
typedef struct {
  int k;                /* neighbours per pixel, 1..32 */
  const int *nbr;       /* device [P][k] cache indices, -1 for none */
  const float *nbr_w;   /* device [P][k] normalised weights (sum 1 over the valid ones) */
  int S;                /* samples per pixel */
  const float *u;       /* device [P][S][4] uniforms in [0, 1): the map choice, then
                           three for the direction; 16-byte aligned */
  const float *albedo;  /* device [P][3] */
  const float *emit;    /* nullable device [P][3]: L_e */
  const float *direct;  /* nullable device [P][3]: the direct-light term */
} drc_indirect_params;

drc_status drc_indirect(drc_ctx *ctx, const drc_caches *caches, const drc_gbuffer *gbuf,
                        const drc_indirect_params *params, float *out_rgb, void *stream);

/* The denoiser's input maps traced from cache points (Sec. 3.1-3.3: the
 * radiance arriving at the first non-specular hit without the direct light,
 * the distance to what is seen and its normal), in an analytic interior:
 * the unit box [0,1]^3 of six diffuse walls, an emitting rectangle on the
 * ceiling z = 1 and diffuse spheres seen from outside.
 *   Texel (a, b) of cache j takes one ray from pos[j] along polar angle
 *   (a + 1/2) pi/2H from nrm[j] and azimuth (b + 1/2) 2 pi/W in the cache
 *   frame of drc_interpolate's LOOKUP mode.  Channel 3 is the distance to the
 *   first hit, channels 4-6 its normal facing the ray, channels 0-2 the
 *   radiance leaving it toward the cache without its own emission: a path of
 *   D bounces, each cosine-weighted about the current normal with uniforms
 *   u[j][a][b][k] = (u0, u1) (r = sqrt(u0), phi = 2 pi u1), adding the
 *   throughput times the next hit's emission and multiplying it by that
 *   hit's albedo.  A texel whose ray hits nothing, or a cache with a zero
 *   normal, is all zeros.
 * pos, nrm: device [n][3] (pos strictly inside the box); u: device
 * [n][H][W][D][2] float32 (8-byte aligned; NULL when D = 0); maps: device
 * [n][7][H][W] float32, drc_denoise's input layout (linear radiance: denoise
 * with DRC_F_ENCODE_INPUT).  INVALID_ARG for nsph outside 0..DRC_MAX_SPHERES,
 * H, W outside 1..4096, D outside 0..64.  Asynchronous on `stream`. */
#define DRC_MAX_SPHERES 64
typedef struct {
  float wall_alb[6][3];  /* albedo of the walls -x, +x, -y, +y, -z, +z */
  float wall_em[6][3];   /* their emitted radiance */
  int has_light;         /* the ceiling rectangle below, when nonzero */
  float light[7];        /* x0, x1, y0, y1 on z = 1, emitted radiance rgb */
  int nsph;
  float sph[DRC_MAX_SPHERES][7]; /* centre xyz, radius, albedo rgb */
} drc_scene;

drc_status drc_gen_maps(drc_ctx *ctx, const drc_scene *scene, int n, const float *pos, const float *nrm, int H,
                        int W, int D, const float *u, float *maps, void *stream);

/* Test harness, not a hot path (the paper has no counterpart): the mean L1
 * loss of the context's network (Sec. 3.3 network, Sec. 4 loss, the loss
 * drc_backward differentiates with DRC_BWD_L1_TARGET) evaluated in FP64 on
 * the GPU with the packed weights given in FP64, for central finite
 * differences of drc_backward's gradient.  weights64: device [n_floats]
 * double; in: device [N][7][H][W] float; target: device [N][3][H][W];
 * flags: DRC_F_ENCODE_INPUT or 0; loss64: device double, written.
 * Allocates its own scratch and synchronises `stream` (slow, direct loops).
 * INVALID_ARG for shapes drc_backward refuses. */
drc_status drc_fd_loss64(drc_ctx *ctx, const double *weights64, const float *in, const float *target, int N, int H,
                         int W, unsigned flags, double *loss64, void *stream);

/* Progressive refinement (Sec. 3.2): the image-plane sample points of pass
 * `pass` (0, 1, ...).  After each pass the distance between grid points is
 * reduced by a constant factor, here 2 (a reading: the factor is not
 * printed); points already evaluated are kept, so pass 0 takes the pixels
 * (x, y) with x and y multiples of s0 = spacing0, and pass t > 0 those that
 * are multiples of s_t = spacing0 / 2^t but not both multiples of s_{t-1}.
 * The interpolation after pass t uses every point so far with
 * r = s_t (the distance between two grid points).  Host-only, no GPU.
 * pix: host [max_points][2] int32 (x, y), row-major order of (y, x); *count
 * receives the number of points (written even when they do not fit, in
 * which case INVALID_ARG is returned and pix is left partial).  spacing0
 * must be a power of two; once s_t would drop below 1 a pass has no points.
 * INVALID_ARG for width or height < 1, pass < 0, NULL count. */
drc_status drc_pass_points(int width, int height, int spacing0, int pass, int *pix, int max_points, int *count);

/* One frame end to end from host memory: drc_denoise of N maps, then
 * drc_interpolate (IRRADIANCE) of a G-buffer from their payloads, with the
 * uploads and the download inside the call (Sec. 3.3 denoising feeding the
 * Sec. 3.2 interpolation).  The maps, then the G-buffer, go to the device on
 * the context's own copy stream; the denoise starts once the maps have
 * landed, the interpolation once the G-buffer has; the image comes back on
 * `stream`.  A call's uploads wait only for the previous call's reads of the
 * same staging, so in a frame loop one frame's maps upload under the
 * previous frame's interpolation and its G-buffer under its own denoise.
 *   maps_host: host [N][7][H][W] float32 (page-locked for overlap);
 *              flags: 0 or DRC_F_ENCODE_INPUT, as drc_denoise;
 *   caches:    DEVICE positions / normals / pixels of the N caches as for
 *              drc_interpolate (caches->n == N); payload and maps are not
 *              read -- the call uses its own denoised payloads;
 *   gbuf_host: the G-buffer with HOST pointers pos, nrm ([P][3] float32,
 *              page-locked for overlap); dir is not read;
 *   params:    as drc_interpolate, mode DRC_INTERP_IRRADIANCE;
 *   rgb_host:  host [P][3] float32, written when `stream` reaches the end
 *              of the call.
 * The host buffers must stay valid and unchanged until then.  The denoised
 * maps and payloads stay in the context's device staging (grown on demand). */
drc_status drc_frame_host(drc_ctx *ctx, const float *maps_host, int N, int H,
                          int W, unsigned flags, const drc_caches *caches,
                          const drc_gbuffer *gbuf_host,
                          const drc_interp_params *params, float *rgb_host,
                          void *stream);

/* drc_backward flags (combine one of the first two with DRC_F_ENCODE_INPUT
 * and DRC_BWD_RECOMPUTE_ENCODER as needed) */
#define DRC_BWD_L1_TARGET 0x10u /* target = ground truth [N][3][H][W] (log
                                   radiance); loss = mean |out - target| */
#define DRC_BWD_GRAD_OUT 0x20u  /* target = dL/dout [N][3][H][W] */
#define DRC_BWD_RECOMPUTE_ENCODER 0x40u /* activation checkpointing: the
                                   decoder overwrites the encoder activations
                                   in place during the forward and the
                                   encoder is run again before its backward
                                   (one more encoder pass, less memory) */

/* Gradient of the loss through the network (Sec. 3.3: the autoencoder is
 * trained with the L1 loss of Eq. 7 on log radiance).  One call runs the
 * forward pass on `in`, forms dL/dout, and runs the reverse pass: the output
 * head, then per decoder stage the weight gradient, bias gradient and data
 * gradient (a stride-2 convolution with the same weights), then per encoder
 * stage the same (a transposed convolution), with the ReLU masks and the
 * skip-connection fan-out.  Data gradients run on the tensor cores in the
 * context's precision (FP32: split-tf32; BF16: bf16 operands), weight and
 * bias gradients accumulate in fp32.
 *   in:       device [N][7][H][W] (as drc_denoise; DRC_F_ENCODE_INPUT may be
 *             given: the gradient then flows through log1p(s L));
 *   target:   device [N][3][H][W] (see the flags); the output is the network
 *             output in log radiance (never decoded);
 *   dweights: device, drc_weight_count() floats, packed like the weights,
 *             overwritten;
 *   dinput:   nullable, device [N][7][H][W];
 *   loss:     nullable, device float scalar, overwritten (L1_TARGET; 0 for
 *             GRAD_OUT).
 * FP8 contexts return DRC_ERR_UNSUPPORTED.  The context keeps the training
 * workspace (activations, ReLU outputs, gradients) in its own device memory,
 * grown on demand. */
drc_status drc_backward(drc_ctx *ctx, const float *in, const float *target,
                        int N, int H, int W, unsigned flags, float *dweights,
                        float *dinput, float *loss, void *stream);

/* Weight gradient of one 3x3, stride-2, pad-1 layer alone (the per-layer
 * step of the training pass above, Sec. 3.3):
 *   dW[m][q][u][v] += sum over n, i, j of R[n][i][j][m] * Q[n][2i+u-1][2j+v-1][q]
 * with Q read as zero outside [0, 2Hb) x [0, 2Wb).  For a conv layer R is the
 * output gradient and Q the input (dW is then [Cout][Cin][3][3]); for a
 * transposed conv R is the input and Q the output gradient (dW [Cin][Cout]
 * [3][3]), the packed weight layouts of drc_create.
 *   R:  device, NHWC [N][Hb][Wb][Mr], channels contiguous;
 *   Q:  device, NHWC [N][2Hb][2Wb][Qc]; only channels q < Qraw enter dW;
 *   dtype: DRC_PREC_FP32 (float operands) or DRC_PREC_BF16 (bfloat16);
 *   dW: device fp32 [Mr][Qraw][3][3], ACCUMULATED into (clear it first).
 * BF16 operands with Mr a multiple of 128, Qc of 64, Wb dividing 64 and 64
 * pixels covering whole rows of whole maps run on the tensor cores (fp32
 * accumulation, the pixel sum split over CTAs and added with atomics, so the
 * summation order varies from run to run); every other shape, and FP32,
 * runs a CUDA-core kernel with fp32 sums.  N = 0 leaves dW unchanged.  The
 * context supplies the device, the status word and the wait bound only. */
drc_status drc_weight_grad(drc_ctx *ctx, const void *R, const void *Q,
                           drc_precision dtype, int N, int Hb, int Wb, int Mr,
                           int Qc, int Qraw, float *dW, void *stream);

/* Training-data augmentation (Sec. 4, Implementation: the training pairs are
 * augmented with combinations of rotation and flipping).  Read as the eight
 * symmetries of a square map: codes[n] = r + 4 f (only its low three bits
 * are used) mirrors the columns of map n if f (column j -> W - 1 - j) and
 * then turns it r quarter turns counter-clockwise (one turn: out[i][j] =
 * in[j][W - 1 - i]), every channel alike; values are not changed.  Give the
 * input maps and the targets of a pair the same code.
 *   in, out: device fp32 [N][C][H][W] (NCHW, contiguous, 16-byte aligned),
 *            H == W, not overlapping;
 *   codes:   device int32 [N] (16-byte aligned).
 * Asynchronous on `stream`.  INVALID_ARG for H != W, a bad shape, host or
 * unaligned pointers, or overlapping buffers; N = 0 does nothing. */
drc_status drc_augment(drc_ctx *ctx, const float *in, float *out, int N, int C,
                       int H, int W, const int *codes, void *stream);

/* One step t >= 1 of Adam (Kingma & Ba 2015, Algorithm 1), the optimiser of
 * the paper's training (Sec. 4: PyTorch's Adam, learning rate 6e-5; PyTorch's
 * defaults beta1 = 0.9, beta2 = 0.999, eps = 1e-8), on n parameters in place:
 *   m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
 *   w -= lr m / (1 - beta1^t) / (sqrt(v / (1 - beta2^t)) + eps).
 * w, grad, m, v: device fp32 [n], 16-byte aligned, caller-owned (m and v
 * start at zero before step 1).  For the network, w is a device copy of the packed weights and
 * grad drc_backward's dweights; drc_set_weights(ctx, w, 1, stream) then
 * makes the new weights current.  Asynchronous on `stream`; INVALID_ARG for
 * t < 1, lr <= 0, a beta outside [0, 1), eps < 0, host or unaligned
 * pointers. */
drc_status drc_adam_step(drc_ctx *ctx, float *w, const float *grad, float *m,
                         float *v, size_t n, int t, float lr, float beta1,
                         float beta2, float eps, void *stream);

/* The paper's own network form (Sec. 3.3, "Neural network") in FP32: a
 * U-Net.  Levels l = 0..levels have depth base * 2^l.  Each
 * encoder level applies two 3x3 convolutions (stride 1, padding 1), each
 * followed by batch normalisation (inference statistics, eps 1e-5) and
 * LeakyReLU (slope 0.01); 2x2 max pooling leads to the next level.  Each
 * decoder level l = levels-1..0 upsamples the deeper features 2x
 * (bilinear, half-pixel centres), concatenates them (first) with the encoder
 * output of level l (second) and applies two 3x3 transposed convolutions
 * (stride 1, padding 1), each followed by batch normalisation and LeakyReLU,
 * except at level 0 (LeakyReLU only).  A 1x1 convolution to out_ch channels
 * with ReLU ends it.  The paper's network: in_ch 7, out_ch 3, base 64,
 * levels 3.
 *   params: device fp32, drc_unet_param_count floats, layer by layer:
 *           encoder levels 0..levels (two convs each: W [Cout][Cin][3][3],
 *           b, gamma, beta, mean, var), decoder levels levels-1..0 (two
 *           transposed convs each: W [Cin][Cout][3][3], b, and gamma, beta,
 *           mean, var except at level 0), the head (W [out_ch][base], b)
 *           -- the PyTorch layouts;
 *   in:     device fp32 [N][in_ch][H][W], H and W multiples of 2^levels;
 *   out:    device fp32 [N][out_ch][H][W];
 *   workspace: device memory of drc_unet_workspace_bytes (folded weights
 *           and every activation), caller-owned.
 * All pointers 16-byte aligned.  Asynchronous on `stream`; INVALID_ARG for a
 * bad shape, a short workspace, host or unaligned pointers.  The two size
 * queries return 0 for shapes the forward pass refuses.
 * Where drc_unet_tensor_cores is 1 for the shape (base a multiple of 32;
 * in_ch <= 8 or a multiple of 32; at every level W >> l dividing 128 and
 * the maps' rows tiling 128-row boxes), the 3x3 layers run on the tensor
 * cores as implicit GEMMs in the split-tf32 product (three tf32 products,
 * each tile's K loop accumulated in chunks of one K block that are added
 * into an fp32 running sum), with NHWC activations in the workspace;
 * otherwise on the CUDA cores in plain fp32.  The workspace size covers
 * either. */
size_t drc_unet_param_count(int in_ch, int out_ch, int base, int levels);
int drc_unet_tensor_cores(int in_ch, int out_ch, int base, int levels, int H,
                          int W);
size_t drc_unet_workspace_bytes(int in_ch, int out_ch, int base, int levels,
                                int N, int H, int W);
drc_status drc_unet_forward(drc_ctx *ctx, int in_ch, int out_ch, int base,
                            int levels, const float *params, const float *in,
                            float *out, int N, int H, int W, void *workspace,
                            size_t workspace_bytes, void *stream);

/* Synchronise `stream` and return (then clear) the latched device status:
 * DRC_OK or DRC_ERR_TIMEOUT. */
drc_status drc_get_status(drc_ctx *ctx, void *stream);

/* Human-readable description of the last error on this context ("" if
 * none).  Valid until the next call on the context. */
const char *drc_last_error(drc_ctx *ctx);

/* Tune the context's conv layers for batches of N maps of H x W: each
 * layer's tile width (GEMM N per tile: its output channels, or half of them)
 * and, for FP32, its A-operand path are timed on the context's own workspace
 * and the fastest kept for every later drc_denoise (results stay within the
 * precision's tolerance).  FP32 decoder layers of at most 64 output channels
 * also time their phase-pair form: the four output parities of the stride-2
 * transposed conv as two GEMMs, each holding the parities (p, 0) and (p, 1)
 * of one output row side by side in a 2 Cout-column tile over the union of
 * their input taps (a tap one of the two parities lacks has zero weights
 * there), with A in tensor memory or in shared memory.
 * Synchronises the device first (calls in flight on any stream finish before
 * the timing launches reuse the workspace) and at the end; grows the
 * workspace to N maps.  No counterpart in
 * the paper. */
drc_status drc_autotune(drc_ctx *ctx, int N, int H, int W);

/* drc_autotune with a persistent cache: `path` is a text file of JSON lines,
 * one per tuned case, keyed by the GPU (name, SM count, compute capability),
 * the network (channels, widths, out_relu, exposure), the precision and the
 * batch shape N x H x W.  If the file holds an entry for this case (the last
 * valid one wins), its tile widths and A paths are applied without timing
 * and *from_cache (nullable) is set to 1; otherwise drc_autotune runs and
 * its choice is appended as a new line (a missing file is created).  An
 * entry whose choices do not fit this context's layers is ignored.  Lines
 * are appended with one write each, so processes sharing the file may add
 * duplicate entries but do not interleave them.  Synchronises the device.
 * INVALID_ARG for a bad shape, an empty path or a file that cannot be
 * written.  No counterpart in the paper. */
drc_status drc_autotune_cached(drc_ctx *ctx, int N, int H, int W,
                               const char *path, int *from_cache);

/* Checkpoints (Sec. 4: the trained network is saved and loaded again by the
 * renderer): the context's current fp32 weights and, optionally, the Adam
 * state of a training run, in one file -- a line of JSON header (format,
 * version, the network: in/out channels, widths, out_relu, exposure; the
 * float count, whether Adam state follows, its step count, the payload size
 * and its 64-bit FNV-1a checksum) followed by the little-endian fp32 arrays:
 * weights [n], then adam_m [n] and adam_v [n] when present (n =
 * drc_weight_count).
 *   save: adam_m / adam_v are device pointers of n floats, both given or
 *         both NULL; adam_step >= 0 is stored with them.  Reads the weights
 *         and state on `stream` and synchronises it; writes a temporary file
 *         renamed over `path`.
 *   load: checks the header against the context's network (precision may
 *         differ: the weights are the fp32 masters) and the checksum, makes
 *         the weights current as drc_set_weights from host memory does,
 *         and, when adam_m / adam_v are given, uploads the state into them
 *         and stores the step in *adam_step (nullable).  Asking for Adam
 *         state from a file without it is INVALID_ARG.
 * INVALID_ARG for a file that cannot be read or written, is not a
 * checkpoint, belongs to another network or is damaged; UNSUPPORTED for a
 * newer format version. */
drc_status drc_save_checkpoint(drc_ctx *ctx, const char *path,
                               const float *adam_m, const float *adam_v,
                               int adam_step, void *stream);
drc_status drc_load_checkpoint(drc_ctx *ctx, const char *path, float *adam_m,
                               float *adam_v, int *adam_step, void *stream);

/* Copy the context's current fp32 weights (drc_weight_count floats, the
 * layout drc_create takes) into `out`: device memory (asynchronous on
 * `stream`) when out_on_device, else host memory (synchronises `stream`).
 * INVALID_ARG before any weights were set. */
drc_status drc_get_weights(drc_ctx *ctx, float *out, int out_on_device,
                           void *stream);

/* Cap the device memory the context allocates from now on -- its packed
 * weights, workspaces, interpolation and training scratch, plans and
 * staging buffers -- at `bytes` in total (0: no cap, the default).  A call
 * that would need more returns DRC_ERR_OOM before allocating, with the
 * sizes in drc_last_error, and leaves the context usable (raising the cap
 * lets the same call succeed).  Memory the caller passes in (inputs,
 * outputs, drc_unet_forward's workspace) is not counted.  A cap below the
 * current use only refuses later growth.  No counterpart in the paper. */
drc_status drc_set_memory_limit(drc_ctx *ctx, size_t bytes);
/* Bytes of device memory the context holds now. */
size_t drc_memory_in_use(const drc_ctx *ctx);

/* FP8 e4m3 contexts: measure the network's activations on a representative
 * batch (in, N, H, W, flags as drc_denoise) and set every layer's
 * per-input-channel scales to the channel's maximum / 448 with one binade of
 * headroom; the scales are folded into the layer's weights before they are
 * quantised with per-output-channel scales.  Two passes (the second with the
 * scales of the first).  Until calibrated, every scale is 1.  Synchronises;
 * other precisions return DRC_ERR_UNSUPPORTED.  No counterpart in the paper
 * (it runs in FP32 on a CPU). */
drc_status drc_calibrate(drc_ctx *ctx, const float *in, int N, int H, int W,
                         unsigned flags, void *stream);

/* The tile width (0 for the head) and A-operand path (-1 default, 0
 * per-thread gathers, 1 TMA + producer conversion, 8 / 9 phase pairs with A
 * in tensor / shared memory -- see drc_autotune; the tile width is then the
 * unpaired fallback's) drc_denoise uses for one layer (0 .. 2S-1). */
drc_status drc_describe_layer(drc_ctx *ctx, int layer, int *bn, int *a_path);

/* ---- Plans: progressive passes with uneven batches ------------------------
 * Sec. 3.2 ("Progressive refinement and interpolation"): every indirect pass
 * shrinks the cache grid by a constant factor, so each pass denoises a
 * different number of cache maps.  A plan is built once for a set of map
 * sizes (classes), each with a maximum count; every pass is then one small
 * kernel (this pass's counts and buffers into the plan's device slots) and
 * one CUDA-graph launch holding the whole network for every class, its
 * tensor-core kernels persistent (one CTA per SM) and sized by the count
 * they read from device memory.  No allocation, synchronisation or host
 * read of the counts per pass.                                              */

typedef struct {
  int H, W;     /* map size of this class (multiples of 2^num_stages, H <= 256) */
  int max_maps; /* largest count a pass may give this class (>= 1) */
} drc_size_class;

typedef struct drc_plan drc_plan;

#define DRC_PLAN_AUTOTUNE 0x1u /* time each conv layer's tile-width (and, for
                                  FP32, A-operand path) candidates on the
                                  class's full-size buffers at creation and
                                  keep the fastest; otherwise the defaults of
                                  drc_denoise */

/* Build a plan on ctx (weights must be set).  Allocates its own activation
 * buffers (max_maps of each class), packed operands and graph; synchronises
 * the device while building.  1 <= n_classes <= 8.  The plan uses the
 * context's weights and status word: destroy it before the context. */
drc_status drc_plan_create(drc_ctx *ctx, const drc_size_class *classes,
                           int n_classes, unsigned flags, drc_plan **plan);

/* Run one pass on `stream`.
 *   counts:  device int[n_classes], maps of each class in this pass; a count
 *            outside 0..max_maps is clamped and latches DRC_ERR_INVALID_ARG
 *            (returned by drc_get_status);
 *   in[k]:   device [counts[k]][7][H_k][W_k] fp32 (host array of pointers);
 *   out[k]:  device [counts[k]][3][H_k][W_k] fp32;
 *   payload: nullable host array; payload[k] nullable device [counts[k]][3];
 *   flags:   DRC_F_ENCODE_INPUT / DRC_F_DECODE_OUTPUT, as drc_denoise.
 * Results equal drc_denoise of each class's maps.  Weights set on the
 * context after the plan was built are repacked before the pass. */
drc_status drc_plan_launch(drc_plan *plan, const int *counts,
                           const float *const *in, float *const *out,
                           float *const *payload, unsigned flags, void *stream);

/* The chosen tile width (GEMM N per tile; 0 for the head) and A-operand
 * path (-1 default, 1 TMA + producer conversion) of one layer of one class. */
drc_status drc_plan_describe(drc_plan *plan, int size_class, int layer,
                             int *bn, int *a_path);

drc_status drc_plan_destroy(drc_plan *plan);

/* ---- Launch accounting (diagnostics; no counterpart in the paper) ---- */

/* Kernel launches this context has issued since it was created (weight
 * packing, denoise, interpolation), counted on the host at each launch. */
drc_status drc_launch_count(drc_ctx *ctx, unsigned long long *count);

/* While enabled, every kernel launch of the context is bracketed by two CUDA
 * events recorded on its stream (a few microseconds of stream work each);
 * off by default. */
drc_status drc_set_timing(drc_ctx *ctx, int enable);

typedef struct {
  char name[32];      /* "conv e1", "convT d2", "head", "interp query", ... */
  long long launches; /* timed launches of this kernel since the last read */
  double total_ms;    /* their summed device time */
} drc_kernel_time;

/* Wait for the timed launches recorded since the last read, then write their
 * per-kernel totals (in first-launch order) to out[0..*n_out) and clear them.
 * capacity too small: the first `capacity` kernels are written and
 * DRC_ERR_INVALID_ARG is returned. */
drc_status drc_read_timing(drc_ctx *ctx, drc_kernel_time *out, int capacity,
                           int *n_out);

#ifdef __cplusplus
}
#endif

#endif /* DRC_H_ */
