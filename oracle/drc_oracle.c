/*
 * drc_oracle.c -- FP64 CPU oracle for the Deep Radiance Caching hot path
 * (Jiang & Kainz, "Deep Radiance Caching: Convolutional Autoencoders Deeper
 * in Ray Tracing", arXiv 1910.02480).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * helper with the CUDA library: it is a plain, slow, direct-loop restatement
 * of what the method computes, in double precision, so that a reader can
 * check it against the paper by eye.
 *
 * Tensors handed in are float32 (the exact bytes the GPU path consumes), or
 * exact double copies of them for the augmentation and the optimiser; every
 * computation is carried out in double.
 *
 * Functions and the passages they follow:
 *   orc_conv3x3s2     3x3 convolution, stride 2, pad 1 (the encoder stages of
 *                     the autoencoder, Sec. 3.3 "Neural network").
 *   orc_convT3x3s2    3x3 transposed convolution, stride 2, pad 1, output
 *                     padding 1 (the decoder "deconvolutions", Sec. 3.3).
 *   orc_forward       encoder / decoder with skip connections (Sec. 3.3),
 *                     optional log encode / decode of the radiance channels.
 *   orc_payload       cosine-weighted integral of a hemispherical lat-long
 *                     radiance map over the upper hemisphere (Eq. 2 for a
 *                     diffuse BRDF; map encoding of Sec. 3.3).
 *   orc_interp        k-nearest cache selection, the weight heuristic
 *                     w = w_p*w_n + w_p + eps and its normalisation, and the
 *                     blend of the cached values (Sec. 3.2, Eqs. 4-6).
 *   orc_l1_backward   L1 loss (Sec. 3.3, Sec. 5.1 Eq. 7) and its exact
 *                     gradient through the network (reverse mode).
 *   orc_augment       training-data augmentation by rotation and flipping
 *                     (Sec. 4, Implementation).
 *   orc_adam_step     one step of the Adam optimiser the training uses
 *                     (Sec. 4), as defined by Kingma & Ba (2015), Alg. 1.
 *   orc_mis_indirect  the indirect term of Eq. 3 estimated with multiple
 *                     importance sampling over the blended cached maps and
 *                     the BRDF (Sec. 3.2); orc_indirect_expected, its
 *                     expectation by quadrature.
 *   orc_gen_maps      the input maps traced from cache points in an
 *                     analytic interior: radiance without the direct light,
 *                     distance, normal (Sec. 3.2-3.3).
 *   orc_unet_forward  the paper's own network form (Sec. 3.3 "Neural
 *                     network"): a U-Net of two 3x3 convolutions per stage
 *                     with batch normalisation and LeakyReLU, 2x2 max
 *                     pooling, 2x bilinear upsampling, concatenated skips
 *                     and a 1x1 convolution with ReLU; with its parts
 *                     orc_conv3x3s1, orc_convT3x3s1, orc_maxpool2 and
 *                     orc_upsample2.
 * Readings of passages the paper leaves open are listed beside each function.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_F_ENCODE_INPUT 1u
#define ORC_F_DECODE_OUTPUT 2u

#define ORC_METRIC_IMAGE 0
#define ORC_METRIC_WORLD 1
#define ORC_WP_INVERSE 0
#define ORC_WP_LINEAR 1
#define ORC_INTERP_IRRADIANCE 0
#define ORC_INTERP_LOOKUP 1

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Convolutions (Sec. 3.3).  Layouts: x [N][C][H][W]; conv weights          */
/* [Cout][Cin][3][3]; transposed-conv weights [Cin][Cout][3][3].            */
/* ------------------------------------------------------------------------ */

/* y[n,o,i,j] = b[o] + sum_{c,u,v} W[o,c,u,v] * x[n,c,2i+u-1,2j+v-1],
 * x taken as zero outside the map.  Output is (H/2) x (W/2). */
void orc_conv3x3s2(const double *x, int N, int Cin, int H, int W,
                   const double *Wt, const double *b, int Cout, double *y)
{
    int Ho = H / 2, Wo = W / 2;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++)
        for (int o = 0; o < Cout; o++)
            for (int i = 0; i < Ho; i++)
                for (int j = 0; j < Wo; j++) {
                    double acc = b ? b[o] : 0.0;
                    for (int c = 0; c < Cin; c++)
                        for (int u = 0; u < 3; u++)
                            for (int v = 0; v < 3; v++) {
                                int yy = 2 * i + u - 1, xx = 2 * j + v - 1;
                                if (yy < 0 || yy >= H || xx < 0 || xx >= W)
                                    continue;
                                acc += Wt[((o * Cin + c) * 3 + u) * 3 + v] *
                                       x[(((long)n * Cin + c) * H + yy) * W + xx];
                            }
                    y[(((long)n * Cout + o) * Ho + i) * Wo + j] = acc;
                }
}

/* y[n,o,p,q] = b[o] + sum over (c,i,j,u,v) with 2i+u-1 = p, 2j+v-1 = q of
 * W[c,o,u,v] * x[n,c,i,j].  Output is (2H) x (2W): written exactly as the
 * scatter of every input pixel through every tap, dropping taps that land
 * outside the output. */
void orc_convT3x3s2(const double *x, int N, int Cin, int H, int W,
                    const double *Wt, const double *b, int Cout, double *y)
{
    int Ho = 2 * H, Wo = 2 * W;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        for (int o = 0; o < Cout; o++)
            for (int p = 0; p < Ho * Wo; p++)
                y[((long)n * Cout + o) * Ho * Wo + p] = b ? b[o] : 0.0;
        for (int c = 0; c < Cin; c++)
            for (int i = 0; i < H; i++)
                for (int j = 0; j < W; j++) {
                    double xv = x[(((long)n * Cin + c) * H + i) * W + j];
                    for (int o = 0; o < Cout; o++)
                        for (int u = 0; u < 3; u++)
                            for (int v = 0; v < 3; v++) {
                                int p = 2 * i + u - 1, q = 2 * j + v - 1;
                                if (p < 0 || p >= Ho || q < 0 || q >= Wo)
                                    continue;
                                y[(((long)n * Cout + o) * Ho + p) * Wo + q] +=
                                    Wt[((c * Cout + o) * 3 + u) * 3 + v] * xv;
                            }
                }
    }
}

/* ------------------------------------------------------------------------ */
/* Network description: packed weights, in order conv_1..conv_S then       */
/* convT_S..convT_1, each layer as W followed by b.                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int S, cin, cout, out_relu;
    int width[9]; /* width[0] = cin, width[1..S] = encoder widths */
    const double *encW[8], *encB[8];
    const double *decW[9], *decB[9]; /* decoder convT_s, s = 1..S */
    long n_floats;
} orc_net;

long orc_weight_count(int S, const int *widths, int cin, int cout)
{
    long n = 0;
    int prev = cin;
    for (int s = 0; s < S; s++) {
        n += 9L * prev * widths[s] + widths[s];
        prev = widths[s];
    }
    for (int s = S - 1; s >= 0; s--) {
        int co = (s == 0) ? cout : widths[s - 1];
        n += 9L * widths[s] * co + co;
    }
    return n;
}

/* Bind the packed (double) weight vector to the layer pointers. */
static int bind_net(orc_net *net, int S, const int *widths, int cin, int cout,
                    int out_relu, const double *w, long n_floats)
{
    if (S < 1 || S > 8)
        return -1;
    net->S = S;
    net->cin = cin;
    net->cout = cout;
    net->out_relu = out_relu;
    net->width[0] = cin;
    for (int s = 0; s < S; s++)
        net->width[s + 1] = widths[s];
    if (orc_weight_count(S, widths, cin, cout) != n_floats)
        return -2;
    long off = 0;
    for (int s = 1; s <= S; s++) {
        net->encW[s - 1] = w + off;
        off += 9L * net->width[s - 1] * net->width[s];
        net->encB[s - 1] = w + off;
        off += net->width[s];
    }
    for (int s = S; s >= 1; s--) {
        int co = (s == 1) ? cout : net->width[s - 1];
        net->decW[s] = w + off;
        off += 9L * net->width[s] * co;
        net->decB[s] = w + off;
        off += co;
    }
    net->n_floats = off;
    return 0;
}

static double *widen(const float *a, long n)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (long i = 0; i < n; i++)
        d[i] = (double)a[i];
    return d;
}

static void relu_inplace(double *a, long n)
{
    for (long i = 0; i < n; i++)
        if (!(a[i] > 0.0))
            a[i] = 0.0;
}

/* Input encode: channels 0..2 carry radiance; log1p(s*L) when the encode flag
 * is set (a reading: the paper does not state a transform for its network,
 * log1p keeps zero radiance at zero). */
static void encode_input(double *x, int N, int C, int H, int W, double s)
{
    for (int n = 0; n < N; n++)
        for (int c = 0; c < 3 && c < C; c++)
            for (long p = 0; p < (long)H * W; p++) {
                double *v = &x[((long)n * C + c) * H * W + p];
                *v = log1p(s * (*v));
            }
}

/* Forward state kept for the backward pass. */
typedef struct {
    int N, H, W;
    double *e[9];  /* e[0] = encoded input, e[s] = ReLU(z[s]) */
    double *z[9];  /* encoder pre-activations */
    double *t[9];  /* decoder: t[S] = e[S]; t[s-1] = ReLU(zd[s]) + e[s-1] */
    double *zd[9]; /* decoder pre-activations, zd[s] = convT_s(t[s]) */
    double *out;   /* network output (log radiance), after optional ReLU */
    double *zout;  /* output pre-activation */
} orc_state;

static long act_size(const orc_net *net, int N, int H, int W, int s)
{
    /* stage s has width[s] channels at (H >> s) x (W >> s) */
    return (long)N * net->width[s] * (H >> s) * (W >> s);
}

static void free_state(orc_state *st, int S)
{
    for (int s = 0; s <= S; s++) {
        free(st->e[s]);
        free(st->z[s]);
        free(st->zd[s]);
        if (s < S)
            free(st->t[s]);
    }
    free(st->out);
    free(st->zout);
}

/* Encoder: e_0 = x, e_s = ReLU(conv_s(e_{s-1})).  Decoder: t = e_S; for
 * s = S..2, t = ReLU(convT_s(t)) + e_{s-1} (skip connection added after the
 * activation -- a reading, the paper only names skip connections); output
 * = convT_1(t), optionally followed by ReLU (the paper's final ReLU). */
static void run_forward(const orc_net *net, const double *x_enc, int N, int H,
                        int W, orc_state *st)
{
    int S = net->S;
    memset(st, 0, sizeof(*st));
    st->N = N;
    st->H = H;
    st->W = W;
    long n0 = (long)N * net->cin * H * W;
    st->e[0] = (double *)malloc(sizeof(double) * n0);
    memcpy(st->e[0], x_enc, sizeof(double) * n0);
    for (int s = 1; s <= S; s++) {
        long ns = act_size(net, N, H, W, s);
        st->z[s] = (double *)malloc(sizeof(double) * ns);
        orc_conv3x3s2(st->e[s - 1], N, net->width[s - 1], H >> (s - 1),
                      W >> (s - 1), net->encW[s - 1], net->encB[s - 1],
                      net->width[s], st->z[s]);
        st->e[s] = (double *)malloc(sizeof(double) * ns);
        memcpy(st->e[s], st->z[s], sizeof(double) * ns);
        relu_inplace(st->e[s], ns);
    }
    st->t[S] = st->e[S];
    for (int s = S; s >= 2; s--) {
        long ns = act_size(net, N, H, W, s - 1);
        st->zd[s] = (double *)malloc(sizeof(double) * ns);
        orc_convT3x3s2(st->t[s], N, net->width[s], H >> s, W >> s,
                       net->decW[s], net->decB[s], net->width[s - 1],
                       st->zd[s]);
        st->t[s - 1] = (double *)malloc(sizeof(double) * ns);
        for (long i = 0; i < ns; i++)
            st->t[s - 1][i] = (st->zd[s][i] > 0.0 ? st->zd[s][i] : 0.0) +
                              st->e[s - 1][i];
    }
    long no = (long)N * net->cout * H * W;
    st->zout = (double *)malloc(sizeof(double) * no);
    orc_convT3x3s2(st->t[1], N, net->width[1], H >> 1, W >> 1, net->decW[1],
                   net->decB[1], net->cout, st->zout);
    st->out = (double *)malloc(sizeof(double) * no);
    memcpy(st->out, st->zout, sizeof(double) * no);
    if (net->out_relu)
        relu_inplace(st->out, no);
}

/* Full denoise: in [N][cin][H][W] (float32) -> out [N][cout][H][W] (double).
 * flags: ORC_F_ENCODE_INPUT applies log1p(s*L) to channels 0..2 first;
 * ORC_F_DECODE_OUTPUT returns expm1(y)/s instead of the log-space y.
 * Returns 0, or a negative code for a bad description. */
int orc_forward(int S, const int *widths, int cin, int cout, int out_relu,
                double s, unsigned flags, const float *weights, long n_floats,
                const float *in, int N, int H, int W, double *out)
{
    if (H % (1 << S) || W % (1 << S))
        return -3;
    double *w = widen(weights, n_floats);
    orc_net net;
    int rc = bind_net(&net, S, widths, cin, cout, out_relu, w, n_floats);
    if (rc) {
        free(w);
        return rc;
    }
    long nin = (long)N * cin * H * W;
    double *x = widen(in, nin);
    if (flags & ORC_F_ENCODE_INPUT)
        encode_input(x, N, cin, H, W, s);
    orc_state st;
    run_forward(&net, x, N, H, W, &st);
    long no = (long)N * cout * H * W;
    for (long i = 0; i < no; i++)
        out[i] = (flags & ORC_F_DECODE_OUTPUT) ? expm1(st.out[i]) / s
                                               : st.out[i];
    free_state(&st, S);
    free(x);
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Irradiance of a hemispherical lat-long map (Eq. 2 with a diffuse BRDF).  */
/* Map layout (a reading of the map encoding in Sec. 3.3): row i covers     */
/* theta in [i*pi/(2H), (i+1)*pi/(2H)] with theta = 0 at the normal;        */
/* column j covers phi in [2*pi*j/W, 2*pi*(j+1)/W).  Each texel's weight is */
/* the exact integral of cos(theta) dOmega over its band:                   */
/*   1/2 (sin^2 theta_{i+1} - sin^2 theta_i) * (2 pi / W).                  */
/* payload = E / pi, i.e. the outgoing radiance of a white Lambertian       */
/* surface lit by the map.                                                  */
/* ------------------------------------------------------------------------ */
void orc_payload(const double *L, int N, int C, int H, int W, double *payload)
{
    for (int n = 0; n < N; n++)
        for (int c = 0; c < C; c++) {
            double E = 0.0;
            for (int i = 0; i < H; i++) {
                double t0 = i * ORC_PI / (2.0 * H);
                double t1 = (i + 1) * ORC_PI / (2.0 * H);
                double band = 0.5 * (sin(t1) * sin(t1) - sin(t0) * sin(t0)) *
                              (2.0 * ORC_PI / W);
                for (int j = 0; j < W; j++)
                    E += L[(((long)n * C + c) * H + i) * W + j] * band;
            }
            payload[(long)n * C + c] = E / ORC_PI;
        }
}

/* ------------------------------------------------------------------------ */
/* Interpolation of cached radiance (Sec. 3.2).                             */
/* ------------------------------------------------------------------------ */

/* Local frame of a cache (map encoding, Sec. 3.3): the normal is the map's
 * Z axis; the up vector is the scene's (+Z) and is turned to +Y only when
 * the normal itself points along Z (reading: |n.z| > 1 - 1e-6).
 * t = normalize(up x n), b = n x t.  Returns 0 for a zero-length normal. */
static int cache_frame(const float *nrm, double t[3], double b[3], double n[3])
{
    double nx = nrm[0], ny = nrm[1], nz = nrm[2];
    double len = sqrt(nx * nx + ny * ny + nz * nz);
    if (!(len > 0.0))
        return 0;
    n[0] = nx / len;
    n[1] = ny / len;
    n[2] = nz / len;
    double up[3] = {0.0, 0.0, 1.0};
    if (fabs(n[2]) > 1.0 - 1e-6) {
        up[0] = 0.0;
        up[1] = 1.0;
        up[2] = 0.0;
    }
    double cx = up[1] * n[2] - up[2] * n[1];
    double cy = up[2] * n[0] - up[0] * n[2];
    double cz = up[0] * n[1] - up[1] * n[0];
    double cl = sqrt(cx * cx + cy * cy + cz * cz);
    t[0] = cx / cl;
    t[1] = cy / cl;
    t[2] = cz / cl;
    b[0] = n[1] * t[2] - n[2] * t[1];
    b[1] = n[2] * t[0] - n[0] * t[2];
    b[2] = n[0] * t[1] - n[1] * t[0];
    return 1;
}

/* Bilinear lookup of channel c of map R (H x W lat-long), continuous texel
 * coordinates (ti, tj) with texel centres at integer + 0.5 of the angle
 * grid: wrap in phi (columns), clamp in theta (rows). */
static double bilinear(const float *R, int H, int W, double ti, double tj)
{
    double fi = floor(ti), fj = floor(tj);
    double ai = ti - fi, aj = tj - fj;
    int i0 = (int)fi, j0 = (int)fj;
    int i1 = i0 + 1, j1 = j0 + 1;
    if (i0 < 0)
        i0 = 0;
    if (i0 > H - 1)
        i0 = H - 1;
    if (i1 < 0)
        i1 = 0;
    if (i1 > H - 1)
        i1 = H - 1;
    j0 = ((j0 % W) + W) % W;
    j1 = ((j1 % W) + W) % W;
    double v00 = R[(long)i0 * W + j0], v01 = R[(long)i0 * W + j1];
    double v10 = R[(long)i1 * W + j0], v11 = R[(long)i1 * W + j1];
    return (1 - ai) * ((1 - aj) * v00 + aj * v01) +
           ai * ((1 - aj) * v10 + aj * v11);
}

/* For pixels p in [p_begin, p_end) of a width x height G-buffer:
 *  1. distance d^2 to every cache: IMAGE metric in integer pixels on the image
 *     plane (Sec. 3.2), WORLD metric between first-hit positions;
 *  2. keep the k smallest by (d^2, cache index);
 *  3. w_p = r/(d + delta_rel*r) (INVERSE, a reading: printed "dist/r" grows
 *     with distance) or max(0, 1 - d/r) (LINEAR);
 *     w_n = max(0, n_j . n_p) with unit normals (reading: the prose says the
 *     normal weight is largest when the normals agree and zero when their dot
 *     product is negative, which the printed 1 - max(0, .) contradicts);
 *     w = w_p * w_n + w_p + eps (Eq. 4);
 *  4. normalise, W_j = w_j / sum w;
 *  5. IRRADIANCE: out = sum W_j payload_j.  LOOKUP: out = sum W_j R_j(l_j),
 *     with l_j the pixel direction in cache j's frame, zero below the cache's
 *     horizon -- the expectation over map choice of the paper's sampling of
 *     maps with probabilities W_j.
 * out is [p_end-p_begin][3].  nbr_idx ([.][k], nullable) receives the
 * selected indices in (d^2, index) order; nbr_d2 ([.][k+1], nullable) the
 * k+1 smallest d^2 (the last is +inf if n <= k) for tie analysis. */
int orc_interp(int n_caches, int mapH, int mapW, const float *maps,
               const float *payload, const float *cpos, const float *cnrm,
               const int *cpix, int width, int height, const float *gpos,
               const float *gnrm, const float *gdir, int k, int metric,
               int wp_form, int mode, double r, double eps, double delta_rel,
               long p_begin, long p_end, double *out, int *nbr_idx,
               double *nbr_d2, double *nbr_w)
{
    if (k < 1 || k > 64 || n_caches < 1)
        return -1;
    if (mode == ORC_INTERP_LOOKUP && (!maps || !gdir))
        return -1;
    (void)height;
#pragma omp parallel for schedule(dynamic, 64)
    for (long p = p_begin; p < p_end; p++) {
        int px = (int)(p % width), py = (int)(p / width);
        double bd[65];
        int bi[65];
        int nb = 0;
        for (int j = 0; j < n_caches; j++) {
            double d2;
            if (metric == ORC_METRIC_IMAGE) {
                double dx = (double)(px - cpix[2 * j]);
                double dy = (double)(py - cpix[2 * j + 1]);
                d2 = dx * dx + dy * dy;
            } else {
                double dx = (double)gpos[3 * p] - cpos[3 * j];
                double dy = (double)gpos[3 * p + 1] - cpos[3 * j + 1];
                double dz = (double)gpos[3 * p + 2] - cpos[3 * j + 2];
                d2 = dx * dx + dy * dy + dz * dz;
            }
            /* insertion into the sorted list of the k+1 best, key (d2, j);
             * j grows, so an equal d2 already in the list ranks first */
            if (nb == k + 1 && !(d2 < bd[k]))
                continue;
            int pos = (nb < k + 1) ? nb++ : k;
            while (pos > 0 && d2 < bd[pos - 1]) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                pos--;
            }
            bd[pos] = d2;
            bi[pos] = j;
        }
        int kk = nb < k ? nb : k;
        double w[64], wsum = 0.0;
        double pn[3] = {gnrm[3 * p], gnrm[3 * p + 1], gnrm[3 * p + 2]};
        double pl = sqrt(pn[0] * pn[0] + pn[1] * pn[1] + pn[2] * pn[2]);
        for (int q = 0; q < kk; q++) {
            int j = bi[q];
            double d = sqrt(bd[q]);
            double wp;
            if (wp_form == ORC_WP_INVERSE)
                wp = r / (d + delta_rel * r);
            else
                wp = 1.0 - d / r > 0.0 ? 1.0 - d / r : 0.0;
            double cn[3] = {cnrm[3 * j], cnrm[3 * j + 1], cnrm[3 * j + 2]};
            double cl = sqrt(cn[0] * cn[0] + cn[1] * cn[1] + cn[2] * cn[2]);
            double wn = 0.0;
            if (pl > 0.0 && cl > 0.0) {
                double dot = (cn[0] * pn[0] + cn[1] * pn[1] + cn[2] * pn[2]) /
                             (cl * pl);
                wn = dot > 0.0 ? dot : 0.0;
            }
            w[q] = wp * wn + wp + eps;
            wsum += w[q];
        }
        double acc[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < kk; q++) {
            int j = bi[q];
            double Wq = w[q] / wsum;
            if (mode == ORC_INTERP_IRRADIANCE) {
                for (int c = 0; c < 3; c++)
                    acc[c] += Wq * payload[3 * j + c];
            } else {
                double t[3], b[3], n[3];
                if (!cache_frame(&cnrm[3 * j], t, b, n))
                    continue;
                double om[3] = {gdir[3 * p], gdir[3 * p + 1], gdir[3 * p + 2]};
                double ol = sqrt(om[0] * om[0] + om[1] * om[1] + om[2] * om[2]);
                if (!(ol > 0.0))
                    continue;
                for (int a = 0; a < 3; a++)
                    om[a] /= ol;
                double lx = om[0] * t[0] + om[1] * t[1] + om[2] * t[2];
                double ly = om[0] * b[0] + om[1] * b[1] + om[2] * b[2];
                double lz = om[0] * n[0] + om[1] * n[1] + om[2] * n[2];
                if (!(lz > 0.0))
                    continue;
                if (lz > 1.0)
                    lz = 1.0;
                double theta = acos(lz);
                double phi = atan2(ly, lx);
                if (phi < 0.0)
                    phi += 2.0 * ORC_PI;
                double ti = theta / (0.5 * ORC_PI) * mapH - 0.5;
                double tj = phi / (2.0 * ORC_PI) * mapW - 0.5;
                for (int c = 0; c < 3; c++) {
                    const float *R = maps + (((long)j * 3 + c) * mapH) * mapW;
                    acc[c] += Wq * bilinear(R, mapH, mapW, ti, tj);
                }
            }
        }
        long o = p - p_begin;
        for (int c = 0; c < 3; c++)
            out[3 * o + c] = acc[c];
        if (nbr_idx)
            for (int q = 0; q < k; q++)
                nbr_idx[o * k + q] = q < kk ? bi[q] : -1;
        if (nbr_d2)
            for (int q = 0; q <= k; q++)
                nbr_d2[o * (k + 1) + q] = q < nb ? bd[q] : INFINITY;
        if (nbr_w)
            for (int q = 0; q < k; q++)
                nbr_w[o * k + q] = q < kk ? w[q] / wsum : 0.0;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The indirect term by multiple importance sampling (Sec. 3.2 with Eq. 3), */
/* a next step of this build.                                               */
/* ------------------------------------------------------------------------ */
/* The paper evaluates the indirect term of Eq. 3, the hemisphere integral of
 * f_r cos(theta_i) R(omega_i), with a small fixed number of samples,
 * alternating between sampling R as an environment map with perfect
 * visibility and sampling the BRDF, combined by multiple importance sampling
 * (Veach).  R at a pixel is the blend of its k nearest caches' maps with the
 * normalised weights of Eq. 4 (orc_interp); drawn as map-selection
 * probabilities the weights make the estimate's expectation the integral of
 * that blend.
 * Readings: a Lambertian BRDF f_r = albedo / pi.  Texel (a, b) of a map holds
 * one radiance over its solid angle: polar angle in [a, a+1) pi / (2H) from
 * the cache normal, azimuth in [b, b+1) 2 pi / W in the cache frame (the
 * frame rule of the lookup above).  Environment sampling picks a texel with
 * probability proportional to its luminance 0.2126 R + 0.7152 G + 0.0722 B
 * times its solid angle, then a direction uniform in solid angle inside it.
 * BRDF sampling is cosine-weighted about the pixel normal (a frame of the
 * same rule).  Sample s takes the environment for even s and the BRDF for
 * odd s; the balance heuristic weighs them by their sample counts, which
 * reduces a sample's contribution to f_r cos R / (n_env pdf_env + n_brdf
 * pdf_brdf).  The random numbers are an input: u [P][S][4] uniform in
 * [0, 1), the map choice and three for the direction. */

static double texel_lum(const float *maps, int j, int H, int W, int a, int b)
{
    const long plane = (long)H * W;
    const float *R = maps + (long)j * 3 * plane + (long)a * W + b;
    return 0.2126 * R[0] + 0.7152 * R[plane] + 0.0722 * R[2 * plane];
}

/* solid angle of a texel in row a */
static double texel_omega(int a, int H, int W)
{
    return (cos(a * 0.5 * ORC_PI / H) - cos((a + 1) * 0.5 * ORC_PI / H)) * 2.0 * ORC_PI / W;
}

/* texel of world direction w in the frame (t, b, n); 0 below the hemisphere */
static int texel_of(const double t[3], const double b[3], const double n[3], const double w[3], int H, int W,
                    int *ta, int *tb)
{
    double lx = w[0] * t[0] + w[1] * t[1] + w[2] * t[2];
    double ly = w[0] * b[0] + w[1] * b[1] + w[2] * b[2];
    double lz = w[0] * n[0] + w[1] * n[1] + w[2] * n[2];
    if (!(lz > 0.0))
        return 0;
    double theta = acos(lz > 1.0 ? 1.0 : lz);
    double phi = atan2(ly, lx);
    if (phi < 0.0)
        phi += 2.0 * ORC_PI;
    int a = (int)floor(theta / (0.5 * ORC_PI) * H), c = (int)floor(phi / (2.0 * ORC_PI) * W);
    *ta = a < 0 ? 0 : (a > H - 1 ? H - 1 : a);
    *tb = c < 0 ? 0 : (c > W - 1 ? W - 1 : c);
    return 1;
}

/* per-map luminance x solid-angle CDF over the H W texels (row-major) */
static double *env_cdfs(int n_caches, int H, int W, const float *maps)
{
    const long plane = (long)H * W;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)(n_caches * plane));
    for (int j = 0; j < n_caches; j++) {
        double acc = 0.0;
        for (int a = 0; a < H; a++)
            for (int b = 0; b < W; b++) {
                acc += texel_lum(maps, j, H, W, a, b) * texel_omega(a, H, W);
                cdf[(long)j * plane + (long)a * W + b] = acc;
            }
    }
    return cdf;
}

/* Two discrete choices of a sample are taken from running sums: the map
 * (u0 against the running sum of the weights) and the environment texel
 * (u1 times the total against the CDF).  The paper fixes no precision for
 * them; a float32 evaluation sums in float32, and near a boundary the two
 * precisions may rightly choose differently.  So both choices are taken in
 * float32 here, from the same float32 operations in the same order as the
 * GPU path: the weights summed one by one, and each map's CDF summed texel
 * by texel in row-major order from float32 luminance
 * (0.2126 R + 0.7152 G) + 0.0722 B times the row's solid angle, that angle
 * being 2 sin(mid) sin(half-width) (2 pi / W) in double rounded to float32.
 * Everything else stays double.
 *
 * margin (nullable, [P]): for the comparison with a float evaluation, the
 * smallest distance, over the pixel's samples, of a value that takes one of
 * the other discrete decisions from the boundary where it changes, in units
 * of the float32 error that value may carry: the texel a direction falls in
 * (polar and azimuthal texel coordinates against integers, units 2e-4
 * texel), the hemisphere tests (cosines against 0, units 2e-6) and the
 * up-vector switch of the frames (|n_z| against 1 - 1e-6, units 2e-6).
 * Below 1, a float32 evaluation may rightly decide the other way.  The
 * estimate does not depend on it. */
static void margin_min(double *m, double v, double unit)
{
    v = fabs(v) / unit;
    if (v < *m)
        *m = v;
}

static float omega_f32(int a, int H, int W)
{
    const double t0 = a * 0.5 * ORC_PI / H, t1 = (a + 1) * 0.5 * ORC_PI / H;
    return (float)(2.0 * sin(0.5 * (t0 + t1)) * sin(0.5 * (t1 - t0)) * (2.0 * ORC_PI / W));
}

/* per-map float32 CDF of the texel choice, summed as described above */
static float *env_cdfs_f32(int n_caches, int H, int W, const float *maps)
{
    const long plane = (long)H * W;
    float *cdf = (float *)malloc(sizeof(float) * (size_t)(n_caches * plane));
    for (int j = 0; j < n_caches; j++) {
        float acc = 0.0f;
        for (int a = 0; a < H; a++) {
            const float om = omega_f32(a, H, W);
            for (int b = 0; b < W; b++) {
                const float *R = maps + (long)j * 3 * plane + (long)a * W + b;
                const float lum = (0.2126f * R[0] + 0.7152f * R[plane]) + 0.0722f * R[2 * plane];
                acc = acc + lum * om;
                cdf[(long)j * plane + (long)a * W + b] = acc;
            }
        }
    }
    return cdf;
}

static double frac_dist(double x)
{
    return fabs(x - floor(x + 0.5));
}

static double frame_margin(const float *nrm)
{
    double nx = nrm[0], ny = nrm[1], nz = nrm[2];
    double len = sqrt(nx * nx + ny * ny + nz * nz);
    return len > 0.0 ? fabs(fabs(nz / len) - (1.0 - 1e-6)) / 2e-6 : 1e30;
}

int orc_mis_indirect(int n_caches, int mapH, int mapW, const float *maps, const float *cnrm, long P, int k,
                     const int *nbr_idx, const double *nbr_w, const float *gnrm, const float *albedo, int S,
                     const double *u, double *out, double *margin)
{
    if (n_caches < 1 || mapH < 1 || mapW < 1 || k < 1 || S < 1)
        return -1;
    const long plane = (long)mapH * mapW;
    double *cdf = env_cdfs(n_caches, mapH, mapW, maps);
    float *cdf_f = env_cdfs_f32(n_caches, mapH, mapW, maps);
    const double n_env = (double)((S + 1) / 2), n_brdf = (double)(S / 2);
#pragma omp parallel for schedule(dynamic, 16)
    for (long p = 0; p < P; p++) {
        double acc[3] = {0.0, 0.0, 0.0};
        double tp[3], bp[3], np_[3];
        double mg = frame_margin(&gnrm[3 * p]);
        if (cache_frame(&gnrm[3 * p], tp, bp, np_)) {
            for (int s = 0; s < S; s++) {
                const double *us = u + ((size_t)p * S + s) * 4;
                /* the map, by the normalised weights (running sum in float32) */
                int q = -1;
                float c = 0.0f;
                for (int i = 0; i < k; i++) {
                    if (nbr_idx[p * k + i] < 0)
                        continue;
                    q = i;
                    c = c + (float)nbr_w[p * k + i];
                    if ((float)us[0] < c)
                        break;
                }
                if (q < 0)
                    continue;
                const int j = nbr_idx[p * k + q];
                double t[3], b[3], n[3];
                margin_min(&mg, frame_margin(&cnrm[3 * j]), 1.0);
                if (!cache_frame(&cnrm[3 * j], t, b, n))
                    continue;
                const double *cj = cdf + (long)j * plane;
                const double total = cj[plane - 1];
                double w[3];
                if (s % 2 == 0) { /* environment: texel by the CDF, direction uniform inside */
                    if (!(total > 0.0))
                        continue;
                    /* the texel, by the float32 CDF */
                    const float *cf = cdf_f + (long)j * plane;
                    const float target = (float)us[1] * cf[plane - 1];
                    long e = 0;
                    while (e < plane - 1 && !(cf[e] > target))
                        e++;
                    const int a = (int)(e / mapW), bc = (int)(e % mapW);
                    const double c0 = cos(a * 0.5 * ORC_PI / mapH), c1 = cos((a + 1) * 0.5 * ORC_PI / mapH);
                    const double mu = c0 - us[2] * (c0 - c1), sn = sqrt(1.0 - mu * mu > 0.0 ? 1.0 - mu * mu : 0.0);
                    const double phi = (bc + us[3]) * 2.0 * ORC_PI / mapW;
                    const double l[3] = {sn * cos(phi), sn * sin(phi), mu};
                    for (int d = 0; d < 3; d++)
                        w[d] = l[0] * t[d] + l[1] * b[d] + l[2] * n[d];
                } else { /* BRDF: cosine-weighted about the pixel normal */
                    const double rr = sqrt(us[1]), phi = 2.0 * ORC_PI * us[2];
                    const double l[3] = {rr * cos(phi), rr * sin(phi), sqrt(1.0 - us[1] > 0.0 ? 1.0 - us[1] : 0.0)};
                    for (int d = 0; d < 3; d++)
                        w[d] = l[0] * tp[d] + l[1] * bp[d] + l[2] * np_[d];
                }
                const double cosp = w[0] * np_[0] + w[1] * np_[1] + w[2] * np_[2];
                margin_min(&mg, cosp, 2e-6);
                if (!(cosp > 0.0))
                    continue;
                {
                    const double lx = w[0] * t[0] + w[1] * t[1] + w[2] * t[2];
                    const double ly = w[0] * b[0] + w[1] * b[1] + w[2] * b[2];
                    const double lz = w[0] * n[0] + w[1] * n[1] + w[2] * n[2];
                    margin_min(&mg, lz, 2e-6);
                    if (lz > 0.0) {
                        const double th = acos(lz > 1.0 ? 1.0 : lz);
                        double ph = atan2(ly, lx);
                        if (ph < 0.0)
                            ph += 2.0 * ORC_PI;
                        margin_min(&mg, frac_dist(th / (0.5 * ORC_PI) * mapH), 2e-4);
                        margin_min(&mg, frac_dist(ph / (2.0 * ORC_PI) * mapW), 2e-4);
                    }
                }
                int ta, tb;
                if (!texel_of(t, b, n, w, mapH, mapW, &ta, &tb))
                    continue; /* below the cache's hemisphere: R = 0 */
                const double pdf_env = total > 0.0 ? texel_lum(maps, j, mapH, mapW, ta, tb) / total : 0.0;
                const double denom = n_env * pdf_env + n_brdf * cosp / ORC_PI;
                if (!(denom > 0.0))
                    continue;
                for (int d = 0; d < 3; d++) {
                    const double R = maps[((long)j * 3 + d) * plane + (long)ta * mapW + tb];
                    acc[d] += albedo[3 * p + d] / ORC_PI * cosp * R / denom;
                }
            }
        }
        for (int d = 0; d < 3; d++)
            out[3 * p + d] = acc[d];
        if (margin)
            margin[p] = mg;
    }
    free(cdf);
    free(cdf_f);
    return 0;
}

/* The estimator's expectation by quadrature: sum over the selected maps of
 * weight x sum over texels of the texel radiance x (albedo / pi) x the
 * integral of max(0, cos to the pixel normal) over the texel, taken on
 * m x m cells of equal solid angle (midpoints in cos theta and phi). */
int orc_indirect_expected(int n_caches, int mapH, int mapW, const float *maps, const float *cnrm, long P, int k,
                          const int *nbr_idx, const double *nbr_w, const float *gnrm, const float *albedo, int m,
                          double *out)
{
    if (n_caches < 1 || mapH < 1 || mapW < 1 || k < 1 || m < 1)
        return -1;
    const long plane = (long)mapH * mapW;
#pragma omp parallel for schedule(dynamic, 4)
    for (long p = 0; p < P; p++) {
        double acc[3] = {0.0, 0.0, 0.0};
        double tp[3], bp[3], np_[3];
        if (cache_frame(&gnrm[3 * p], tp, bp, np_)) {
            for (int i = 0; i < k; i++) {
                const int j = nbr_idx[p * k + i];
                if (j < 0)
                    continue;
                double t[3], b[3], n[3];
                if (!cache_frame(&cnrm[3 * j], t, b, n))
                    continue;
                for (int a = 0; a < mapH; a++) {
                    const double c0 = cos(a * 0.5 * ORC_PI / mapH), c1 = cos((a + 1) * 0.5 * ORC_PI / mapH);
                    const double cell = (c0 - c1) / m * (2.0 * ORC_PI / mapW) / m;
                    for (int bc = 0; bc < mapW; bc++) {
                        double integ = 0.0;
                        for (int x = 0; x < m; x++) {
                            const double mu = c0 - (x + 0.5) * (c0 - c1) / m;
                            const double sn = sqrt(1.0 - mu * mu);
                            for (int y = 0; y < m; y++) {
                                const double phi = (bc + (y + 0.5) / m) * 2.0 * ORC_PI / mapW;
                                const double l[3] = {sn * cos(phi), sn * sin(phi), mu};
                                double cp = 0.0;
                                for (int d = 0; d < 3; d++)
                                    cp += (l[0] * t[d] + l[1] * b[d] + l[2] * n[d]) * np_[d];
                                if (cp > 0.0)
                                    integ += cp * cell;
                            }
                        }
                        for (int d = 0; d < 3; d++)
                            acc[d] += nbr_w[p * k + i] * albedo[3 * p + d] / ORC_PI *
                                      maps[((long)j * 3 + d) * plane + (long)a * mapW + bc] * integ;
                    }
                }
            }
        }
        for (int d = 0; d < 3; d++)
            out[3 * p + d] = acc[d];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Input-map generation, a next step of this build: the maps are traced    */
/* from the first intersection point (Sec. 3.1-3.2), radiance with the     */
/* direct light excluded, distance and normal (Sec. 3.3's seven channels). */
/* ------------------------------------------------------------------------ */
/* Readings (the paper's scenes are not available):
 *  - the scene is an interior: the unit box [0,1]^3 of six diffuse walls
 *    (albedo and emission per wall, in the order -x, +x, -y, +y, -z, +z),
 *    an extra emitting rectangle on the ceiling z = 1 (x in [x0, x1], y in
 *    [y0, y1], radiance Le), and diffuse spheres (centre, radius, albedo)
 *    seen from outside;
 *  - texel (a, b) of a cache's map takes one ray from the cache point along
 *    its centre direction: polar angle (a + 1/2) pi / (2H) from the cache
 *    normal, azimuth (b + 1/2) 2 pi / W in the cache frame (the lookup's
 *    frame rule);
 *  - channels 3 and 4-6 are the distance to the first hit and the hit's
 *    normal facing the ray; channels 0-2 the radiance leaving the first hit
 *    toward the cache point without the hit's own emission (the direct
 *    light the paper leaves out of R), from a path of D bounces: each takes
 *    a cosine-weighted direction about the current normal (in a frame of the
 *    same rule), adds the throughput times the next hit's emission and
 *    multiplies the throughput by that hit's albedo, the Lambertian estimate
 *    of one bounce; the random numbers are an input u [n][H][W][D][2]. */

typedef struct {
    const double *wall_alb, *wall_em; /* [6][3] */
    const double *light;              /* x0 x1 y0 y1 Le[3] */
    int nsph;
    const double *sph; /* [nsph][7]: centre, radius, albedo[3] */
} orc_scene;

/* nearest hit of the ray o + t d (d unit, t > 0): distance, normal facing
 * the ray, albedo and emission there; 0 when nothing is hit.  mg
 * (nullable): lowered to the margins of the hit's discrete decisions, in
 * units of the float32 error the values may carry after a few bounces --
 * the gap from the nearest surface to the next one along the ray (units
 * 1e-5), the hit's distance to the ceiling light's border (1e-5), a sphere's
 * B^2 - C at a grazing ray (1e-4: near tangency the hit point moves by
 * about the error of B^2 - C over its square root, so the distance and
 * normal are ill-conditioned there, not only the hit-or-miss decision) and,
 * for the next bounce's frame, |n_z| of a sphere normal against 1 - 1e-6
 * (2e-6). */
static int scene_hit(const orc_scene *sc, const double o[3], const double d[3], double *th, double nh[3],
                     double alb[3], double em[3], double *mg)
{
    double best = INFINITY, second = INFINITY;
    int which = -1; /* 0..5 wall, 6 + s sphere s */
    for (int i = 0; i < 3; i++) {
        double t = -1.0;
        int w = -1;
        if (d[i] > 0.0) {
            t = (1.0 - o[i]) / d[i];
            w = 2 * i + 1;
        } else if (d[i] < 0.0) {
            t = -o[i] / d[i];
            w = 2 * i;
        }
        if (w >= 0 && t > 1e-12) {
            if (t < best) { second = best; best = t; which = w; }
            else if (t < second) second = t;
        }
    }
    for (int s = 0; s < sc->nsph; s++) {
        const double *sp = sc->sph + 7 * s;
        const double oc[3] = {o[0] - sp[0], o[1] - sp[1], o[2] - sp[2]};
        const double B = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
        const double C = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - sp[3] * sp[3];
        const double disc = B * B - C;
        if (mg && C > 0.0 && B < 0.0)
            margin_min(mg, disc, 1e-4);
        if (C <= 0.0 || disc < 0.0)
            continue; /* seen from outside only */
        const double t = -B - sqrt(disc);
        if (t > 1e-12) {
            if (t < best) { second = best; best = t; which = 6 + s; }
            else if (t < second) second = t;
        }
    }
    if (which < 0)
        return 0;
    if (mg && second < INFINITY)
        margin_min(mg, second - best, 1e-5);
    *th = best;
    const double h[3] = {o[0] + best * d[0], o[1] + best * d[1], o[2] + best * d[2]};
    if (which < 6) {
        const int axis = which / 2, side = which % 2;
        nh[0] = nh[1] = nh[2] = 0.0;
        nh[axis] = side ? -1.0 : 1.0; /* inward */
        for (int c = 0; c < 3; c++) {
            alb[c] = sc->wall_alb[3 * which + c];
            em[c] = sc->wall_em[3 * which + c];
        }
        if (which == 5 && sc->light && mg) {
            const double ex = fmin(fabs(h[0] - sc->light[0]), fabs(h[0] - sc->light[1]));
            const double ey = fmin(fabs(h[1] - sc->light[2]), fabs(h[1] - sc->light[3]));
            margin_min(mg, fmin(ex, ey), 1e-5);
        }
        if (which == 5 && sc->light && h[0] >= sc->light[0] && h[0] <= sc->light[1] && h[1] >= sc->light[2] &&
            h[1] <= sc->light[3])
            for (int c = 0; c < 3; c++)
                em[c] += sc->light[4 + c];
    } else {
        const double *sp = sc->sph + 7 * (which - 6);
        for (int c = 0; c < 3; c++) {
            nh[c] = (h[c] - sp[c]) / sp[3];
            alb[c] = sp[4 + c];
            em[c] = 0.0;
        }
        if (mg) {
            const float nf[3] = {(float)nh[0], (float)nh[1], (float)nh[2]};
            margin_min(mg, frame_margin(nf), 1.0);
        }
    }
    return 1;
}

/* margin (nullable, [n][H][W]): per texel the smallest margin of the
 * decisions along its path (scene_hit), for the comparison with a float32
 * evaluation: below 1 it may rightly take another surface or light. */
int orc_gen_maps(int n, const float *pos, const float *nrm, int H, int W, const double *wall_alb,
                 const double *wall_em, const double *light, int nsph, const double *sph, int D, const double *u,
                 double *maps, double *margin)
{
    if (n < 0 || H < 1 || W < 1 || D < 0 || nsph < 0)
        return -1;
    for (int j = 0; j < n; j++)
        for (int c = 0; c < 3; c++)
            if (!(pos[3 * j + c] > 0.0f && pos[3 * j + c] < 1.0f))
                return -1;
    const orc_scene sc = {wall_alb, wall_em, light, nsph, sph};
    const long plane = (long)H * W;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int j = 0; j < n; j++) {
        double t[3], b[3], nn[3];
        if (!cache_frame(&nrm[3 * j], t, b, nn)) {
            bad = 1;
            continue;
        }
        const double x[3] = {pos[3 * j], pos[3 * j + 1], pos[3 * j + 2]};
        double *out = maps + (long)j * 7 * plane;
        for (int a = 0; a < H; a++)
            for (int bc = 0; bc < W; bc++) {
                const long e = (long)a * W + bc;
                const double th = (a + 0.5) * 0.5 * ORC_PI / H, ph = (bc + 0.5) * 2.0 * ORC_PI / W;
                const double l[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
                double d[3];
                for (int c = 0; c < 3; c++)
                    d[c] = l[0] * t[c] + l[1] * b[c] + l[2] * nn[c];
                double dist, nh[3], alb[3], em[3];
                double mgv = 1e30, *mg = margin ? &mgv : NULL;
                for (int c = 0; c < 7; c++)
                    out[c * plane + e] = 0.0;
                if (margin)
                    margin[(long)j * plane + e] = 1e30;
                if (!scene_hit(&sc, x, d, &dist, nh, alb, em, mg))
                    continue;
                out[3 * plane + e] = dist;
                for (int c = 0; c < 3; c++)
                    out[(4 + c) * plane + e] = nh[c];
                /* the path from the first hit: its emission left out */
                double thr[3] = {alb[0], alb[1], alb[2]}, L[3] = {0.0, 0.0, 0.0};
                double o[3] = {x[0] + dist * d[0], x[1] + dist * d[1], x[2] + dist * d[2]};
                double nc[3] = {nh[0], nh[1], nh[2]};
                for (int k = 0; k < D; k++) {
                    const double *uk = u + ((((long)j * H + a) * W + bc) * D + k) * 2;
                    const float nf[3] = {(float)nc[0], (float)nc[1], (float)nc[2]};
                    double tt[3], bb[3], n2[3];
                    cache_frame(nf, tt, bb, n2);
                    const double rr = sqrt(uk[0]), phi = 2.0 * ORC_PI * uk[1];
                    const double lz = sqrt(1.0 - uk[0] > 0.0 ? 1.0 - uk[0] : 0.0);
                    double dn[3];
                    for (int c = 0; c < 3; c++)
                        dn[c] = rr * cos(phi) * tt[c] + rr * sin(phi) * bb[c] + lz * nc[c];
                    double t2, nh2[3], alb2[3], em2[3];
                    if (!scene_hit(&sc, o, dn, &t2, nh2, alb2, em2, mg))
                        break;
                    for (int c = 0; c < 3; c++) {
                        L[c] += thr[c] * em2[c];
                        thr[c] *= alb2[c];
                        o[c] = o[c] + t2 * dn[c];
                        nc[c] = nh2[c];
                    }
                }
                for (int c = 0; c < 3; c++)
                    out[c * plane + e] = L[c];
                if (margin)
                    margin[(long)j * plane + e] = mgv;
            }
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Loss and gradient (training, Sec. 4; L1 of Sec. 3.3 and Eq. 7).          */
/* ------------------------------------------------------------------------ */

/* Adjoint of orc_conv3x3s2: accumulates dx (nullable), dW, db from g. */
static void conv_adjoint(const double *x, int N, int Cin, int H, int W,
                         const double *Wt, int Cout, const double *g,
                         double *dx, double *dW, double *db)
{
    int Ho = H / 2, Wo = W / 2;
#pragma omp parallel for schedule(static)
    for (int o = 0; o < Cout; o++) {
        double sb = 0.0;
        for (int n = 0; n < N; n++)
            for (int i = 0; i < Ho; i++)
                for (int j = 0; j < Wo; j++) {
                    double gv = g[(((long)n * Cout + o) * Ho + i) * Wo + j];
                    sb += gv;
                    for (int c = 0; c < Cin; c++)
                        for (int u = 0; u < 3; u++)
                            for (int v = 0; v < 3; v++) {
                                int yy = 2 * i + u - 1, xx = 2 * j + v - 1;
                                if (yy < 0 || yy >= H || xx < 0 || xx >= W)
                                    continue;
                                dW[((o * Cin + c) * 3 + u) * 3 + v] +=
                                    gv * x[(((long)n * Cin + c) * H + yy) * W + xx];
                            }
                }
        db[o] += sb;
    }
    if (!dx)
        return;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++)
        for (int o = 0; o < Cout; o++)
            for (int i = 0; i < Ho; i++)
                for (int j = 0; j < Wo; j++) {
                    double gv = g[(((long)n * Cout + o) * Ho + i) * Wo + j];
                    for (int c = 0; c < Cin; c++)
                        for (int u = 0; u < 3; u++)
                            for (int v = 0; v < 3; v++) {
                                int yy = 2 * i + u - 1, xx = 2 * j + v - 1;
                                if (yy < 0 || yy >= H || xx < 0 || xx >= W)
                                    continue;
                                dx[(((long)n * Cin + c) * H + yy) * W + xx] +=
                                    Wt[((o * Cin + c) * 3 + u) * 3 + v] * gv;
                            }
                }
}

/* Adjoint of orc_convT3x3s2 (input H x W, output 2H x 2W). */
static void convT_adjoint(const double *x, int N, int Cin, int H, int W,
                          const double *Wt, int Cout, const double *g,
                          double *dx, double *dW, double *db)
{
    int Ho = 2 * H, Wo = 2 * W;
#pragma omp parallel for schedule(static)
    for (int o = 0; o < Cout; o++) {
        double sb = 0.0;
        for (int n = 0; n < N; n++)
            for (int p = 0; p < Ho * Wo; p++)
                sb += g[((long)n * Cout + o) * Ho * Wo + p];
        db[o] += sb;
        for (int c = 0; c < Cin; c++)
            for (int n = 0; n < N; n++)
                for (int i = 0; i < H; i++)
                    for (int j = 0; j < W; j++) {
                        double xv = x[(((long)n * Cin + c) * H + i) * W + j];
                        for (int u = 0; u < 3; u++)
                            for (int v = 0; v < 3; v++) {
                                int p = 2 * i + u - 1, q = 2 * j + v - 1;
                                if (p < 0 || p >= Ho || q < 0 || q >= Wo)
                                    continue;
                                dW[((c * Cout + o) * 3 + u) * 3 + v] +=
                                    xv * g[(((long)n * Cout + o) * Ho + p) * Wo + q];
                            }
                    }
    }
    if (!dx)
        return;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++)
        for (int c = 0; c < Cin; c++)
            for (int i = 0; i < H; i++)
                for (int j = 0; j < W; j++) {
                    double acc = 0.0;
                    for (int o = 0; o < Cout; o++)
                        for (int u = 0; u < 3; u++)
                            for (int v = 0; v < 3; v++) {
                                int p = 2 * i + u - 1, q = 2 * j + v - 1;
                                if (p < 0 || p >= Ho || q < 0 || q >= Wo)
                                    continue;
                                acc += Wt[((c * Cout + o) * 3 + u) * 3 + v] *
                                       g[(((long)n * Cout + o) * Ho + p) * Wo + q];
                            }
                    dx[(((long)n * Cin + c) * H + i) * W + j] += acc;
                }
}

/* Weight gradient of one layer alone (training, Sec. 3.3), the dW part of
 * the adjoints above: transposed = 0, a conv with input x [N][Cin][H][W] and
 * output gradient g [N][Cout][H/2][W/2], dW [Cout][Cin][3][3]; transposed =
 * 1, a transposed conv with input x [N][Cin][H][W] and output gradient g
 * [N][Cout][2H][2W], dW [Cin][Cout][3][3].  dW is overwritten. */
void orc_conv_wgrad(const double *x, int N, int Cin, int H, int W,
                    const double *g, int Cout, int transposed, double *dW)
{
    double *db = calloc((size_t)Cout, sizeof(double));
    memset(dW, 0, sizeof(double) * 9 * (size_t)Cin * Cout);
    if (transposed)
        convT_adjoint(x, N, Cin, H, W, NULL, Cout, g, NULL, dW, db);
    else
        conv_adjoint(x, N, Cin, H, W, NULL, Cout, g, NULL, dW, db);
    free(db);
}

/* Loss and exact gradient.  mode 0: target is the ground truth y (log
 * radiance, [N][cout][H][W]); loss = mean |out - y| and dL/dout =
 * sign(out - y)/numel with sign(0) = 0.  mode 1: target is dL/dout itself and
 * the loss is not formed (reported as 0).
 * Outputs: dweights (packed like the weights, overwritten), dinput (nullable,
 * [N][cin][H][W], gradient with respect to the caller's input -- through the
 * log encode when that flag is set), returns the loss. */
double orc_l1_backward(int S, const int *widths, int cin, int cout,
                       int out_relu, double s, unsigned flags,
                       const float *weights, long n_floats, const float *in,
                       const float *target, int N, int H, int W, int mode,
                       double *dweights, double *dinput, int *rc_out)
{
    *rc_out = 0;
    if (H % (1 << S) || W % (1 << S)) {
        *rc_out = -3;
        return 0.0;
    }
    double *w = widen(weights, n_floats);
    orc_net net;
    int rc = bind_net(&net, S, widths, cin, cout, out_relu, w, n_floats);
    if (rc) {
        free(w);
        *rc_out = rc;
        return 0.0;
    }
    long nin = (long)N * cin * H * W;
    double *x = widen(in, nin);
    double *x_raw = widen(in, nin);
    if (flags & ORC_F_ENCODE_INPUT)
        encode_input(x, N, cin, H, W, s);
    orc_state st;
    run_forward(&net, x, N, H, W, &st);

    long no = (long)N * cout * H * W;
    double *g = (double *)calloc(no, sizeof(double));
    double loss = 0.0;
    if (mode == 0) {
        for (long i = 0; i < no; i++) {
            double dlt = st.out[i] - (double)target[i];
            loss += fabs(dlt);
            g[i] = (dlt > 0.0 ? 1.0 : (dlt < 0.0 ? -1.0 : 0.0)) / (double)no;
        }
        loss /= (double)no;
    } else {
        for (long i = 0; i < no; i++)
            g[i] = (double)target[i];
    }
    if (out_relu)
        for (long i = 0; i < no; i++)
            if (!(st.zout[i] > 0.0))
                g[i] = 0.0;

    /* gradient buffers, one per packed layer, bound to dweights */
    memset(dweights, 0, sizeof(double) * n_floats);
    orc_net dnet;
    bind_net(&dnet, S, widths, cin, cout, out_relu, dweights, n_floats);
    double *ge[9];
    for (int q = 0; q <= S; q++)
        ge[q] = (double *)calloc(act_size(&net, N, H, W, q), sizeof(double));

    /* output head: out = convT_1(t_1) */
    long n1 = act_size(&net, N, H, W, 1);
    double *gt = (double *)calloc(n1, sizeof(double));
    convT_adjoint(st.t[1], N, net.width[1], H >> 1, W >> 1, net.decW[1],
                  cout, g, gt, (double *)dnet.decW[1], (double *)dnet.decB[1]);
    free(g);
    /* decoder, reversed: t_{q-1} = ReLU(zd_q) + e_{q-1}, zd_q = convT_q(t_q) */
    for (int q = 2; q <= S; q++) {
        long nq1 = act_size(&net, N, H, W, q - 1);
        long nq = act_size(&net, N, H, W, q);
        for (long i = 0; i < nq1; i++)
            ge[q - 1][i] += gt[i]; /* skip branch */
        double *gz = (double *)malloc(sizeof(double) * nq1);
        for (long i = 0; i < nq1; i++)
            gz[i] = st.zd[q][i] > 0.0 ? gt[i] : 0.0;
        double *gtn = (double *)calloc(nq, sizeof(double));
        convT_adjoint(st.t[q], N, net.width[q], H >> q, W >> q, net.decW[q],
                      net.width[q - 1], gz, gtn, (double *)dnet.decW[q],
                      (double *)dnet.decB[q]);
        free(gz);
        free(gt);
        gt = gtn;
    }
    /* t_S = e_S */
    {
        long nS = act_size(&net, N, H, W, S);
        for (long i = 0; i < nS; i++)
            ge[S][i] += gt[i];
        free(gt);
    }
    /* encoder, reversed: e_q = ReLU(z_q), z_q = conv_q(e_{q-1}) */
    for (int q = S; q >= 1; q--) {
        long nq = act_size(&net, N, H, W, q);
        for (long i = 0; i < nq; i++)
            if (!(st.z[q][i] > 0.0))
                ge[q][i] = 0.0;
        conv_adjoint(st.e[q - 1], N, net.width[q - 1], H >> (q - 1),
                     W >> (q - 1), net.encW[q - 1], net.width[q], ge[q],
                     ge[q - 1], (double *)dnet.encW[q - 1],
                     (double *)dnet.encB[q - 1]);
    }
    if (dinput) {
        for (long i = 0; i < nin; i++)
            dinput[i] = ge[0][i];
        if (flags & ORC_F_ENCODE_INPUT)
            for (int n = 0; n < N; n++)
                for (int c = 0; c < 3 && c < cin; c++)
                    for (long p = 0; p < (long)H * W; p++) {
                        long i = ((long)n * cin + c) * H * W + p;
                        dinput[i] *= s / (1.0 + s * x_raw[i]);
                    }
    }
    for (int q = 0; q <= S; q++)
        free(ge[q]);
    free_state(&st, S);
    free(x);
    free(x_raw);
    free(w);
    return loss;
}

/* ------------------------------------------------------------------------ */
/* Training (Sec. 4, Implementation): augmentation and the optimiser step.  */
/* ------------------------------------------------------------------------ */

/* Reading: the paper augments the training pairs with "combinations of
 * rotation and flipping" of the maps and says no more.  Taken here as the
 * eight symmetries of the square H = W map, the same one for every channel
 * of a map (and for the input and target of a pair): code = r + 4 f, first
 * a mirror of the columns when f = 1 (column j -> W - 1 - j), then r
 * quarter turns counter-clockwise, one turn being b[i][j] = a[j][W - 1 - i].
 * Channel values are not changed.  Done literally, one operation after the
 * other on a scratch image.  x, y: [N][C][H][W]; codes: [N] in 0..7. */
void orc_augment(const double *x, int N, int C, int H, int W, const int *codes, double *y)
{
    const long plane = (long)H * W;
    double *a = (double *)malloc(sizeof(double) * (size_t)plane);
    double *b = (double *)malloc(sizeof(double) * (size_t)plane);
    for (int n = 0; n < N; ++n) {
        const int f = codes[n] / 4, r = codes[n] % 4;
        for (int c = 0; c < C; ++c) {
            const double *src = x + ((long)n * C + c) * plane;
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j)
                    a[i * W + j] = f ? src[i * W + (W - 1 - j)] : src[i * W + j];
            for (int q = 0; q < r; ++q) {
                for (int i = 0; i < H; ++i)
                    for (int j = 0; j < W; ++j)
                        b[i * W + j] = a[j * W + (W - 1 - i)];
                memcpy(a, b, sizeof(double) * (size_t)plane);
            }
            memcpy(y + ((long)n * C + c) * plane, a, sizeof(double) * (size_t)plane);
        }
    }
    free(a);
    free(b);
}

/* Adam (Kingma & Ba 2015, Algorithm 1), step t >= 1, on n parameters in
 * place: m <- b1 m + (1 - b1) g; v <- b2 v + (1 - b2) g^2; the bias
 * corrections m^ = m / (1 - b1^t), v^ = v / (1 - b2^t); w <- w - lr m^ /
 * (sqrt(v^) + eps).  The paper uses PyTorch's optimiser, whose update is
 * this one, with lr = 6e-5 (Sec. 4) and PyTorch's defaults b1 = 0.9,
 * b2 = 0.999, eps = 1e-8. */
void orc_adam_step(double *w, const double *g, double *m, double *v, long n, int t, double lr, double b1,
                   double b2, double eps)
{
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        const double mh = m[i] / c1, vh = v[i] / c2;
        w[i] = w[i] - lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* The paper's network form (Sec. 3.3, "Neural network").  Each encoder    */
/* stage takes two 3x3 convolutions and doubles the depth, each decoder    */
/* stage two 3x3 deconvolutions halving it; intermediate stages use batch  */
/* normalisation and LeakyReLU; the output stage has two deconvolutions    */
/* with LeakyReLU and a final 1x1 convolution with ReLU; downsampling is   */
/* 2x2 max pooling, upsampling 2x bilinear.  Base depth 64, three          */
/* downsizing steps (4x4 at the bottom for 32x32 maps).                    */
/*                                                                          */
/* Readings (the paper's network diagram is missing):                       */
/*  - the convolutions have stride 1 and zero padding 1, the deconvolutions */
/*    are stride-1 transposed convolutions, padding 1;                      */
/*  - levels l = 0..L have depths c_l = base 2^l; the deepest level (l = L) */
/*    is the 4x4 bottleneck, reached by L poolings;                         */
/*  - U-Net skips: a decoder stage upsamples the deeper features and        */
/*    concatenates them (first) with the encoder output of its level        */
/*    (second), then applies its two deconvolutions;                        */
/*  - the output stage is decoder level 0: its deconvolutions take          */
/*    LeakyReLU without batch normalisation;                                 */
/*  - PyTorch's conventions, the paper's framework: LeakyReLU slope 0.01,   */
/*    batch normalisation at inference y = g (x - mu) / sqrt(var + 1e-5) +  */
/*    b, bilinear sampling at half-pixel centres (source (i + 1/2)/2 - 1/2, */
/*    clamped at 0; the upper neighbour clamped at the last row / column).  */
/* Packed parameters, layer by layer: encoder levels 0..L (two 3x3 convs    */
/* each, W [Cout][Cin][3][3], b, g, beta, mu, var), decoder levels L-1..0   */
/* (two 3x3 deconvs each, W [Cin][Cout][3][3], b, and g, beta, mu, var      */
/* below level 0), then the head (W [Cout][c_0], b).                        */
/* ------------------------------------------------------------------------ */

static const double ORC_LRELU_SLOPE = 0.01, ORC_BN_EPS = 1e-5;

/* y[n,o,i,j] = b[o] + sum_{c,u,v} W[o,c,u,v] z[n,c,i+u-1,j+v-1], z the
 * channel concatenation of x1 (C1 channels) and x2 (C2, may be 0), zero
 * outside the map.  Output H x W. */
void orc_conv3x3s1(const double *x1, int C1, const double *x2, int C2, int N, int H, int W,
                   const double *Wt, const double *b, int Cout, double *y)
{
    const int Cin = C1 + C2;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++)
        for (int o = 0; o < Cout; o++)
            for (int i = 0; i < H; i++)
                for (int j = 0; j < W; j++) {
                    double acc = b ? b[o] : 0.0;
                    for (int c = 0; c < Cin; c++) {
                        const double *src = c < C1 ? x1 + ((long)n * C1 + c) * H * W
                                                   : x2 + ((long)n * C2 + (c - C1)) * H * W;
                        for (int u = 0; u < 3; u++)
                            for (int v = 0; v < 3; v++) {
                                int yy = i + u - 1, xx = j + v - 1;
                                if (yy < 0 || yy >= H || xx < 0 || xx >= W)
                                    continue;
                                acc += Wt[((o * Cin + c) * 3 + u) * 3 + v] * src[yy * W + xx];
                            }
                    }
                    y[(((long)n * Cout + o) * H + i) * W + j] = acc;
                }
}

/* y[n,o,p,q] = b[o] + sum over (c,i,j,u,v) with i+u-1 = p, j+v-1 = q of
 * W[c,o,u,v] z[n,c,i,j] (z as above): the scatter of every input pixel
 * through every tap, dropping taps outside the map.  Output H x W. */
void orc_convT3x3s1(const double *x1, int C1, const double *x2, int C2, int N, int H, int W,
                    const double *Wt, const double *b, int Cout, double *y)
{
    const int Cin = C1 + C2;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        double *yn = y + (long)n * Cout * H * W;
        for (int o = 0; o < Cout; o++)
            for (long e = 0; e < (long)H * W; e++)
                yn[(long)o * H * W + e] = b ? b[o] : 0.0;
        for (int c = 0; c < Cin; c++) {
            const double *src = c < C1 ? x1 + ((long)n * C1 + c) * H * W
                                       : x2 + ((long)n * C2 + (c - C1)) * H * W;
            for (int i = 0; i < H; i++)
                for (int j = 0; j < W; j++)
                    for (int o = 0; o < Cout; o++)
                        for (int u = 0; u < 3; u++)
                            for (int v = 0; v < 3; v++) {
                                int p = i + u - 1, q = j + v - 1;
                                if (p < 0 || p >= H || q < 0 || q >= W)
                                    continue;
                                yn[((long)o * H + p) * W + q] += Wt[((c * Cout + o) * 3 + u) * 3 + v] * src[i * W + j];
                            }
        }
    }
}

/* y[n,c,i,j] = max of x[n,c,2i..2i+1,2j..2j+1].  Output (H/2) x (W/2). */
void orc_maxpool2(const double *x, int N, int C, int H, int W, double *y)
{
    const int Ho = H / 2, Wo = W / 2;
    for (long nc = 0; nc < (long)N * C; nc++)
        for (int i = 0; i < Ho; i++)
            for (int j = 0; j < Wo; j++) {
                const double *s = x + nc * H * W;
                double m = s[(2 * i) * W + 2 * j];
                if (s[(2 * i) * W + 2 * j + 1] > m) m = s[(2 * i) * W + 2 * j + 1];
                if (s[(2 * i + 1) * W + 2 * j] > m) m = s[(2 * i + 1) * W + 2 * j];
                if (s[(2 * i + 1) * W + 2 * j + 1] > m) m = s[(2 * i + 1) * W + 2 * j + 1];
                y[(nc * Ho + i) * Wo + j] = m;
            }
}

/* Bilinear 2x upsampling at half-pixel centres: output row p samples input
 * row s = (p + 1/2) / 2 - 1/2 (s >= 0), between floor(s) and the next row
 * (clamped to the last), weights 1 - (s - floor s) and s - floor s; columns
 * alike.  Output (2H) x (2W). */
static void up_index(int p, int n, int *i0, int *i1, double *f)
{
    double s = (p + 0.5) / 2.0 - 0.5;
    if (s < 0.0) s = 0.0;
    *i0 = (int)floor(s);
    *i1 = *i0 + 1 < n ? *i0 + 1 : n - 1;
    *f = s - *i0;
}
void orc_upsample2(const double *x, int N, int C, int H, int W, double *y)
{
    const int Ho = 2 * H, Wo = 2 * W;
    for (long nc = 0; nc < (long)N * C; nc++)
        for (int p = 0; p < Ho; p++)
            for (int q = 0; q < Wo; q++) {
                int i0, i1, j0, j1;
                double fi, fj;
                up_index(p, H, &i0, &i1, &fi);
                up_index(q, W, &j0, &j1, &fj);
                const double *s = x + nc * H * W;
                const double top = (1.0 - fj) * s[i0 * W + j0] + fj * s[i0 * W + j1];
                const double bot = (1.0 - fj) * s[i1 * W + j0] + fj * s[i1 * W + j1];
                y[(nc * Ho + p) * Wo + q] = (1.0 - fi) * top + fi * bot;
            }
}

/* batch normalisation at inference (when g is given), then LeakyReLU. */
static void bn_lrelu(double *x, int N, int C, long HW, const double *g, const double *beta, const double *mu,
                     const double *var)
{
    for (int n = 0; n < N; n++)
        for (int c = 0; c < C; c++) {
            double *p = x + ((long)n * C + c) * HW;
            for (long e = 0; e < HW; e++) {
                double z = p[e];
                if (g)
                    z = g[c] * (z - mu[c]) / sqrt(var[c] + ORC_BN_EPS) + beta[c];
                p[e] = z >= 0.0 ? z : ORC_LRELU_SLOPE * z;
            }
        }
}

static long unet_layer_floats(int cin, int cout, int bn) { return 9L * cin * cout + cout + (bn ? 4L * cout : 0); }

long orc_unet_param_count(int cin, int cout, int base, int levels)
{
    long n = 0;
    for (int l = 0; l <= levels; l++) {
        const int c = base << l, ci = l == 0 ? cin : base << (l - 1);
        n += unet_layer_floats(ci, c, 1) + unet_layer_floats(c, c, 1);
    }
    for (int l = levels - 1; l >= 0; l--) {
        const int c = base << l;
        n += unet_layer_floats(2 * c + c, c, l > 0) + unet_layer_floats(c, c, l > 0);
    }
    return n + (long)cout * base + cout;
}

/* The forward pass of the U-Net above on x [N][cin][H][W] (H and W multiples
 * of 2^levels) into out [N][cout][H][W].  Returns 0, or -1 for a parameter
 * count or shape that does not fit. */
int orc_unet_forward(int cin, int cout, int base, int levels, const float *params, long n_params, const float *xf,
                     int N, int H, int W, double *out)
{
    if (levels < 1 || levels > 6 || base < 1 || H % (1 << levels) || W % (1 << levels) ||
        n_params != orc_unet_param_count(cin, cout, base, levels))
        return -1;
    double *P = widen(params, n_params);
    const double *p = P;
    double *enc[8];
    double *x = widen(xf, (long)N * cin * H * W);
    int h = H, w = W;
    const double *in = x;
    int ci = cin;
    double *pooled = NULL;
    for (int l = 0; l <= levels; l++) {
        const int c = base << l;
        const long hw = (long)h * w;
        double *a = (double *)malloc(sizeof(double) * N * c * hw);
        enc[l] = (double *)malloc(sizeof(double) * N * c * hw);
        for (int k = 0; k < 2; k++) {
            const int kin = k == 0 ? ci : c;
            const double *Wt = p, *b = p + 9L * kin * c, *g = b + c, *be = g + c, *mu = be + c, *var = mu + c;
            p = var + c;
            double *dst = k == 0 ? a : enc[l];
            orc_conv3x3s1(k == 0 ? in : a, kin, NULL, 0, N, h, w, Wt, b, c, dst);
            bn_lrelu(dst, N, c, hw, g, be, mu, var);
        }
        free(a);
        free(pooled);
        pooled = NULL;
        if (l < levels) {
            pooled = (double *)malloc(sizeof(double) * N * c * (hw / 4));
            orc_maxpool2(enc[l], N, c, h, w, pooled);
            h /= 2;
            w /= 2;
            in = pooled;
            ci = c;
        }
    }
    double *d = enc[levels];
    for (int l = levels - 1; l >= 0; l--) {
        const int c = base << l, cd = base << (l + 1);
        h *= 2;
        w *= 2;
        const long hw = (long)h * w;
        double *u = (double *)malloc(sizeof(double) * N * cd * hw);
        orc_upsample2(d, N, cd, h / 2, w / 2, u);
        double *a = (double *)malloc(sizeof(double) * N * c * hw);
        double *dn = (double *)malloc(sizeof(double) * N * c * hw);
        const int bn = l > 0;
        for (int k = 0; k < 2; k++) {
            const int kin = k == 0 ? cd + c : c;
            const double *Wt = p, *b = p + 9L * kin * c;
            const double *g = bn ? b + c : NULL, *be = bn ? b + 2 * c : NULL, *mu = bn ? b + 3 * c : NULL,
                         *var = bn ? b + 4 * c : NULL;
            p = b + c + (bn ? 4 * c : 0);
            if (k == 0)
                orc_convT3x3s1(u, cd, enc[l], c, N, h, w, Wt, b, c, a);
            else
                orc_convT3x3s1(a, c, NULL, 0, N, h, w, Wt, b, c, dn);
            bn_lrelu(k == 0 ? a : dn, N, c, hw, g, be, mu, var);
        }
        free(u);
        free(a);
        free(d);
        d = dn;
    }
    /* head: 1x1 convolution c_0 -> cout, ReLU */
    const double *Wh = p, *bh = p + (long)cout * base;
    const long hw = (long)H * W;
    for (int n = 0; n < N; n++)
        for (int o = 0; o < cout; o++)
            for (long e = 0; e < hw; e++) {
                double acc = bh[o];
                for (int c = 0; c < base; c++) acc += Wh[o * base + c] * d[((long)n * base + c) * hw + e];
                out[((long)n * cout + o) * hw + e] = acc > 0.0 ? acc : 0.0;
            }
    free(d);
    for (int l = 0; l < levels; l++) free(enc[l]);
    free(x);
    free(P);
    return 0;
}

/* Thread control for timing (not arithmetic): the OpenMP team size of the
 * loops above, and the current setting. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
