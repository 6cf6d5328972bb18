"""Seeded synthetic inputs for the Deep Radiance Caching hot path.

This module only makes input bytes.  It holds none of the method's
arithmetic (no convolution, no interpolation weights, no lat-long lookup of
the method's frames): the CUDA path and the FP64 oracle both consume what it
returns, so neither can borrow from the other through it.

The scenes and the 16 000-example dataset of arXiv 1910.02480 (Sec. 4) are
not available; these fields stand in for them with the paper's shapes:
7 x 32 x 32 hemispherical maps (radiance RGB, distance, normal -- Sec. 3.3),
noisy low-sample radiance, interior-room geometry (a unit box).

Recipe (all draws from numpy's PCG64 ``default_rng(seed)``):
  * weights: He init, W ~ N(0, 2 / (9 * Cin)) for every conv and transposed
    conv, b = 0 (or U(-0.1, 0.1) when ``bias=True``).  The paper-form U-Net
    adds batch-normalisation statistics gamma, var ~ U(0.5, 1.5) and beta,
    mean ~ U(-0.1, 0.1).
  * environment: m = 8 spherical-Gaussian lobes
    L(w) = sum_l a_l exp(lam_l (mu_l . w - 1)), mu_l uniform on the sphere,
    lam_l ~ U[2, 50], a_l RGB ~ U[0.1, 2] (or log-uniform on [1e-3, 1e3]).
  * one map: a first-hit point o uniform in the unit box and a normal n
    uniform on the sphere; texel (i, j) looks along the direction with polar
    angle (i + 0.5) * (pi/2) / H from n and azimuth (j + 0.5) * 2 pi / W about
    n in a tangent frame drawn at random per map.  Channels 0-2 =
    log1p(L) + N(0, sigma^2) (sigma = 0.3), channel 3 = distance from o to the
    box wall along the texel direction, channels 4-6 = inward normal of the
    wall hit.
  * G-buffer: positions uniform in the unit box, normals uniform on the
    sphere; lookup direction = mirror of the camera ray (0, 0, 1) about the
    camera-facing normal.
  * cache grid: g_x x g_y caches at pixels (floor((i + 0.5) W / g_x),
    floor((j + 0.5) H / g_y)); a cache takes the G-buffer's position and
    normal at its pixel.
"""
from __future__ import annotations

import numpy as np

CIN = 7
COUT = 3


def layer_shapes(widths, cin=CIN, cout=COUT):
    """(kind, W shape, b length) for conv_1..conv_S then convT_S..convT_1.

    conv W is [Cout, Cin, 3, 3]; convT W is [Cin, Cout, 3, 3] (the usual
    Conv2d / ConvTranspose2d layouts)."""
    out = []
    prev = cin
    for c in widths:
        out.append(("conv", (c, prev, 3, 3), c))
        prev = c
    S = len(widths)
    for s in range(S - 1, -1, -1):
        co = cout if s == 0 else widths[s - 1]
        out.append(("convT", (widths[s], co, 3, 3), co))
    return out


def weight_count(widths, cin=CIN, cout=COUT) -> int:
    return sum(int(np.prod(w)) + b for _, w, b in layer_shapes(widths, cin, cout))


def he_weights(widths, cin=CIN, cout=COUT, seed=0, bias=False) -> np.ndarray:
    """Packed float32 weights: each layer's W then b, in layer_shapes order."""
    rng = np.random.default_rng(seed)
    parts = []
    for kind, wshape, blen in layer_shapes(widths, cin, cout):
        fan_in = 9 * (wshape[1] if kind == "conv" else wshape[0])
        parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=wshape).ravel())
        if bias:
            parts.append(rng.uniform(-0.1, 0.1, size=blen))
        else:
            parts.append(np.zeros(blen))
    return np.concatenate(parts).astype(np.float32)


def unet_layer_shapes(base=64, levels=3, cin=CIN, cout=COUT):
    """The packed layout of the paper-form U-Net: (kind, W shape, number of
    per-channel vectors after W: bias, then gamma, beta, mean, var when the
    layer has batch normalisation).  Encoder levels 0..L (two convs each),
    decoder levels L-1..0 (two transposed convs each; the first takes the
    upsampled deeper features and the level's skip, concatenated; level 0
    without batch normalisation), then the 1x1 head."""
    out = []
    for lvl in range(levels + 1):
        c = base << lvl
        ci = cin if lvl == 0 else base << (lvl - 1)
        out.append(("conv", (c, ci, 3, 3), 5))
        out.append(("conv", (c, c, 3, 3), 5))
    for lvl in range(levels - 1, -1, -1):
        c = base << lvl
        nvec = 5 if lvl > 0 else 1
        out.append(("convT", (3 * c, c, 3, 3), nvec))
        out.append(("convT", (c, c, 3, 3), nvec))
    out.append(("head", (cout, base), 1))
    return out


def unet_params(base=64, levels=3, cin=CIN, cout=COUT, seed=0) -> np.ndarray:
    """Packed float32 U-Net parameters: He-initialised W, b ~ U(-0.1, 0.1),
    and batch-normalisation statistics gamma ~ U(0.5, 1.5), beta ~
    U(-0.1, 0.1), mean ~ U(-0.1, 0.1), var ~ U(0.5, 1.5)."""
    rng = np.random.default_rng(seed)
    parts = []
    for kind, wshape, nvec in unet_layer_shapes(base, levels, cin, cout):
        fan_in = wshape[1] if kind == "head" else 9 * (wshape[1] if kind == "conv" else wshape[0])
        parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), size=wshape).ravel())
        co = wshape[0] if kind in ("conv", "head") else wshape[1]
        parts.append(rng.uniform(-0.1, 0.1, size=co))
        if nvec == 5:
            parts += [rng.uniform(0.5, 1.5, size=co), rng.uniform(-0.1, 0.1, size=co),
                      rng.uniform(-0.1, 0.1, size=co), rng.uniform(0.5, 1.5, size=co)]
    return np.concatenate(parts).astype(np.float32)


def unpack_weights(w, widths, cin=CIN, cout=COUT):
    """Split a packed vector into [(W, b)] in layer_shapes order."""
    out, off = [], 0
    for _, wshape, blen in layer_shapes(widths, cin, cout):
        n = int(np.prod(wshape))
        out.append((w[off:off + n].reshape(wshape), w[off + n:off + n + blen]))
        off += n + blen
    assert off == w.size
    return out


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def lobes(seed=1, m=8, log_uniform=False):
    rng = np.random.default_rng(seed)
    mu = _unit(rng, m)
    lam = rng.uniform(2.0, 50.0, size=m)
    if log_uniform:
        a = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), size=(m, 3)))
    else:
        a = rng.uniform(0.1, 2.0, size=(m, 3))
    return mu, lam, a


def _radiance(dirs, lobe):
    """Environment radiance along unit directions dirs [..., 3] -> [..., 3]."""
    mu, lam, a = lobe
    cosang = np.einsum("...k,lk->...l", dirs, mu)
    return np.einsum("...l,lc->...c", np.exp(lam * (cosang - 1.0)), a)


def _box_exit(o, d):
    """Distance from o (inside [0,1]^3) to the box wall along d, and the
    inward normal of the wall hit.  o [..., 3], d [..., 3]."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t_hi = np.where(d > 0, (1.0 - o) / d, np.inf)
        t_lo = np.where(d < 0, (0.0 - o) / d, np.inf)
    t = np.minimum(t_hi, t_lo)
    axis = np.argmin(t, axis=-1)
    dist = np.take_along_axis(t, axis[..., None], axis=-1)[..., 0]
    nrm = np.zeros(d.shape, dtype=np.float64)
    sgn = -np.sign(np.take_along_axis(d, axis[..., None], axis=-1)[..., 0])
    np.put_along_axis(nrm, axis[..., None], sgn[..., None], axis=-1)
    return dist, nrm


def _random_frames(rng, nrm):
    """A tangent frame per normal with a random azimuth (data synthesis only)."""
    a = _unit(rng, nrm.shape[0])
    t = a - np.sum(a * nrm, axis=1, keepdims=True) * nrm
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    b = np.cross(nrm, t)
    return t, b


def hemisphere_maps(pos, nrm, H=32, W=32, lobe=None, sigma=0.3, seed=3,
                    frame_seed=7, noise="gauss", spp=4):
    """Noisy input maps [N,7,H,W] and the clean log radiance [N,3,H,W].

    noise="gauss": log1p(L) + N(0, sigma^2) on channels 0-2.
    noise="poisson": L * Poisson(spp)/spp per texel (shared over RGB), then
    log1p -- a stand-in for a low-sample path-traced estimate."""
    if lobe is None:
        lobe = lobes()
    pos = np.asarray(pos, dtype=np.float64)
    nrm = np.asarray(nrm, dtype=np.float64)
    nrm = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    N = pos.shape[0]
    t, b = _random_frames(np.random.default_rng(frame_seed), nrm)
    th = (np.arange(H) + 0.5) * (0.5 * np.pi) / H
    ph = (np.arange(W) + 0.5) * (2.0 * np.pi) / W
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    lx = st * np.cos(ph)[None, :]
    ly = st * np.sin(ph)[None, :]
    lz = np.broadcast_to(ct, (H, W))
    maps = np.empty((N, CIN, H, W), dtype=np.float32)
    clean = np.empty((N, 3, H, W), dtype=np.float32)
    rng = np.random.default_rng(seed)
    chunk = 256
    for n0 in range(0, N, chunk):
        n1 = min(N, n0 + chunk)
        d = (lx[None, :, :, None] * t[n0:n1, None, None, :]
             + ly[None, :, :, None] * b[n0:n1, None, None, :]
             + lz[None, :, :, None] * nrm[n0:n1, None, None, :])
        L = _radiance(d, lobe)  # [n,H,W,3]
        logL = np.log1p(L)
        clean[n0:n1] = np.moveaxis(logL, -1, 1)
        if noise == "gauss":
            noisy = logL + rng.normal(0.0, sigma, size=logL.shape)
        else:
            k = rng.poisson(spp, size=L.shape[:-1])[..., None] / float(spp)
            noisy = np.log1p(L * k)
        dist, wn = _box_exit(pos[n0:n1, None, None, :], d)
        maps[n0:n1, 0:3] = np.moveaxis(noisy, -1, 1)
        maps[n0:n1, 3] = dist
        maps[n0:n1, 4:7] = np.moveaxis(wn, -1, 1)
    return maps, clean


def gbuffer(width, height, seed=2):
    """Uniform first-hit positions in the unit box, random unit normals, and
    the mirror direction of the camera ray (0,0,1) about each normal."""
    rng = np.random.default_rng(seed)
    P = width * height
    pos = rng.uniform(0.0, 1.0, size=(P, 3))
    nrm = _unit(rng, P)
    view = np.array([0.0, 0.0, 1.0])
    facing = np.where((nrm @ view)[:, None] > 0, -nrm, nrm)
    d = view[None, :] - 2.0 * (facing @ view)[:, None] * facing
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return {"width": width, "height": height,
            "pos": pos.astype(np.float32), "nrm": nrm.astype(np.float32),
            "dir": d.astype(np.float32)}


def cache_grid(gbuf, gx, gy):
    """Caches at a regular gx x gy grid of pixels, taking the G-buffer's
    position and normal there.  Returns dict pos, nrm, pix (int32 x, y)."""
    W, H = gbuf["width"], gbuf["height"]
    xs = np.floor((np.arange(gx) + 0.5) * W / gx).astype(np.int64)
    ys = np.floor((np.arange(gy) + 0.5) * H / gy).astype(np.int64)
    px, py = np.meshgrid(xs, ys)
    px, py = px.ravel(), py.ravel()
    idx = py * W + px
    return {"pos": gbuf["pos"][idx].copy(), "nrm": gbuf["nrm"][idx].copy(),
            "pix": np.stack([px, py], axis=1).astype(np.int32)}


def image_radius(width, height, gx, gy):
    """Grid spacing in pixels, sqrt((W/gx)(H/gy))."""
    return float(np.sqrt((width / gx) * (height / gy)))


def world_radius(n):
    """Mean spacing of n points in the unit box, n^(-1/3)."""
    return float(n ** (-1.0 / 3.0))


def pass_counts(seed=4, passes=8, lo=200, hi=6000):
    """Cache counts per progressive pass and a 16x16 / 32x32 size per map."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(lo, hi + 1, size=passes)
    sizes = [np.where(rng.uniform(size=c) < 0.5, 16, 32) for c in counts]
    return counts, sizes
