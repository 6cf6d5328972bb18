"""FP64 CPU oracle for the Deep Radiance Caching hot path (arXiv 1910.02480).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or runs it,
and the two share no code: the oracle is ``drc_oracle.c``, direct loops in
double precision, compiled with gcc into ``_drc_oracle.so`` and called here
through ctypes on numpy arrays.

Functions (each cites the passage its C routine follows, see drc_oracle.c):
  conv3x3s2, convT3x3s2   the encoder / decoder layers (Sec. 3.3)
  conv_weight_grad        one layer's weight gradient (training, Sec. 3.3)
  forward                 the autoencoder with skip connections (Sec. 3.3)
  payload                 cosine-weighted hemisphere integral (Eq. 2, Sec. 3.3)
  interpolate             kNN + weights w = w_p w_n + w_p + eps (Sec. 3.2)
  l1_backward             L1 loss (Sec. 3.3, Eq. 7) and its exact gradient
  augment                 rotation / flip of training maps (Sec. 4)
  adam_step               the Adam step of the training (Sec. 4; Kingma & Ba)
  mis_indirect            the indirect term of Eq. 3 by multiple importance
                          sampling over the blended maps and the BRDF
                          (Sec. 3.2), with indirect_expected, its expectation
  gen_maps                the 7-channel input maps traced from cache points
                          in an analytic interior (Sec. 3.2-3.3)
  unet_forward            the paper's own network form: a U-Net (Sec. 3.3),
                          with its parts conv3x3s1, convT3x3s1, maxpool2,
                          upsample2 and unet_param_count

Pins (the tests under ``tests/test_oracle_*.py``) tie every function to
values fixed by the paper or by mathematics; the one function without such a
pin is marked "parity unpinned" below.  None is unpinned at present.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drc_oracle.c")
_SO = os.path.join(_HERE, "_drc_oracle.so")

F_ENCODE_INPUT = 1
F_DECODE_OUTPUT = 2
METRIC_IMAGE, METRIC_WORLD = 0, 1
WP_INVERSE, WP_LINEAR = 0, 1
INTERP_IRRADIANCE, INTERP_LOOKUP = 0, 1


def build(force: bool = False) -> str:
    """Compile drc_oracle.c with gcc (OpenMP, strict IEEE double)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i, l, d, u = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_uint
        lib.orc_conv3x3s2.argtypes = [P, i, i, i, i, P, P, i, P]
        lib.orc_convT3x3s2.argtypes = [P, i, i, i, i, P, P, i, P]
        lib.orc_weight_count.argtypes = [i, P, i, i]
        lib.orc_weight_count.restype = l
        lib.orc_forward.argtypes = [i, P, i, i, i, d, u, P, l, P, i, i, i, P]
        lib.orc_forward.restype = i
        lib.orc_payload.argtypes = [P, i, i, i, i, P]
        lib.orc_interp.argtypes = [i, i, i, P, P, P, P, P, i, i, P, P, P,
                                   i, i, i, i, d, d, d, l, l, P, P, P, P]
        lib.orc_mis_indirect.argtypes = [i, i, i, P, P, l, i, P, P, P, P, i, P, P, P]
        lib.orc_mis_indirect.restype = i
        lib.orc_indirect_expected.argtypes = [i, i, i, P, P, l, i, P, P, P, P, i, P]
        lib.orc_indirect_expected.restype = i
        lib.orc_gen_maps.argtypes = [i, P, P, i, i, P, P, P, i, P, i, P, P, P]
        lib.orc_gen_maps.restype = i
        lib.orc_interp.restype = i
        lib.orc_l1_backward.argtypes = [i, P, i, i, i, d, u, P, l, P, P, i, i,
                                        i, i, P, P, P]
        lib.orc_l1_backward.restype = d
        lib.orc_conv_wgrad.argtypes = [P, i, i, i, i, P, i, i, P]
        lib.orc_augment.argtypes = [P, i, i, i, i, P, P]
        lib.orc_conv3x3s1.argtypes = [P, i, P, i, i, i, i, P, P, i, P]
        lib.orc_convT3x3s1.argtypes = [P, i, P, i, i, i, i, P, P, i, P]
        lib.orc_maxpool2.argtypes = [P, i, i, i, i, P]
        lib.orc_upsample2.argtypes = [P, i, i, i, i, P]
        lib.orc_unet_param_count.argtypes = [i, i, i, i]
        lib.orc_unet_param_count.restype = l
        lib.orc_unet_forward.argtypes = [i, i, i, i, P, l, P, i, i, i, P]
        lib.orc_unet_forward.restype = i
        lib.orc_adam_step.argtypes = [P, P, P, P, l, i, d, d, d, d]
        lib.orc_set_threads.argtypes = [i]
        lib.orc_get_threads.restype = i
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's loops (timing only)."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def weight_count(widths, cin=7, cout=3) -> int:
    w = np.asarray(widths, dtype=np.int32)
    return int(_load().orc_weight_count(len(w), _ptr(w), cin, cout))


def conv3x3s2(x, w, b=None):
    """3x3 conv, stride 2, pad 1.  x [N,Cin,H,W], w [Cout,Cin,3,3]."""
    x, w = _f64(x), _f64(w)
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    assert w.shape == (Cout, Cin, 3, 3) and H % 2 == 0 and W % 2 == 0
    y = np.empty((N, Cout, H // 2, W // 2))
    bb = None if b is None else _f64(b)
    _load().orc_conv3x3s2(_ptr(x), N, Cin, H, W, _ptr(w), _ptr(bb), Cout, _ptr(y))
    return y


def convT3x3s2(x, w, b=None):
    """3x3 transposed conv, stride 2, pad 1, output pad 1.  w [Cin,Cout,3,3]."""
    x, w = _f64(x), _f64(w)
    N, Cin, H, W = x.shape
    Cout = w.shape[1]
    assert w.shape == (Cin, Cout, 3, 3)
    y = np.empty((N, Cout, 2 * H, 2 * W))
    bb = None if b is None else _f64(b)
    _load().orc_convT3x3s2(_ptr(x), N, Cin, H, W, _ptr(w), _ptr(bb), Cout, _ptr(y))
    return y


def conv_weight_grad(x, g, transposed=False):
    """Weight gradient of one layer from its input x [N,Cin,H,W] and output
    gradient g: a conv (g [N,Cout,H/2,W/2]) -> dW [Cout,Cin,3,3], or a
    transposed conv (g [N,Cout,2H,2W]) -> dW [Cin,Cout,3,3] (Sec. 3.3)."""
    x, g = _f64(x), _f64(g)
    N, Cin, H, W = x.shape
    Cout = g.shape[1]
    if transposed:
        assert g.shape == (N, Cout, 2 * H, 2 * W)
        dw = np.empty((Cin, Cout, 3, 3))
    else:
        assert g.shape == (N, Cout, H // 2, W // 2) and H % 2 == 0 and W % 2 == 0
        dw = np.empty((Cout, Cin, 3, 3))
    _load().orc_conv_wgrad(_ptr(x), N, Cin, H, W, _ptr(g), Cout, int(transposed), _ptr(dw))
    return dw


def forward(weights, x, widths, cin=7, cout=3, out_relu=False, exposure=1.0,
            flags=0):
    """Denoise [N,cin,H,W] float32 maps -> [N,cout,H,W] float64."""
    w = _f32(weights)
    x = _f32(x)
    wd = np.asarray(widths, dtype=np.int32)
    N, C, H, W = x.shape
    assert C == cin
    out = np.empty((N, cout, H, W))
    rc = _load().orc_forward(len(wd), _ptr(wd), cin, cout, int(out_relu),
                             float(exposure), flags, _ptr(w), w.size, _ptr(x),
                             N, H, W, _ptr(out))
    if rc:
        raise ValueError("oracle forward: bad network description (%d)" % rc)
    return out


def payload(L):
    """E/pi per map and channel from linear radiance maps [N,C,H,W]."""
    L = _f64(L)
    N, C, H, W = L.shape
    out = np.empty((N, C))
    _load().orc_payload(_ptr(L), N, C, H, W, _ptr(out))
    return out


def interpolate(caches, gbuf, k, metric, wp_form, mode, r, eps=1e-6,
                delta_rel=1e-3, p_range=None, want_neighbors=False, want_weights=False):
    """Blend cached values at every G-buffer pixel (Sec. 3.2).

    caches: dict with 'payload' [n,3], 'pos' [n,3], 'nrm' [n,3], 'pix' [n,2]
            int32 (x, y), and 'maps' [n,3,H,W] linear radiance for LOOKUP.
    gbuf:   dict with 'width', 'height', 'pos' [P,3], 'nrm' [P,3],
            'dir' [P,3] (LOOKUP only).
    Returns out [p1-p0, 3] (and neighbour indices [.,k], the k+1 smallest
    squared distances [.,k+1] when want_neighbors; and the normalised weights
    [.,k] last when want_weights).
    """
    n = caches["pos"].shape[0]
    maps = caches.get("maps")
    mH = mW = 0
    if maps is not None:
        maps = _f32(maps)
        mH, mW = maps.shape[2], maps.shape[3]
    pay = _f32(caches["payload"]) if caches.get("payload") is not None else None
    cpos, cnrm = _f32(caches["pos"]), _f32(caches["nrm"])
    cpix = np.ascontiguousarray(caches["pix"], dtype=np.int32)
    width, height = int(gbuf["width"]), int(gbuf["height"])
    gpos, gnrm = _f32(gbuf["pos"]), _f32(gbuf["nrm"])
    gdir = _f32(gbuf["dir"]) if gbuf.get("dir") is not None else None
    p0, p1 = (0, width * height) if p_range is None else p_range
    out = np.empty((p1 - p0, 3))
    idx = np.empty((p1 - p0, k), dtype=np.int32) if want_neighbors else None
    d2 = np.empty((p1 - p0, k + 1)) if want_neighbors else None
    wts = np.empty((p1 - p0, k)) if want_weights else None
    rc = _load().orc_interp(n, mH, mW, _ptr(maps), _ptr(pay), _ptr(cpos),
                            _ptr(cnrm), _ptr(cpix), width, height, _ptr(gpos),
                            _ptr(gnrm), _ptr(gdir), k, metric, wp_form, mode,
                            float(r), float(eps), float(delta_rel), p0, p1,
                            _ptr(out), _ptr(idx), _ptr(d2), _ptr(wts))
    if rc:
        raise ValueError("oracle interpolate: bad arguments (%d)" % rc)
    res = (out,) + ((idx, d2) if want_neighbors else ()) + ((wts,) if want_weights else ())
    return res if len(res) > 1 else out


def l1_backward(weights, x, target, widths, cin=7, cout=3, out_relu=False,
                exposure=1.0, flags=0, grad_out=False):
    """Loss and gradients: returns (loss, dweights [n_floats], dinput)."""
    w, x, t = _f32(weights), _f32(x), _f32(target)
    wd = np.asarray(widths, dtype=np.int32)
    N, C, H, W = x.shape
    dw = np.empty(w.size)
    dx = np.empty(x.shape)
    rc = ctypes.c_int(0)
    loss = _load().orc_l1_backward(len(wd), _ptr(wd), cin, cout, int(out_relu),
                                   float(exposure), flags, _ptr(w), w.size,
                                   _ptr(x), _ptr(t), N, H, W, int(grad_out),
                                   _ptr(dw), _ptr(dx), ctypes.byref(rc))
    if rc.value:
        raise ValueError("oracle backward: bad network description (%d)" % rc.value)
    return loss, dw, dx


def augment(x, codes):
    """The eight symmetries of square maps, one per map: code = r + 4 f is a
    column mirror (f = 1) followed by r counter-clockwise quarter turns.
    x [N, C, H, W] (H == W), codes [N] in 0..7; returns float64."""
    x = _f64(x)
    N, C, H, W = x.shape
    if H != W:
        raise ValueError("augment: maps must be square")
    cd = np.ascontiguousarray(codes, dtype=np.int32)
    if cd.shape != (N,) or np.any((cd < 0) | (cd > 7)):
        raise ValueError("augment: one code in 0..7 per map")
    y = np.empty_like(x)
    _load().orc_augment(_ptr(x), N, C, H, W, _ptr(cd), _ptr(y))
    return y


def adam_step(w, g, m, v, t, lr=6e-5, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Alg. 1) on copies: returns the new
    (w, m, v) in float64."""
    w, g, m, v = _f64(w).copy(), _f64(g), _f64(m).copy(), _f64(v).copy()
    if not (w.shape == g.shape == m.shape == v.shape):
        raise ValueError("adam_step: shapes differ")
    if t < 1:
        raise ValueError("adam_step: t counts from 1")
    _load().orc_adam_step(_ptr(w), _ptr(g), _ptr(m), _ptr(v), w.size, int(t), float(lr), float(beta1),
                          float(beta2), float(eps))
    return w, m, v


def conv3x3s1(x, w, b=None, x2=None):
    """3x3 convolution, stride 1, padding 1, of x (concatenated with x2 along
    channels when given): x [N, C1, H, W], w [Cout, C1 + C2, 3, 3]."""
    x = _f64(x)
    N, C1, H, W = x.shape
    x2 = None if x2 is None else _f64(x2)
    C2 = 0 if x2 is None else x2.shape[1]
    w = _f64(w)
    y = np.empty((N, w.shape[0], H, W))
    _load().orc_conv3x3s1(_ptr(x), C1, _ptr(x2), C2, N, H, W, _ptr(w), _ptr(None if b is None else _f64(b)),
                          w.shape[0], _ptr(y))
    return y


def convT3x3s1(x, w, b=None, x2=None):
    """3x3 transposed convolution, stride 1, padding 1: w [C1 + C2, Cout, 3, 3]."""
    x = _f64(x)
    N, C1, H, W = x.shape
    x2 = None if x2 is None else _f64(x2)
    C2 = 0 if x2 is None else x2.shape[1]
    w = _f64(w)
    y = np.empty((N, w.shape[1], H, W))
    _load().orc_convT3x3s1(_ptr(x), C1, _ptr(x2), C2, N, H, W, _ptr(w), _ptr(None if b is None else _f64(b)),
                           w.shape[1], _ptr(y))
    return y


def maxpool2(x):
    x = _f64(x)
    N, C, H, W = x.shape
    y = np.empty((N, C, H // 2, W // 2))
    _load().orc_maxpool2(_ptr(x), N, C, H, W, _ptr(y))
    return y


def upsample2(x):
    """Bilinear 2x upsampling at half-pixel centres."""
    x = _f64(x)
    N, C, H, W = x.shape
    y = np.empty((N, C, 2 * H, 2 * W))
    _load().orc_upsample2(_ptr(x), N, C, H, W, _ptr(y))
    return y


def unet_param_count(base=64, levels=3, cin=7, cout=3) -> int:
    return int(_load().orc_unet_param_count(cin, cout, base, levels))


def unet_forward(params, x, base=64, levels=3, cin=7, cout=3):
    """The paper's U-Net (readings in drc_oracle.c) on x [N, cin, H, W]."""
    p, x = _f32(params), _f32(x)
    N, C, H, W = x.shape
    out = np.empty((N, cout, H, W))
    rc = _load().orc_unet_forward(cin, cout, base, levels, _ptr(p), p.size, _ptr(x), N, H, W, _ptr(out))
    if rc:
        raise ValueError("oracle unet: parameter count or shape does not fit")
    return out


def _mis_args(caches, nbr_idx, nbr_w, gnrm, albedo):
    maps = _f32(caches["maps"])
    n, _, H, W = maps.shape
    idx = np.ascontiguousarray(nbr_idx, dtype=np.int32)
    P, k = idx.shape
    w = _f64(nbr_w)
    if w.shape != (P, k):
        raise ValueError("nbr_w must match nbr_idx")
    return maps, n, H, W, _f32(caches["nrm"]), idx, P, k, w, _f32(gnrm), _f32(albedo)


def mis_indirect(caches, nbr_idx, nbr_w, gnrm, albedo, u, want_margin=False):
    """The indirect term at P pixels: caches 'maps' [n,3,H,W] (linear
    radiance) and 'nrm'; the pixels' k caches and normalised weights
    [P,k]; pixel normals and albedos [P,3]; uniforms u [P,S,4].  Readings
    in drc_oracle.c.  Returns [P,3], and with want_margin also [P]: per
    pixel the smallest distance of a sample's continuous-valued decision
    (texel of a direction, hemisphere, frame) from where it changes, in
    units of the float32 error of that value (below 1: a float evaluation
    may rightly decide otherwise)."""
    maps, n, H, W, cnrm, idx, P, k, w, gn, alb = _mis_args(caches, nbr_idx, nbr_w, gnrm, albedo)
    u = _f64(u)
    if u.shape[0] != P or u.shape[2] != 4:
        raise ValueError("u must be [P, S, 4]")
    out = np.empty((P, 3))
    margin = np.empty(P) if want_margin else None
    rc = _load().orc_mis_indirect(n, H, W, _ptr(maps), _ptr(cnrm), P, k, _ptr(idx), _ptr(w), _ptr(gn), _ptr(alb),
                                  u.shape[1], _ptr(u), _ptr(out), _ptr(margin))
    if rc:
        raise ValueError("oracle mis_indirect: bad arguments")
    return (out, margin) if want_margin else out


def indirect_expected(caches, nbr_idx, nbr_w, gnrm, albedo, m=16):
    """The expectation of mis_indirect by quadrature (m x m cells per texel)."""
    maps, n, H, W, cnrm, idx, P, k, w, gn, alb = _mis_args(caches, nbr_idx, nbr_w, gnrm, albedo)
    out = np.empty((P, 3))
    rc = _load().orc_indirect_expected(n, H, W, _ptr(maps), _ptr(cnrm), P, k, _ptr(idx), _ptr(w), _ptr(gn),
                                       _ptr(alb), int(m), _ptr(out))
    if rc:
        raise ValueError("oracle indirect_expected: bad arguments")
    return out


def gen_maps(pos, nrm, H, W, wall_alb, wall_em=None, light=None, spheres=(), D=3, u=None, want_margin=False):
    """Maps [n, 7, H, W] traced from cache points pos [n,3] (inside the unit
    box) with normals nrm [n,3]: radiance leaving the first hit without its
    own emission (D cosine-sampled bounces), distance, hit normal.  wall_alb,
    wall_em: [6,3] for -x, +x, -y, +y, -z, +z; light: (x0, x1, y0, y1, Le
    rgb) on the ceiling; spheres: rows (cx, cy, cz, r, albedo rgb); u:
    uniforms [n, H, W, D, 2] (default zeros).  With want_margin also
    [n, H, W]: per texel the smallest margin of its path's discrete
    decisions in units of their float32 error (below 1: a float evaluation
    may rightly hit another surface or light)."""
    pos, nrm = _f32(pos), _f32(nrm)
    n = pos.shape[0]
    wa = _f64(wall_alb).reshape(6, 3)
    we = np.zeros((6, 3)) if wall_em is None else _f64(wall_em).reshape(6, 3)
    lt = None if light is None else _f64(light).reshape(7)
    sp = _f64(np.asarray(spheres, dtype=np.float64).reshape(-1, 7)) if len(spheres) else np.zeros((0, 7))
    u = np.zeros((n, H, W, max(D, 1), 2)) if u is None else _f64(u)
    if u.shape[:3] != (n, H, W) or u.shape[3] < D or u.shape[4] != 2:
        raise ValueError("u must be [n, H, W, D, 2]")
    u = np.ascontiguousarray(u[:, :, :, :max(D, 1)])
    out = np.empty((n, 7, H, W))
    margin = np.empty((n, H, W)) if want_margin else None
    rc = _load().orc_gen_maps(n, _ptr(pos), _ptr(nrm), H, W, _ptr(wa), _ptr(we), _ptr(lt), sp.shape[0], _ptr(sp),
                              D, _ptr(u), _ptr(out), _ptr(margin))
    if rc:
        raise ValueError("oracle gen_maps: points must lie inside the unit box, normals nonzero")
    return (out, margin) if want_margin else out

