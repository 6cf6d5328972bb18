"""Deep Radiance Caching hot path on one GB300 (sm_103a).

Python binding of the C ABI in ``include/drc.h`` (``libdrc.so``, built from
``csrc/`` by ``build.py``).  This module only marshals arguments: device
memory and streams come from PyTorch, every step of the computation runs in
the library's CUDA kernels.  There is no CPU fallback: if the library is
missing or no sm_103a device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_INTERNAL = range(7)
STATUS_NAMES = {0: "DRC_OK", 1: "DRC_ERR_INVALID_ARG", 2: "DRC_ERR_UNSUPPORTED", 3: "DRC_ERR_OOM",
                4: "DRC_ERR_CUDA", 5: "DRC_ERR_TIMEOUT", 6: "DRC_ERR_INTERNAL"}
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}

F_ENCODE_INPUT = 0x1
F_DECODE_OUTPUT = 0x2
F_DEBUG_STALL = 0x100
METRIC_IMAGE, METRIC_WORLD = 0, 1
WP_INVERSE, WP_LINEAR = 0, 1
INTERP_IRRADIANCE, INTERP_LOOKUP = 0, 1
BWD_L1_TARGET, BWD_GRAD_OUT, BWD_RECOMPUTE_ENCODER = 0x10, 0x20, 0x40


class DrcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("in_channels", ctypes.c_int), ("out_channels", ctypes.c_int),
                ("num_stages", ctypes.c_int), ("widths", ctypes.c_int * 8),
                ("out_relu", ctypes.c_int), ("precision", ctypes.c_int),
                ("exposure", ctypes.c_float), ("max_maps", ctypes.c_int),
                ("max_hw", ctypes.c_int), ("wait_timeout_ms", ctypes.c_int)]


class Caches(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("maps", ctypes.c_void_p), ("payload", ctypes.c_void_p),
                ("pos", ctypes.c_void_p), ("nrm", ctypes.c_void_p), ("pix", ctypes.c_void_p)]


class GBuffer(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("pos", ctypes.c_void_p),
                ("nrm", ctypes.c_void_p), ("dir", ctypes.c_void_p)]


class SizeClass(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("max_maps", ctypes.c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


class InterpParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("metric", ctypes.c_int), ("wp_form", ctypes.c_int),
                ("mode", ctypes.c_int), ("r", ctypes.c_float), ("eps", ctypes.c_float),
                ("delta_rel", ctypes.c_float), ("nbr_out", ctypes.c_void_p), ("nbr_w", ctypes.c_void_p)]


class Scene(ctypes.Structure):
    _fields_ = [("wall_alb", (ctypes.c_float * 3) * 6), ("wall_em", (ctypes.c_float * 3) * 6),
                ("has_light", ctypes.c_int), ("light", ctypes.c_float * 7), ("nsph", ctypes.c_int),
                ("sph", (ctypes.c_float * 7) * 64)]


def make_scene(wall_alb, wall_em=None, light=None, spheres=()):
    """A drc_scene: wall albedos / emissions [6,3] (-x, +x, -y, +y, -z,
    +z), an optional ceiling light (x0, x1, y0, y1, Le rgb) and sphere rows
    (cx, cy, cz, r, albedo rgb)."""
    import numpy as np
    sc = Scene()
    wa = np.asarray(wall_alb, dtype=np.float32).reshape(6, 3)
    we = np.zeros((6, 3), np.float32) if wall_em is None else np.asarray(wall_em, dtype=np.float32).reshape(6, 3)
    for i in range(6):
        for c in range(3):
            sc.wall_alb[i][c] = float(wa[i, c])
            sc.wall_em[i][c] = float(we[i, c])
    if light is not None:
        sc.has_light = 1
        for i, v in enumerate(np.asarray(light, dtype=np.float32).reshape(7)):
            sc.light[i] = float(v)
    sp = np.asarray(spheres, dtype=np.float32).reshape(-1, 7) if len(spheres) else np.zeros((0, 7), np.float32)
    if sp.shape[0] > 64:
        raise ValueError("at most 64 spheres")
    sc.nsph = sp.shape[0]
    for s_ in range(sp.shape[0]):
        for c in range(7):
            sc.sph[s_][c] = float(sp[s_, c])
    return sc


class IndirectParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("nbr", ctypes.c_void_p), ("nbr_w", ctypes.c_void_p), ("S", ctypes.c_int),
                ("u", ctypes.c_void_p), ("albedo", ctypes.c_void_p), ("emit", ctypes.c_void_p),
                ("direct", ctypes.c_void_p)]


_lib = None


def load_library():
    """Load libdrc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdrc.so is not built: run paper_1910_02480_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, U = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint
    lib.drc_weight_count.argtypes = [ctypes.POINTER(Config)]
    lib.drc_weight_count.restype = ctypes.c_size_t
    lib.drc_create.argtypes = [ctypes.POINTER(Config), P, ctypes.c_size_t, ctypes.POINTER(P)]
    lib.drc_create.restype = I
    lib.drc_set_weights.argtypes = [P, P, I, P]
    lib.drc_set_weights.restype = I
    lib.drc_destroy.argtypes = [P]
    lib.drc_destroy.restype = I
    lib.drc_denoise.argtypes = [P, P, P, P, I, I, I, U, P]
    lib.drc_denoise.restype = I
    lib.drc_interpolate.argtypes = [P, ctypes.POINTER(Caches), ctypes.POINTER(GBuffer),
                                    ctypes.POINTER(InterpParams), P, P]
    lib.drc_interpolate.restype = I
    lib.drc_interpolate_static.argtypes = [ctypes.POINTER(Caches), ctypes.POINTER(GBuffer),
                                           ctypes.POINTER(InterpParams), P, P]
    lib.drc_interpolate_static.restype = I
    lib.drc_indirect.argtypes = [P, ctypes.POINTER(Caches), ctypes.POINTER(GBuffer), ctypes.POINTER(IndirectParams),
                                 P, P]
    lib.drc_indirect.restype = I
    lib.drc_gen_maps.argtypes = [P, ctypes.POINTER(Scene), I, P, P, I, I, I, P, P, P]
    lib.drc_gen_maps.restype = I
    lib.drc_fd_loss64.argtypes = [P, P, P, P, I, I, I, U, P, P]
    lib.drc_fd_loss64.restype = I
    lib.drc_pass_points.argtypes = [I, I, I, I, P, I, ctypes.POINTER(I)]
    lib.drc_pass_points.restype = I
    lib.drc_backward.argtypes = [P, P, P, I, I, I, U, P, P, P, P]
    lib.drc_backward.restype = I
    lib.drc_frame_host.argtypes = [P, P, I, I, I, U, ctypes.POINTER(Caches), ctypes.POINTER(GBuffer),
                                   ctypes.POINTER(InterpParams), P, P]
    lib.drc_frame_host.restype = I
    lib.drc_weight_grad.argtypes = [P, P, P, I, I, I, I, I, I, I, P, P]
    lib.drc_weight_grad.restype = I
    lib.drc_augment.argtypes = [P, P, P, I, I, I, I, P, P]
    lib.drc_augment.restype = I
    F = ctypes.c_float
    lib.drc_adam_step.argtypes = [P, P, P, P, P, ctypes.c_size_t, I, F, F, F, F, P]
    lib.drc_adam_step.restype = I
    SZ = ctypes.c_size_t
    lib.drc_unet_param_count.argtypes = [I, I, I, I]
    lib.drc_unet_param_count.restype = SZ
    lib.drc_unet_workspace_bytes.argtypes = [I, I, I, I, I, I, I]
    lib.drc_unet_workspace_bytes.restype = SZ
    lib.drc_unet_tensor_cores.argtypes = [I, I, I, I, I, I]
    lib.drc_unet_tensor_cores.restype = I
    lib.drc_unet_forward.argtypes = [P, I, I, I, I, P, P, P, I, I, I, P, SZ, P]
    lib.drc_unet_forward.restype = I
    lib.drc_get_status.argtypes = [P, P]
    lib.drc_get_status.restype = I
    lib.drc_last_error.argtypes = [P]
    lib.drc_last_error.restype = ctypes.c_char_p
    lib.drc_launch_count.argtypes = [P, ctypes.POINTER(ctypes.c_ulonglong)]
    lib.drc_launch_count.restype = I
    lib.drc_set_timing.argtypes = [P, I]
    lib.drc_set_timing.restype = I
    lib.drc_read_timing.argtypes = [P, ctypes.POINTER(KernelTime), I, ctypes.POINTER(I)]
    lib.drc_read_timing.restype = I
    PP = ctypes.POINTER(P)
    lib.drc_plan_create.argtypes = [P, ctypes.POINTER(SizeClass), I, U, PP]
    lib.drc_plan_create.restype = I
    lib.drc_plan_launch.argtypes = [P, P, PP, PP, PP, U, P]
    lib.drc_plan_launch.restype = I
    lib.drc_plan_describe.argtypes = [P, I, I, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.drc_plan_describe.restype = I
    lib.drc_calibrate.argtypes = [P, P, I, I, I, U, P]
    lib.drc_calibrate.restype = I
    lib.drc_autotune.argtypes = [P, I, I, I]
    lib.drc_autotune.restype = I
    lib.drc_describe_layer.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.drc_describe_layer.restype = I
    lib.drc_autotune_cached.argtypes = [P, I, I, I, ctypes.c_char_p, ctypes.POINTER(I)]
    lib.drc_autotune_cached.restype = I
    lib.drc_save_checkpoint.argtypes = [P, ctypes.c_char_p, P, P, I, P]
    lib.drc_save_checkpoint.restype = I
    lib.drc_load_checkpoint.argtypes = [P, ctypes.c_char_p, P, P, ctypes.POINTER(I), P]
    lib.drc_load_checkpoint.restype = I
    lib.drc_set_memory_limit.argtypes = [P, ctypes.c_size_t]
    lib.drc_set_memory_limit.restype = I
    lib.drc_memory_in_use.argtypes = [P]
    lib.drc_memory_in_use.restype = ctypes.c_size_t
    lib.drc_get_weights.argtypes = [P, P, I, P]
    lib.drc_get_weights.restype = I
    lib.drc_plan_destroy.argtypes = [P]
    lib.drc_plan_destroy.restype = I
    _lib = lib
    return lib


def make_config(widths, precision="fp32", exposure=1.0, out_relu=False, max_maps=0, max_hw=0,
                wait_timeout_ms=0, in_channels=7, out_channels=3):
    c = Config()
    c.in_channels = in_channels
    c.out_channels = out_channels
    c.num_stages = len(widths)
    for i, w in enumerate(widths):
        c.widths[i] = int(w)
    c.out_relu = int(bool(out_relu))
    c.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    c.exposure = float(exposure)
    c.max_maps = int(max_maps)
    c.max_hw = int(max_hw)
    c.wait_timeout_ms = int(wait_timeout_ms)
    return c


def weight_count(widths) -> int:
    cfg = make_config(widths)
    return int(load_library().drc_weight_count(ctypes.byref(cfg)))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def pass_points(width, height, spacing0, pass_):
    """drc_pass_points: the image-plane sample points (int32 [n, 2], x, y)
    of progressive pass `pass_` on grids halving from spacing0 (Sec. 3.2)."""
    import numpy as np
    lib = load_library()
    cnt = ctypes.c_int(0)
    rc = lib.drc_pass_points(int(width), int(height), int(spacing0), int(pass_), None, 0, ctypes.byref(cnt))
    if rc not in (OK, ERR_INVALID_ARG):
        raise DrcError("drc_pass_points: %s" % STATUS_NAMES.get(rc, rc))
    pix = np.zeros((max(cnt.value, 1), 2), dtype=np.int32)
    rc = lib.drc_pass_points(int(width), int(height), int(spacing0), int(pass_),
                             pix.ctypes.data_as(ctypes.c_void_p), cnt.value, ctypes.byref(cnt))
    if rc != OK:
        raise DrcError("drc_pass_points: %s" % STATUS_NAMES.get(rc, rc))
    return pix[:cnt.value]


class Context:
    """One drc_ctx: a network (widths, precision, exposure) with its weights."""

    def __init__(self, widths, weights=None, precision="fp32", exposure=1.0, out_relu=False,
                 max_maps=0, max_hw=0, wait_timeout_ms=0):
        self._lib = load_library()
        self.widths = list(widths)
        self.precision = precision
        self.exposure = float(exposure)
        self.cfg = make_config(widths, precision, exposure, out_relu, max_maps, max_hw, wait_timeout_ms)
        self.n_weights = int(self._lib.drc_weight_count(ctypes.byref(self.cfg)))
        self._ctx = ctypes.c_void_p()
        wh = None
        if weights is not None and not hasattr(weights, "is_cuda"):
            wh = np.ascontiguousarray(weights, dtype=np.float32)
            if wh.size != self.n_weights:
                raise ValueError("expected %d weights, got %d" % (self.n_weights, wh.size))
        rc = self._lib.drc_create(ctypes.byref(self.cfg),
                                  None if wh is None else wh.ctypes.data_as(ctypes.c_void_p),
                                  self.n_weights if wh is not None else 0, ctypes.byref(self._ctx))
        if rc != OK:
            raise DrcError(rc, "drc_create failed")
        if weights is not None and hasattr(weights, "is_cuda"):
            self.set_weights(weights)

    def _check(self, rc, what):
        if rc != OK:
            msg = self._lib.drc_last_error(self._ctx).decode()
            raise DrcError(rc, "%s: %s" % (what, msg))

    def close(self):
        if self._ctx:
            self._lib.drc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, weights, stream=None):
        if hasattr(weights, "is_cuda") and weights.is_cuda:
            assert weights.dtype.itemsize == 4 and weights.numel() == self.n_weights
            w = weights.contiguous()
            self._check(self._lib.drc_set_weights(self._ctx, _ptr(w), 1, _stream(stream)), "drc_set_weights")
        else:
            w = np.ascontiguousarray(weights, dtype=np.float32)
            if w.size != self.n_weights:
                raise ValueError("expected %d weights, got %d" % (self.n_weights, w.size))
            self._check(self._lib.drc_set_weights(self._ctx, w.ctypes.data_as(ctypes.c_void_p), 0, None),
                        "drc_set_weights")

    def denoise(self, x, out=None, payload=None, flags=0, stream=None, want_payload=False):
        """x: cuda float32 [N,7,H,W] -> out [N,3,H,W] (and payload [N,3])."""
        import torch
        N, C, H, W = x.shape
        if out is None:
            out = torch.empty((N, 3, H, W), dtype=torch.float32, device=x.device)
        if payload is None and want_payload:
            payload = torch.empty((N, 3), dtype=torch.float32, device=x.device)
        rc = self._lib.drc_denoise(self._ctx, _ptr(x), _ptr(out), _ptr(payload), N, H, W, flags,
                                   _stream(stream))
        self._check(rc, "drc_denoise")
        return (out, payload) if (payload is not None) else out

    def interpolate(self, caches, gbuf, k, metric, wp_form, mode, r, eps=1e-6, delta_rel=1e-3,
                    out=None, nbr_out=None, nbr_w=None, stream=None):
        """caches / gbuf: dicts of cuda tensors (see drc.h).  nbr_out [P,k]
        int32 and nbr_w [P,k] float32 (which needs nbr_out) receive the
        chosen caches and their normalised weights."""
        import torch
        c = Caches()
        c.n = int(caches["nrm"].shape[0])
        maps = caches.get("maps")
        c.H = int(maps.shape[2]) if maps is not None else 0
        c.W = int(maps.shape[3]) if maps is not None else 0
        c.maps = _ptr(maps)
        c.payload = _ptr(caches.get("payload"))
        c.pos = _ptr(caches.get("pos"))
        c.nrm = _ptr(caches.get("nrm"))
        c.pix = _ptr(caches.get("pix"))
        g = GBuffer()
        g.width, g.height = int(gbuf["width"]), int(gbuf["height"])
        g.pos = _ptr(gbuf.get("pos"))
        g.nrm = _ptr(gbuf.get("nrm"))
        g.dir = _ptr(gbuf.get("dir"))
        p = InterpParams()
        p.k, p.metric, p.wp_form, p.mode = int(k), int(metric), int(wp_form), int(mode)
        p.r, p.eps, p.delta_rel = float(r), float(eps), float(delta_rel)
        p.nbr_out = _ptr(nbr_out)
        p.nbr_w = _ptr(nbr_w)
        P = g.width * g.height
        if out is None:
            dev = caches["nrm"].device
            out = torch.empty((P, 3), dtype=torch.float32, device=dev)
        rc = self._lib.drc_interpolate(self._ctx, ctypes.byref(c), ctypes.byref(g), ctypes.byref(p),
                                       _ptr(out), _stream(stream))
        self._check(rc, "drc_interpolate")
        return out

    def fd_loss64(self, weights64, x, target, flags=0, stream=None):
        """drc_fd_loss64 (test harness): the mean L1 loss in FP64 on the GPU
        for cuda float64 packed weights; returns a cuda float64 scalar."""
        import torch
        N, _, H, W = x.shape
        loss = torch.empty((), dtype=torch.float64, device=x.device)
        rc = self._lib.drc_fd_loss64(self._ctx, _ptr(weights64), _ptr(x), _ptr(target), N, H, W, flags, _ptr(loss),
                                     _stream(stream))
        self._check(rc, "drc_fd_loss64")
        return loss

    def gen_maps(self, scene, pos, nrm, H, W, u=None, out=None, stream=None):
        """drc_gen_maps: maps [n,7,H,W] traced from cache points pos / nrm
        ([n,3] cuda float32) in `scene` (make_scene), with the uniforms u
        [n,H,W,D,2] of the D bounces (None: D = 0)."""
        import torch
        n = int(pos.shape[0])
        D = 0 if u is None else int(u.shape[3])
        if out is None:
            out = torch.empty((n, 7, H, W), dtype=torch.float32, device=pos.device)
        rc = self._lib.drc_gen_maps(self._ctx, ctypes.byref(scene), n, _ptr(pos), _ptr(nrm), int(H), int(W), D,
                                    _ptr(u), _ptr(out), _stream(stream))
        self._check(rc, "drc_gen_maps")
        return out

    def indirect(self, maps, cache_nrm, gnrm, width, height, nbr, nbr_w, u, albedo, emit=None, direct=None,
                 out=None, stream=None):
        """drc_indirect: the indirect term of Eq. 3 by multiple importance
        sampling, plus emit and direct when given.  maps [n,3,H,W] linear
        radiance, cache_nrm [n,3], gnrm [P,3], nbr [P,k] int32, nbr_w [P,k],
        u [P,S,4], albedo / emit / direct [P,3]; all cuda float32."""
        import torch
        c = Caches()
        c.n = int(maps.shape[0])
        c.H, c.W = int(maps.shape[2]), int(maps.shape[3])
        c.maps = _ptr(maps)
        c.nrm = _ptr(cache_nrm)
        g = GBuffer()
        g.width, g.height = int(width), int(height)
        g.nrm = _ptr(gnrm)
        p = IndirectParams()
        p.k = int(nbr.shape[1])
        p.nbr, p.nbr_w = _ptr(nbr), _ptr(nbr_w)
        p.S = int(u.shape[1])
        p.u, p.albedo, p.emit, p.direct = _ptr(u), _ptr(albedo), _ptr(emit), _ptr(direct)
        if out is None:
            out = torch.empty((g.width * g.height, 3), dtype=torch.float32, device=maps.device)
        rc = self._lib.drc_indirect(self._ctx, ctypes.byref(c), ctypes.byref(g), ctypes.byref(p), _ptr(out),
                                    _stream(stream))
        self._check(rc, "drc_indirect")
        return out

    def frame_host(self, maps_host, caches, gbuf_host, k, metric, wp_form, r, rgb_host=None, flags=0, eps=1e-6,
                   delta_rel=1e-3, stream=None):
        """drc_frame_host: denoise the host maps [N,7,H,W] (CPU float32,
        pinned for overlap) and interpolate the G-buffer given as CPU tensors
        gbuf_host["pos"], ["nrm"] ([P,3]) from their payloads; caches: dict of
        CUDA tensors pos / nrm / pix of the N caches.  Returns rgb_host [P,3]
        (a new pinned tensor unless given), valid once `stream` has reached
        the end of the call."""
        import torch
        N, C, H, W = maps_host.shape
        if maps_host.is_cuda or gbuf_host["nrm"].is_cuda:
            raise ValueError("frame_host takes host (CPU) maps and G-buffer")
        c = Caches()
        c.n = int(caches["nrm"].shape[0])
        c.pos = _ptr(caches.get("pos"))
        c.nrm = _ptr(caches.get("nrm"))
        c.pix = _ptr(caches.get("pix"))
        g = GBuffer()
        g.width, g.height = int(gbuf_host["width"]), int(gbuf_host["height"])
        g.pos = ctypes.c_void_p(gbuf_host["pos"].data_ptr()) if gbuf_host.get("pos") is not None else None
        g.nrm = ctypes.c_void_p(gbuf_host["nrm"].data_ptr())
        p = InterpParams()
        p.k, p.metric, p.wp_form, p.mode = int(k), int(metric), int(wp_form), INTERP_IRRADIANCE
        p.r, p.eps, p.delta_rel = float(r), float(eps), float(delta_rel)
        P = g.width * g.height
        if rgb_host is None:
            rgb_host = torch.empty((P, 3), dtype=torch.float32).pin_memory()
        rc = self._lib.drc_frame_host(self._ctx, ctypes.c_void_p(maps_host.data_ptr()), N, H, W, flags,
                                      ctypes.byref(c), ctypes.byref(g), ctypes.byref(p),
                                      ctypes.c_void_p(rgb_host.data_ptr()), _stream(stream))
        self._check(rc, "drc_frame_host")
        return rgb_host

    def backward(self, x, target, flags=BWD_L1_TARGET, want_dinput=False, want_loss=True, stream=None):
        """drc_backward: (loss or None, dweights [n_weights], dinput or None).
        flags: BWD_L1_TARGET (target = ground truth) or BWD_GRAD_OUT (target =
        dL/dout), optionally | F_ENCODE_INPUT | BWD_RECOMPUTE_ENCODER."""
        import torch
        N, C, H, W = x.shape
        dweights = torch.empty(self.n_weights, dtype=torch.float32, device=x.device)
        dinput = torch.empty_like(x) if want_dinput else None
        loss = torch.empty((), dtype=torch.float32, device=x.device) if want_loss else None
        rc = self._lib.drc_backward(self._ctx, _ptr(x), _ptr(target), N, H, W, flags, _ptr(dweights),
                                    _ptr(dinput), _ptr(loss), _stream(stream))
        self._check(rc, "drc_backward")
        return loss, dweights, dinput

    def weight_grad(self, R, Q, qraw=None, dW=None, stream=None):
        """drc_weight_grad: one layer's weight gradient
        dW[m][q][u][v] += sum R[n,i,j,m] Q[n,2i+u-1,2j+v-1,q] from NHWC CUDA
        tensors R [N,Hb,Wb,Mr] and Q [N,2Hb,2Wb,Qc] (both float32 or both
        bfloat16).  Returns dW [Mr, qraw, 3, 3] float32 (a new zeroed tensor
        unless dW is given, which is accumulated into)."""
        import torch
        N, Hb, Wb, Mr = R.shape
        Qc = Q.shape[3]
        if tuple(Q.shape) != (N, 2 * Hb, 2 * Wb, Qc):
            raise ValueError("Q must be [N, 2Hb, 2Wb, Qc]")
        if R.dtype != Q.dtype or R.dtype not in (torch.float32, torch.bfloat16):
            raise ValueError("R and Q must both be float32 or both bfloat16")
        qraw = Qc if qraw is None else int(qraw)
        if dW is None:
            dW = torch.zeros((Mr, qraw, 3, 3), dtype=torch.float32, device=R.device)
        dtype = PREC["bf16"] if R.dtype == torch.bfloat16 else PREC["fp32"]
        rc = self._lib.drc_weight_grad(self._ctx, _ptr(R), _ptr(Q), dtype, N, Hb, Wb, Mr, Qc, qraw, _ptr(dW),
                                       _stream(stream))
        self._check(rc, "drc_weight_grad")
        return dW

    def augment(self, x, codes, out=None, stream=None):
        """drc_augment: the symmetry codes[n] (r + 4 f: column mirror, then r
        counter-clockwise quarter turns) of each square map.  x: cuda float32
        [N, C, S, S]; codes: cuda int32 [N]."""
        import torch
        N, C, H, W = x.shape
        if out is None:
            out = torch.empty_like(x)
        rc = self._lib.drc_augment(self._ctx, _ptr(x), _ptr(out), N, C, H, W, _ptr(codes), _stream(stream))
        self._check(rc, "drc_augment")
        return out

    def adam_step(self, w, grad, m, v, t, lr=6e-5, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        """drc_adam_step: one Adam step t >= 1 on cuda float32 tensors w, m, v
        (updated in place) from grad, all of one size."""
        n = w.numel()
        if not (grad.numel() == m.numel() == v.numel() == n):
            raise ValueError("w, grad, m and v must have one size")
        rc = self._lib.drc_adam_step(self._ctx, _ptr(w), _ptr(grad), _ptr(m), _ptr(v), n, int(t), float(lr),
                                     float(beta1), float(beta2), float(eps), _stream(stream))
        self._check(rc, "drc_adam_step")
        return w

    def status(self, stream=None):
        """Synchronise and return the latched device status code."""
        rc = self._lib.drc_get_status(self._ctx, _stream(stream))
        return rc

    def calibrate(self, x, flags=0, stream=None):
        """FP8: set per-channel activation scales from a representative batch
        x (device [N,7,H,W] float32); synchronises."""
        N, C, H, W = x.shape
        self._check(self._lib.drc_calibrate(self._ctx, _ptr(x), N, H, W, flags, _stream(stream)), "drc_calibrate")

    def autotune(self, N, H, W, cache=None):
        """Time each conv layer's tile candidates for N maps of H x W and keep
        the fastest for later denoise calls (synchronises).  cache: path of
        a JSON-lines tile cache (drc_autotune_cached) -- a hit applies the
        stored choice without timing.  Returns True on a cache hit."""
        if cache is None:
            self._check(self._lib.drc_autotune(self._ctx, int(N), int(H), int(W)), "drc_autotune")
            return False
        hit = ctypes.c_int(0)
        self._check(self._lib.drc_autotune_cached(self._ctx, int(N), int(H), int(W), os.fsencode(cache),
                                                  ctypes.byref(hit)), "drc_autotune_cached")
        return bool(hit.value)

    def save_checkpoint(self, path, adam_m=None, adam_v=None, adam_step=0, stream=None):
        """drc_save_checkpoint: the current weights (and the Adam state, cuda
        float32 tensors of n_weights, when given) to one file."""
        self._check(self._lib.drc_save_checkpoint(self._ctx, os.fsencode(path), _ptr(adam_m) if adam_m is not None
                                                  else None, _ptr(adam_v) if adam_v is not None else None,
                                                  int(adam_step), _stream(stream)), "drc_save_checkpoint")

    def load_checkpoint(self, path, adam_m=None, adam_v=None, stream=None):
        """drc_load_checkpoint: make the file's weights current (and fill the
        Adam state tensors when given); returns the stored Adam step."""
        step = ctypes.c_int(0)
        self._check(self._lib.drc_load_checkpoint(self._ctx, os.fsencode(path), _ptr(adam_m) if adam_m is not None
                                                  else None, _ptr(adam_v) if adam_v is not None else None,
                                                  ctypes.byref(step), _stream(stream)), "drc_load_checkpoint")
        return step.value

    def get_weights(self, out=None, stream=None):
        """drc_get_weights: the current fp32 weights, into `out` (a cuda
        float32 tensor of n_weights) or as a new numpy array."""
        if out is not None:
            self._check(self._lib.drc_get_weights(self._ctx, _ptr(out), 1, _stream(stream)), "drc_get_weights")
            return out
        w = np.empty(self.n_weights, dtype=np.float32)
        self._check(self._lib.drc_get_weights(self._ctx, w.ctypes.data, 0, _stream(stream)), "drc_get_weights")
        return w

    def set_memory_limit(self, nbytes):
        """drc_set_memory_limit: cap the device memory this context allocates
        (0: no cap)."""
        self._check(self._lib.drc_set_memory_limit(self._ctx, int(nbytes)), "drc_set_memory_limit")

    def memory_in_use(self):
        return int(self._lib.drc_memory_in_use(self._ctx))

    def describe_layer(self, layer):
        bn, path = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self._lib.drc_describe_layer(self._ctx, layer, ctypes.byref(bn), ctypes.byref(path)),
                    "drc_describe_layer")
        return bn.value, path.value

    def launch_count(self):
        """Kernel launches this context has issued since it was created."""
        v = ctypes.c_ulonglong(0)
        self._check(self._lib.drc_launch_count(self._ctx, ctypes.byref(v)), "drc_launch_count")
        return int(v.value)

    def set_timing(self, enable):
        """Bracket every following kernel launch with CUDA events (diagnostics)."""
        self._check(self._lib.drc_set_timing(self._ctx, 1 if enable else 0), "drc_set_timing")

    def read_timing(self):
        """{kernel name: (launches, total device ms)} of the timed launches since the last read."""
        cap = 64
        buf = (KernelTime * cap)()
        n = ctypes.c_int(0)
        self._check(self._lib.drc_read_timing(self._ctx, buf, cap, ctypes.byref(n)), "drc_read_timing")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(n.value)}


PLAN_AUTOTUNE = 0x1


class Plan:
    """A drc_plan: progressive passes over several map sizes, one CUDA-graph
    launch per pass, counts read from device memory."""

    def __init__(self, ctx, classes, autotune=False):
        self._ctx = ctx
        self._lib = ctx._lib
        self.classes = [tuple(int(v) for v in c) for c in classes]
        arr = (SizeClass * len(classes))(*[SizeClass(h, w, m) for h, w, m in self.classes])
        self._plan = ctypes.c_void_p()
        rc = self._lib.drc_plan_create(ctx._ctx, arr, len(classes), PLAN_AUTOTUNE if autotune else 0,
                                       ctypes.byref(self._plan))
        ctx._check(rc, "drc_plan_create")

    def launch(self, counts, ins, outs, payloads=None, flags=0, stream=None):
        """counts: device int32 tensor [n_classes]; ins / outs / payloads: one
        device tensor (or None for a payload) per class."""
        n = len(self.classes)
        P = ctypes.c_void_p
        pin = (P * n)(*[t.data_ptr() for t in ins])
        pout = (P * n)(*[t.data_ptr() for t in outs])
        ppay = None if payloads is None else (P * n)(*[0 if t is None else t.data_ptr() for t in payloads])
        rc = self._lib.drc_plan_launch(self._plan, _ptr(counts), pin, pout, ppay, flags, _stream(stream))
        self._ctx._check(rc, "drc_plan_launch")

    def describe(self, k, layer):
        bn, path = ctypes.c_int(0), ctypes.c_int(0)
        rc = self._lib.drc_plan_describe(self._plan, k, layer, ctypes.byref(bn), ctypes.byref(path))
        if rc != OK:
            raise DrcError(rc, "drc_plan_describe")
        return bn.value, path.value

    def close(self):
        if self._plan:
            self._lib.drc_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class DenoiseFunction(torch.autograd.Function):
        """out = network(x; weights) through drc_denoise; the backward is
        drc_backward with the incoming gradient (BWD_GRAD_OUT).  The weights
        tensor must be the values the context holds (set_weights)."""

        @staticmethod
        def forward(ctx_, x, weights, drc_ctx, flags):
            ctx_.drc = drc_ctx
            ctx_.flags = flags
            ctx_.save_for_backward(x)
            return drc_ctx.denoise(x.contiguous(), flags=flags & F_ENCODE_INPUT)

        @staticmethod
        def backward(ctx_, grad_out):
            (x,) = ctx_.saved_tensors
            _, dw, dx = ctx_.drc.backward(x.contiguous(), grad_out.contiguous(),
                                          flags=BWD_GRAD_OUT | (ctx_.flags & F_ENCODE_INPUT),
                                          want_dinput=ctx_.needs_input_grad[0], want_loss=False)
            return dx, dw, None, None

    return DenoiseFunction


def denoise_autograd(drc_ctx, x, weights, flags=0):
    """Differentiable denoise: gradients flow to x and to `weights` (a float32
    CUDA tensor holding the context's packed weights)."""
    return _autograd_function().apply(x, weights, drc_ctx, flags)


class Trainer:
    """The training step of Sec. 4 through the C ABI: augment each pair (one
    code per pair, drc_augment on input and target), the L1 loss and its
    gradient (drc_backward), one Adam step (drc_adam_step) on a device copy
    of the weights, which drc_set_weights then makes current.  The defaults
    are the paper's: lr 6e-5 and PyTorch's Adam constants."""

    def __init__(self, ctx, weights, lr=6e-5, beta1=0.9, beta2=0.999, eps=1e-8, flags=BWD_L1_TARGET):
        import torch
        self.ctx = ctx
        self.w = torch.as_tensor(np.ascontiguousarray(weights, dtype=np.float32)).cuda()
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.t = 0
        self.lr, self.beta1, self.beta2, self.eps, self.flags = lr, beta1, beta2, eps, flags
        ctx.set_weights(self.w)

    def step(self, x, target, codes, stream=None):
        """One step on the pairs (x [N,7,S,S], target [N,3,S,S], cuda float32)
        with the symmetries codes (cuda int32 [N]); returns the loss tensor."""
        xa = self.ctx.augment(x, codes, stream=stream)
        ta = self.ctx.augment(target, codes, stream=stream)
        loss, dw, _ = self.ctx.backward(xa, ta, flags=self.flags, stream=stream)
        self.t += 1
        self.ctx.adam_step(self.w, dw, self.m, self.v, self.t, self.lr, self.beta1, self.beta2, self.eps,
                           stream=stream)
        self.ctx.set_weights(self.w, stream=stream)
        return loss

    def save(self, path, stream=None):
        """Checkpoint of the run: the weights and the Adam state and step."""
        self.ctx.save_checkpoint(path, self.m, self.v, self.t, stream=stream)

    def load(self, path, stream=None):
        """Resume from save(): weights, Adam state and step."""
        self.t = self.ctx.load_checkpoint(path, self.m, self.v, stream=stream)
        self.ctx.get_weights(out=self.w, stream=stream)


def unet_param_count(base=64, levels=3, in_ch=7, out_ch=3):
    """drc_unet_param_count: packed parameters of the paper-form U-Net (0 for
    a shape the forward pass refuses)."""
    return int(load_library().drc_unet_param_count(in_ch, out_ch, base, levels))


def unet_tensor_cores(base, levels, H, W, in_ch=7, out_ch=3):
    """drc_unet_tensor_cores: whether drc_unet_forward runs this shape's 3x3
    layers on the tensor cores (else on the CUDA cores)."""
    return bool(load_library().drc_unet_tensor_cores(in_ch, out_ch, base, levels, H, W))


class UNet:
    """The paper's own network form (a U-Net, Sec. 3.3) through
    drc_unet_forward, on a context's stream and error reporting.  params:
    the packed layout of drc.h (e.g. synth.unet_params); the workspace is
    kept per batch shape."""

    def __init__(self, ctx, params, base=64, levels=3, in_ch=7, out_ch=3):
        import torch
        self.ctx, self.base, self.levels, self.in_ch, self.out_ch = ctx, base, levels, in_ch, out_ch
        n = unet_param_count(base, levels, in_ch, out_ch)
        p = np.ascontiguousarray(params, dtype=np.float32)
        if n == 0 or p.size != n:
            raise ValueError("expected %d U-Net parameters, got %d" % (n, p.size))
        self.params = torch.from_numpy(p).cuda()
        self._ws, self._ws_shape = None, None

    def workspace_bytes(self, N, H, W):
        return int(self.ctx._lib.drc_unet_workspace_bytes(self.in_ch, self.out_ch, self.base, self.levels, N, H, W))

    def forward(self, x, out=None, stream=None):
        """x: cuda float32 [N, in_ch, H, W] -> out [N, out_ch, H, W]."""
        import torch
        N, C, H, W = x.shape
        if out is None:
            out = torch.empty((N, self.out_ch, H, W), dtype=torch.float32, device=x.device)
        if self._ws_shape != (N, H, W):
            nb = max(self.workspace_bytes(N, H, W), 16)
            self._ws = torch.empty(nb, dtype=torch.uint8, device=x.device)
            self._ws_shape = (N, H, W)
        rc = self.ctx._lib.drc_unet_forward(self.ctx._ctx, self.in_ch, self.out_ch, self.base, self.levels,
                                            _ptr(self.params), _ptr(x), _ptr(out), N, H, W, _ptr(self._ws),
                                            self._ws.numel(), _stream(stream))
        self.ctx._check(rc, "drc_unet_forward")
        return out

