"""Shared helpers for the parity tests (no method arithmetic here)."""
import numpy as np

# FP32 bar: max over elements of |gpu - oracle| / max(|oracle|, FLOOR * rms(oracle)).
# A plain fp32 evaluation of these networks already carries an absolute error of
# about 2e-6 rms (measured against fp64), so near-zero outputs are judged against
# a tenth of the tensor's rms rather than their own magnitude.
FP32_TOL = 1e-4
FLOOR = 0.1


def rel_err(g, o, floor=FLOOR):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    if o.size == 0:
        return 0.0
    rms = np.sqrt(np.mean(o * o))
    den = np.maximum(np.abs(o), floor * rms)
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.abs(g - o) / den))


def unet_float32(params, x, base, levels, cin=7, cout=3):
    """The paper-form U-Net evaluated in plain IEEE float32 by PyTorch's CPU
    operators (conv2d, conv_transpose2d, batch_norm, leaky_relu, max_pool2d,
    bilinear interpolate with half-pixel centres, cat): the error any
    correct fp32 evaluation carries, the basis of the U-Net's bar."""
    import torch
    from paper_1910_02480_gb300 import synth
    F = torch.nn.functional
    p = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32))
    layers, off = [], 0
    for kind, ws, nvec in synth.unet_layer_shapes(base, levels, cin, cout):
        n = int(np.prod(ws))
        w = p[off:off + n].reshape(ws)
        off += n
        co = ws[0] if kind in ("conv", "head") else ws[1]
        vec = []
        for _ in range(nvec):
            vec.append(p[off:off + co])
            off += co
        layers.append((kind, w, vec))

    def layer(t, li):
        kind, w, vec = layers[li]
        z = (F.conv2d if kind == "conv" else F.conv_transpose2d)(t, w, vec[0], padding=1)
        if len(vec) == 5:
            z = F.batch_norm(z, vec[3], vec[4], weight=vec[1], bias=vec[2], training=False, eps=1e-5)
        return F.leaky_relu(z, 0.01)

    with torch.no_grad():
        t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
        li, enc = 0, []
        for lvl in range(levels + 1):
            if lvl > 0:
                t = F.max_pool2d(t, 2)
            t = layer(layer(t, li), li + 1)
            li += 2
            enc.append(t)
        d = enc[levels]
        for lvl in range(levels - 1, -1, -1):
            u = F.interpolate(d, scale_factor=2, mode="bilinear", align_corners=False)
            d = layer(layer(torch.cat([u, enc[lvl]], 1), li), li + 1)
            li += 2
        _, w, vec = layers[li]
        y = torch.relu(F.conv2d(d, w[:, :, None, None], vec[0]))
    return y.numpy()


def median_rel(g, o, floor=FLOOR):
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    rms = np.sqrt(np.mean(o * o))
    den = np.maximum(np.abs(o), floor * rms)
    den = np.where(den > 0, den, 1.0)
    return float(np.median(np.abs(g - o) / den))


def relu_margin(weights, x, widths, out_relu=False, exposure=1.0, encode=False):
    """Smallest |pre-activation| / rms(pre-activations of that layer) over
    every ReLU of the network (FP64, from the oracle's layer functions).
    Where a pre-activation lies within the FP32 path's rounding error of 0,
    the ReLU derivative -- and so the gradient -- may rightly differ between
    FP32 and FP64; gradient parity cases use inputs whose margin is larger."""
    import oracle
    from paper_1910_02480_gb300 import synth
    W = synth.unpack_weights(weights, widths)
    e = np.asarray(x, dtype=np.float64).copy()
    if encode:
        e[:, :3] = np.log1p(exposure * e[:, :3])
    S = len(widths)
    margins, enc = [], [e]
    for s in range(S):
        w, b = W[s]
        z = oracle.conv3x3s2(enc[-1], w, b)
        margins.append(np.min(np.abs(z)) / np.sqrt(np.mean(z * z)))
        enc.append(np.maximum(z, 0.0))
    t = enc[S]
    for s in range(S - 1, -1, -1):
        w, b = W[2 * S - 1 - s]
        z = oracle.convT3x3s2(t, w, b)
        if s > 0 or out_relu:
            margins.append(np.min(np.abs(z)) / np.sqrt(np.mean(z * z)))
        t = np.maximum(z, 0.0) + enc[s] if s > 0 else z
    return float(min(margins))


def kink_free_biases(weights, x, widths, out_relu=False, window=0.05):
    """Weights whose biases are shifted, layer by layer in forward order, so
    that zero sits in the middle of the widest gap among each channel's
    pre-activations within `window` x rms of zero: no pre-activation is then
    near a ReLU kink (large batches have too many pre-activations for a
    random input to avoid them).  Returns a new packed float32 vector."""
    import oracle
    from paper_1910_02480_gb300 import synth
    w = np.array(weights, dtype=np.float32, copy=True)
    S = len(widths)
    layers = synth.layer_shapes(widths)
    offs, off = [], 0
    for _, ws, bn in layers:
        n = int(np.prod(ws))
        offs.append((off, n, bn))
        off += n + bn

    def shift(z, li):
        o, n, bn = offs[li]
        b = w[o + n:o + n + bn]
        zt = np.moveaxis(z, 1, 0).reshape(z.shape[1], -1)
        rms = np.sqrt(np.mean(zt * zt))
        for c in range(zt.shape[0]):
            v = np.sort(zt[c][np.abs(zt[c]) < window * rms])
            if v.size < 2:
                continue
            gaps = np.diff(v)
            k = int(np.argmax(gaps))
            b[c] -= np.float32(0.5 * (v[k] + v[k + 1]))
        w[o + n:o + n + bn] = b

    W = synth.unpack_weights(w, widths)
    e = [np.asarray(x, dtype=np.float64)]
    for s in range(S):
        shift(oracle.conv3x3s2(e[-1], *W[s]), s)
        W = synth.unpack_weights(w, widths)
        e.append(np.maximum(oracle.conv3x3s2(e[-1], *W[s]), 0.0))
    t = e[S]
    for s in range(S - 1, -1, -1):
        li = 2 * S - 1 - s
        if s > 0 or out_relu:
            shift(oracle.convT3x3s2(t, *W[li]), li)
            W = synth.unpack_weights(w, widths)
        z = oracle.convT3x3s2(t, *W[li])
        t = np.maximum(z, 0.0) + e[s] if s > 0 else z
    return w
