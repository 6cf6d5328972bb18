"""drc_backward's FP32 gradient against FP64 central finite differences
taken on the GPU (drc_fd_loss64, a test harness: the network's mean L1 loss
in FP64), on the training configuration's 8-map slice (7 x 64 x 64 maps,
widths 64/128/256/512; Sec. 4).  The harness itself is pinned to the FP64
oracle's loss.

The loss is piecewise linear in any one weight (ReLU network, L1 loss), so a
central difference is exact unless a ReLU or the L1 sign switches within the
step; the biases are shifted off the ReLU kinks and the targets sit away
from the outputs, and each probe is taken with two steps, h and h/2, which
must agree (else a switch lies within the step and the probe is skipped)."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth
from parity import kink_free_biases

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def drc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_02480_gb300 import build
    build.build()
    import paper_1910_02480_gb300 as m
    return m


def _pairs(N, H, W, seed):
    g = synth.gbuffer(N, 1, seed=seed)
    x, clean = synth.hemisphere_maps(g["pos"], g["nrm"], H=H, W=W, seed=seed + 1, noise="poisson", spp=4)
    return np.ascontiguousarray(x, np.float32), np.ascontiguousarray(clean, np.float32)


def test_fp64_harness_matches_oracle_loss(drc):
    widths, N, H, W = [16, 32], 2, 16, 16
    w = synth.he_weights(widths, seed=0, bias=True)
    x, _ = _pairs(N, H, W, seed=3)
    out = oracle.forward(w, x, widths)
    target = (out + np.random.default_rng(4).uniform(0.01, 0.1, size=out.shape)).astype(np.float32)
    loss_o, _, _ = oracle.l1_backward(w, x, target, widths)
    ctx = drc.Context(widths, w, precision="fp32")
    loss = ctx.fd_loss64(torch.from_numpy(w.astype(np.float64)).cuda(), torch.from_numpy(x).cuda(),
                         torch.from_numpy(target).cuda())
    np.testing.assert_allclose(float(loss.item()), float(loss_o), rtol=1e-12)
    # with the log encode of the input
    xl = np.ascontiguousarray(np.expm1(np.clip(x, 0.0, None)), np.float32)
    loss_oe, _, _ = oracle.l1_backward(w, xl, target, widths, flags=oracle.F_ENCODE_INPUT)
    loss_e = ctx.fd_loss64(torch.from_numpy(w.astype(np.float64)).cuda(), torch.from_numpy(xl).cuda(),
                           torch.from_numpy(target).cuda(), flags=drc.F_ENCODE_INPUT)
    np.testing.assert_allclose(float(loss_e.item()), float(loss_oe), rtol=1e-12)


def test_fp32_gradient_against_gpu_finite_differences(drc):
    widths, N, H, W = [64, 128, 256, 512], 8, 64, 64
    x, _ = _pairs(N, H, W, seed=5)
    w = kink_free_biases(synth.he_weights(widths, seed=0), x, widths)
    out = oracle.forward(w, x, widths)
    target = (out + np.random.default_rng(6).choice([-1.0, 1.0], size=out.shape)
              * np.random.default_rng(7).uniform(0.01, 0.1, size=out.shape)).astype(np.float32)
    ctx = drc.Context(widths, w, precision="fp32")
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(target).cuda()
    _, dw, _ = ctx.backward(xd, td)
    g = dw.cpu().numpy().astype(np.float64)
    w64 = torch.from_numpy(w.astype(np.float64)).cuda()
    # probes: per layer, the weight and the bias element of largest gradient
    # and two more of at least a tenth of the layer's largest
    rng = np.random.default_rng(8)
    probes, off = [], 0
    for _, ws, bn in synth.layer_shapes(widths):
        for lo, n in ((off, int(np.prod(ws))), (off + int(np.prod(ws)), bn)):
            seg = np.abs(g[lo:lo + n])
            probes.append(lo + int(np.argmax(seg)))
            big = np.nonzero(seg >= 0.1 * seg.max())[0]
            probes.extend((lo + rng.choice(big, size=min(2, big.size), replace=False)).tolist())
        off += int(np.prod(ws)) + bn

    def loss_at(i, d):
        w64[i] += d
        v = float(ctx.fd_loss64(w64, xd, td).item())
        w64[i] -= d
        return v

    fd, got, used = [], [], 0
    for i in probes:
        h = 1e-6 * max(1.0, abs(float(w[i])))
        d1 = (loss_at(i, h) - loss_at(i, -h)) / (2 * h)
        d2 = (loss_at(i, h / 2) - loss_at(i, -h / 2)) / h
        if abs(d1 - d2) > 1e-4 * max(abs(d1), 1e-9):
            continue  # a switch lies within the step
        fd.append(d1)
        got.append(g[i])
        used += 1
    fd, got = np.array(fd), np.array(got)
    print("finite differences: %d of %d probes; max rel %.3e, normwise %.3e"
          % (used, len(probes), np.max(np.abs(got - fd) / np.abs(fd)), np.linalg.norm(got - fd) / np.linalg.norm(fd)))
    assert used >= 0.9 * len(probes)
    assert np.linalg.norm(got - fd) / np.linalg.norm(fd) <= 1e-4
    assert np.max(np.abs(got - fd) / np.abs(fd)) <= 1e-3
