"""The algorithmic counts behind bench.py's rooflines, pinned on the CPU: a
convolution of an all-ones map with all-ones weights (the oracle's layers)
counts, at each output, exactly its in-map taps times the input channels, so
the sum over outputs is the layer's valid multiply-adds."""
import os
import sys

import numpy as np
import pytest

import oracle

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _ones_macs(layer, cin, cout, H, W):
    x = np.ones((1, cin, H, W))
    if layer == "conv":
        return oracle.conv3x3s2(x, np.ones((cout, cin, 3, 3))).sum()
    if layer == "convT":
        return oracle.convT3x3s2(x, np.ones((cin, cout, 3, 3))).sum()
    if layer == "conv1":
        return oracle.conv3x3s1(x, np.ones((cout, cin, 3, 3))).sum()
    raise ValueError(layer)


@pytest.mark.parametrize("widths,H,W", [([64, 128, 256], 32, 32), ([32, 64, 128], 16, 16), ([8, 16], 8, 12)])
def test_benchmark_network_macs(widths, H, W):
    got = bench.valid_macs_per_layer(widths, H, W)
    prev, h, w = 7, H, W
    for s, c in enumerate(widths, 1):
        assert got["conv e%d" % s] == _ones_macs("conv", prev, c, h, w)
        prev, h, w = c, h // 2, w // 2
    S = len(widths)
    for s in range(S, 0, -1):
        ci, co = widths[s - 1], 3 if s == 1 else widths[s - 2]
        name = "head" if s == 1 else "convT d%d" % s
        assert got[name] == _ones_macs("convT", ci, co, H >> s, W >> s)


@pytest.mark.parametrize("base,levels,H,W", [(64, 3, 32, 32), (4, 2, 16, 8), (2, 1, 6, 4)])
def test_unet_flops(base, levels, H, W):
    macs = 0.0
    for lvl in range(levels + 1):
        h, w, c = H >> lvl, W >> lvl, base << lvl
        ci = 7 if lvl == 0 else base << (lvl - 1)
        macs += _ones_macs("conv1", ci, c, h, w) + _ones_macs("conv1", c, c, h, w)
    for lvl in range(levels - 1, -1, -1):
        h, w, c = H >> lvl, W >> lvl, base << lvl
        macs += _ones_macs("conv1", 3 * c, c, h, w) + _ones_macs("conv1", c, c, h, w)
    macs += H * W * base * 3  # the 1x1 head
    assert bench.unet_flops_per_map(base, levels, H, W) == pytest.approx(2.0 * macs, rel=1e-12)
