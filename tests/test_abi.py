"""The C-ABI library builds, loads and exports every entry point declared in
include/drc.h; host-side argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(drc_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1910_02480_gb300 import build
    build.build()
    import paper_1910_02480_gb300 as drc
    return drc.load_library()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"drc_create", "drc_denoise", "drc_interpolate", "drc_backward"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), "libdrc.so does not export " + n


def test_weight_count_matches_layer_table(lib):
    import paper_1910_02480_gb300 as drc
    from paper_1910_02480_gb300 import synth
    for widths in ([32, 64, 128], [64, 128, 256], [64, 128, 256, 512], [16]):
        assert drc.weight_count(widths) == synth.weight_count(widths)
    assert drc.weight_count([32, 64, 128]) == 187523
    assert drc.weight_count([64, 128, 256]) == 743683
    assert drc.weight_count([64, 128, 256, 512]) == 3103747


@pytest.mark.parametrize("field,value", [("in_channels", 6), ("out_channels", 4), ("num_stages", 0),
                                         ("num_stages", 7), ("precision", 9), ("exposure", 0.0),
                                         ("wait_timeout_ms", -1)])
def test_create_rejects_bad_config_without_touching_the_gpu(lib, field, value):
    import paper_1910_02480_gb300 as drc
    cfg = drc.make_config([32, 64, 128])
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert lib.drc_create(ctypes.byref(cfg), None, 0, ctypes.byref(h)) == drc.ERR_INVALID_ARG
    assert not h.value


def test_create_rejects_bad_widths(lib):
    import paper_1910_02480_gb300 as drc
    for widths in ([8, 64], [24, 64], [32, 2048]):
        cfg = drc.make_config(widths)
        h = ctypes.c_void_p()
        assert lib.drc_create(ctypes.byref(cfg), None, 0, ctypes.byref(h)) == drc.ERR_INVALID_ARG


def test_null_context_is_rejected(lib):
    import paper_1910_02480_gb300 as drc
    assert lib.drc_denoise(None, None, None, None, 1, 32, 32, 0, None) == drc.ERR_INVALID_ARG
    assert lib.drc_get_status(None, None) == drc.ERR_INVALID_ARG
    assert lib.drc_destroy(None) == drc.ERR_INVALID_ARG


def test_unet_size_queries(lib):
    """The paper-form U-Net's two host-side size queries: the parameter count
    agrees with the oracle's and with the seeded generator's layout; the
    workspace holds the folded weights plus every activation and grows with
    the batch; shapes the forward pass refuses give 0."""
    import numpy as np

    import oracle
    import paper_1910_02480_gb300 as drc
    from paper_1910_02480_gb300 import synth
    for base, levels in ((64, 3), (8, 2), (20, 1), (4, 4)):
        n = drc.unet_param_count(base, levels)
        assert n == oracle.unet_param_count(base, levels) == synth.unet_params(base, levels).size
    ws = lambda N, H, W, base=64, levels=3: int(lib.drc_unet_workspace_bytes(7, 3, base, levels, N, H, W))
    # per level l (c = 64 2^l channels): enc_a, enc; the pooled input (c / 2,
    # l > 0); up (2c), dec_a, dec (l < 3)
    floats_per_map = sum((64 << l) * ((32 >> l) ** 2) * (2 + (0.5 if l > 0 else 0) + (4 if l < 3 else 0))
                         for l in range(4))
    assert ws(256, 32, 32) - ws(0, 32, 32) >= 256 * floats_per_map * 4
    # folded weights: the parameters less the batch-normalisation statistics
    bn_floats = sum(4 * (w[0] if k == "conv" else w[1]) for k, w, nvec in synth.unet_layer_shapes(64, 3) if nvec == 5)
    assert ws(0, 32, 32) >= 4 * (drc.unet_param_count(64, 3) - bn_floats)
    assert ws(512, 32, 32) > ws(256, 32, 32) > ws(1, 32, 32)
    assert ws(1, 24, 32) > 0  # 24 is a multiple of 2^3
    assert ws(1, 20, 32) == 0 and ws(-1, 32, 32) == 0 and ws(1, 32, 32, levels=0) == 0
    assert drc.unet_param_count(64, 7) == 0 and drc.unet_param_count(0, 3) == 0
    assert np.isfinite(ws(1, 32, 32))
    # which shapes take the tensor cores: whole K blocks of channels and maps
    # whose rows tile 128-row boxes at every level
    tc = lambda cin, base, levels, H, W: int(lib.drc_unet_tensor_cores(cin, 3, base, levels, H, W))
    assert tc(7, 64, 3, 32, 32) == 1 and tc(32, 64, 3, 32, 32) == 1 and tc(7, 32, 2, 32, 16) == 1
    assert tc(7, 8, 2, 16, 16) == 0    # 8 channels: not a whole K block
    assert tc(16, 64, 3, 32, 32) == 0  # 16 input channels: neither tap boxes nor whole K blocks
    assert tc(7, 64, 3, 24, 32) == 0   # 3 x 4 bottleneck: 12-row maps do not tile 128 rows
    assert tc(7, 64, 1, 256, 256) == 0  # rows wider than a tile
    assert tc(7, 64, 3, 20, 32) == 0 and tc(7, 64, 0, 32, 32) == 0  # shapes the forward pass refuses
