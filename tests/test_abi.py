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
