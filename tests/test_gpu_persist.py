"""The context's persistence and memory control through the C ABI:
checkpoints of the weights and Adam state (drc_save_checkpoint /
drc_load_checkpoint, Sec. 4's saved and reloaded network), the autotune tile
cache (drc_autotune_cached) and the device memory cap (drc_set_memory_limit),
whose refusals are the out-of-memory path tested without exhausting the GPU."""
import json

import numpy as np
import pytest

from paper_1910_02480_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

WIDTHS = [32, 64, 128]


@pytest.fixture(scope="module")
def drc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_02480_gb300 import build
    build.build()
    import paper_1910_02480_gb300 as m
    return m


def _maps(N, seed, H=32, W=32):
    g = synth.gbuffer(N, 1, seed=seed)
    x, _ = synth.hemisphere_maps(g["pos"], g["nrm"], H=H, W=W, seed=seed + 1)
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def test_checkpoint_round_trip(drc, tmp_path):
    """Weights, Adam moments and step come back bit for bit, and the loaded
    context denoises exactly like the one that saved them."""
    w1 = synth.he_weights(WIDTHS, seed=1, bias=True)
    w2 = synth.he_weights(WIDTHS, seed=2, bias=True)
    a = drc.Context(WIDTHS, w1, precision="fp32")
    b = drc.Context(WIDTHS, w2, precision="fp32")
    n = a.n_weights
    g = torch.Generator(device="cuda").manual_seed(3)
    m = torch.randn(n, device="cuda", generator=g)
    v = torch.rand(n, device="cuda", generator=g)
    path = str(tmp_path / "run.ckpt")
    a.save_checkpoint(path, m, v, 7)
    with open(path, "rb") as f:
        head = json.loads(f.readline())
    assert head["format"] == "drc-checkpoint" and head["n_floats"] == n and head["adam"] == 1
    assert head["widths"] == WIDTHS and head["adam_step"] == 7
    with open(path, "rb") as f:
        assert len(f.read()) == len(open(path, "rb").readline()) + 3 * 4 * n  # header line, then 3 arrays
    m2, v2 = torch.zeros_like(m), torch.zeros_like(v)
    assert b.load_checkpoint(path, m2, v2) == 7
    assert np.array_equal(b.get_weights(), w1.astype(np.float32))
    assert torch.equal(m2, m) and torch.equal(v2, v)
    x = _maps(6, 20)
    ya, yb = a.denoise(x), b.denoise(x)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
    # weights alone: no Adam state in the file, and asking for it is an error
    path2 = str(tmp_path / "weights.ckpt")
    b.save_checkpoint(path2)
    a.load_checkpoint(path2)
    with pytest.raises(drc.DrcError, match="no optimizer state"):
        a.load_checkpoint(path2, m2, v2)
    with pytest.raises(drc.DrcError, match="both"):
        a.save_checkpoint(path2, m, None)
    a.close()
    b.close()


def test_checkpoint_rejects_other_networks_and_damage(drc, tmp_path):
    w = synth.he_weights(WIDTHS, seed=4)
    a = drc.Context(WIDTHS, w, precision="fp32")
    path = str(tmp_path / "a.ckpt")
    a.save_checkpoint(path)
    other = drc.Context([32, 64], synth.he_weights([32, 64], seed=4), precision="fp32")
    with pytest.raises(drc.DrcError, match="another network") as ei:
        other.load_checkpoint(path)
    assert ei.value.args[0].startswith("DRC_ERR_INVALID_ARG")
    # the same network in another precision loads (the weights are fp32 masters)
    bf = drc.Context(WIDTHS, synth.he_weights(WIDTHS, seed=5), precision="bf16")
    bf.load_checkpoint(path)
    assert np.array_equal(bf.get_weights(), w.astype(np.float32))
    raw = bytearray(open(path, "rb").read())
    raw[-5] ^= 0x40  # one flipped bit in the payload
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(drc.DrcError, match="checksum"):
        a.load_checkpoint(bad)
    open(bad, "wb").write(bytes(raw[:-4]))  # truncated
    with pytest.raises(drc.DrcError, match="payload"):
        a.load_checkpoint(bad)
    with pytest.raises(drc.DrcError):
        a.load_checkpoint(str(tmp_path / "missing.ckpt"))
    # the failed loads left the weights as they were
    assert np.array_equal(a.get_weights(), w.astype(np.float32))
    for c in (a, other, bf):
        c.close()


def test_trainer_resumes_from_checkpoint(drc, tmp_path):
    """A run saved after three steps resumes in a new context with exactly the
    saved weights, Adam moments and step count, and then takes the steps the
    uninterrupted run takes (equal up to the order of the gradient's float
    atomics: the losses to 1e-5, the weights to 1 % of a learning-rate step
    normwise)."""
    widths = [32, 64]
    w0 = synth.he_weights(widths, seed=6, bias=True)
    rng = np.random.default_rng(7)
    x = _maps(8, 30)
    t = (x[:, :3] + torch.from_numpy(rng.uniform(0.01, 0.1, (8, 3, 32, 32)).astype(np.float32)).cuda()).contiguous()
    codes = [torch.from_numpy(rng.integers(0, 8, 8).astype(np.int32)).cuda() for _ in range(5)]
    ca = drc.Context(widths, w0, precision="fp32")
    ta = drc.Trainer(ca, w0)
    for k in range(3):
        ta.step(x, t, codes[k])
    path = str(tmp_path / "train.ckpt")
    ta.save(path)
    saved = (ta.w.clone(), ta.m.clone(), ta.v.clone())
    straight = [ta.step(x, t, codes[k]).item() for k in (3, 4)]
    cb = drc.Context(widths, synth.he_weights(widths, seed=9), precision="fp32")
    tb = drc.Trainer(cb, synth.he_weights(widths, seed=9))
    tb.load(path)
    torch.cuda.synchronize()
    assert tb.t == 3
    assert torch.equal(tb.w, saved[0]) and torch.equal(tb.m, saved[1]) and torch.equal(tb.v, saved[2])
    assert np.array_equal(cb.get_weights(), saved[0].cpu().numpy())
    resumed = [tb.step(x, t, codes[k]).item() for k in (3, 4)]
    torch.cuda.synchronize()
    np.testing.assert_allclose(resumed, straight, rtol=1e-5)
    dw = (ta.w - tb.w).double().norm().item()
    assert dw <= 0.01 * ta.lr * np.sqrt(ta.w.numel())
    ca.close()
    cb.close()


def test_autotune_cache_hit_applies_the_stored_tiles(drc, tmp_path):
    w = synth.he_weights(WIDTHS, seed=10)
    cache = str(tmp_path / "tiles.jsonl")
    with open(cache, "w") as f:  # lines that are not entries for this case are skipped
        f.write("not json\n")
        f.write(json.dumps({"format": "drc-autotune", "version": 1, "device": "another GPU", "sms": 1, "cc": 1,
                            "precision": "fp32", "shape": [64, 32, 32], "tile_n": [16] * 6, "a_path": [-1] * 6})
                + "\n")
    a = drc.Context(WIDTHS, w, precision="fp32")
    assert a.autotune(64, 32, 32, cache=cache) is False  # a miss: timed, then appended
    lines = open(cache).read().splitlines()
    assert len(lines) == 3
    entry = json.loads(lines[-1])
    tiles = [a.describe_layer(li) for li in range(2 * len(WIDTHS))]
    assert entry["tile_n"] == [t[0] for t in tiles] and entry["a_path"] == [t[1] for t in tiles]
    assert entry["shape"] == [64, 32, 32] and entry["widths"] == WIDTHS
    b = drc.Context(WIDTHS, w, precision="fp32")
    assert b.autotune(64, 32, 32, cache=cache) is True  # a hit: applied without timing
    assert [b.describe_layer(li) for li in range(2 * len(WIDTHS))] == tiles
    assert len(open(cache).read().splitlines()) == 3
    x = _maps(64, 40)
    ya, yb = a.denoise(x), b.denoise(x)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
    # another batch shape is another entry
    assert b.autotune(16, 32, 32, cache=cache) is False
    assert len(open(cache).read().splitlines()) == 4
    # a later entry whose tiles do not fit the layers is skipped: the earlier
    # valid entry still answers
    bad = dict(entry, tile_n=[48] * len(entry["tile_n"]))
    c = drc.Context(WIDTHS, w, precision="fp32")
    with open(cache, "a") as f:
        f.write(json.dumps(bad) + "\n")
    assert c.autotune(64, 32, 32, cache=cache) is True
    assert [c.describe_layer(li) for li in range(2 * len(WIDTHS))] == tiles
    for ctx in (a, b, c):
        ctx.close()


def test_memory_cap_refuses_growth_and_recovers(drc):
    """A request past the cap returns DRC_ERR_OOM before allocating and leaves
    the context working; raising the cap lets the same call through."""
    w = synth.he_weights(WIDTHS, seed=11)
    ref = drc.Context(WIDTHS, w, precision="fp32")
    c = drc.Context(WIDTHS, w, precision="fp32")
    base = c.memory_in_use()
    assert base > 0
    x = _maps(512, 50)
    c.set_memory_limit(base + (1 << 20))  # 1 MB of headroom: the 512-map workspace needs far more
    with pytest.raises(drc.DrcError, match="memory limit") as ei:
        c.denoise(x)
    assert ei.value.args[0].startswith("DRC_ERR_OOM")
    assert c.memory_in_use() == base  # nothing was allocated
    assert c.status() == drc.OK
    small = _maps(2, 60)
    y_small = c.denoise(small)  # a batch that fits under the cap still runs
    c.set_memory_limit(0)
    y = c.denoise(x)
    torch.cuda.synchronize()
    assert c.memory_in_use() > base + (1 << 20)
    assert torch.equal(y, ref.denoise(x)) and torch.equal(y_small, ref.denoise(small))
    # the cap covers the interpolation scratch too
    gb = synth.gbuffer(256, 256, seed=70)
    cg = synth.cache_grid(gb, 16, 16)
    cg["payload"] = np.ones((len(cg["pos"]), 3), dtype=np.float32)
    cu = lambda d: {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) else v
                    for k, v in d.items()}
    c.set_memory_limit(c.memory_in_use() + 1024)
    with pytest.raises(drc.DrcError, match="memory limit"):
        c.interpolate(cu(cg), cu(gb), 8, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, 0.2)
    c.set_memory_limit(0)
    out = c.interpolate(cu(cg), cu(gb), 8, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, 0.2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), 1.0, rtol=3e-6)
    ref.close()
    c.close()
