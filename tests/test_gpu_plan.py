"""drc_plan_*: progressive passes with uneven counts and mixed map sizes
(Sec. 3.2 progressive refinement) in one graph launch per pass, checked
against drc_denoise of each class and against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth
from parity import FP32_TOL, rel_err

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


def _maps(N, H, W, seed):
    g = synth.gbuffer(max(N, 1), 1, seed=seed + 10)
    maps, _ = synth.hemisphere_maps(g["pos"][:N], g["nrm"][:N], H=H, W=W, seed=seed)
    return np.ascontiguousarray(maps, dtype=np.float32)


WIDTHS = [32, 64, 128]
CLASSES = [(32, 32, 300), (16, 16, 200)]


def _run_pass(plan, counts, xs, flags=0, want_payload=True, sentinel=7.0):
    outs = [torch.full((m, 3, h, w), sentinel, device="cuda") for (h, w, m) in plan.classes]
    pays = [torch.full((m, 3), sentinel, device="cuda") for (h, w, m) in plan.classes] if want_payload else None
    ins = [torch.from_numpy(x).cuda() if x.shape[0] else torch.empty((1, 7, h, w), device="cuda")
           for x, (h, w, _) in zip(xs, plan.classes)]
    plan.launch(torch.tensor(counts, dtype=torch.int32, device="cuda"), ins, outs, pays, flags=flags)
    torch.cuda.synchronize()
    return outs, pays


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_plan_equals_denoise_per_class(drc, precision):
    w = synth.he_weights(WIDTHS, seed=0, bias=True)
    ctx = drc.Context(WIDTHS, w, precision=precision)
    plan = drc.Plan(ctx, CLASSES)
    for it, counts in enumerate([(137, 45), (300, 0), (1, 200)]):
        xs = [_maps(n, h, h, seed=20 + 3 * it + k) for k, (n, (h, _, _)) in enumerate(zip(counts, CLASSES))]
        outs, pays = _run_pass(plan, counts, xs)
        assert ctx.status() == drc.OK
        for k, n in enumerate(counts):
            if n == 0:
                assert torch.all(outs[k] == 7.0)
                continue
            ref, rpay = ctx.denoise(torch.from_numpy(xs[k]).cuda(), want_payload=True)
            torch.cuda.synchronize()
            assert torch.equal(outs[k][:n], ref), (precision, it, k)
            # payloads are summed with atomics: equal up to the order of the adds
            assert rel_err(pays[k][:n].cpu().numpy(), rpay.cpu().numpy()) <= 1e-6
            assert torch.all(outs[k][n:] == 7.0) and torch.all(pays[k][n:] == 7.0)
    plan.close()


def test_plan_fp32_matches_oracle_with_flags(drc):
    w = synth.he_weights(WIDTHS, seed=1, bias=True)
    s = 0.75
    ctx = drc.Context(WIDTHS, w, precision="fp32", exposure=s)
    plan = drc.Plan(ctx, CLASSES)
    counts = (9, 6)
    xs = []
    for k, (n, (h, _, _)) in enumerate(zip(counts, CLASSES)):
        x = _maps(n, h, h, seed=40 + k)
        x[:, :3] = np.expm1(np.clip(x[:, :3], 0.0, None))  # linear radiance in, encoded by the plan
        xs.append(x)
    outs, pays = _run_pass(plan, counts, xs, flags=drc.F_ENCODE_INPUT | drc.F_DECODE_OUTPUT)
    for k, n in enumerate(counts):
        ref = oracle.forward(w, xs[k], WIDTHS, exposure=s, flags=3)
        assert rel_err(outs[k][:n].cpu().numpy(), ref) <= FP32_TOL
        assert rel_err(pays[k][:n].cpu().numpy(), oracle.payload(ref)) <= FP32_TOL


def test_plan_autotuned_bf16(drc):
    w = synth.he_weights(WIDTHS, seed=0)
    ctx = drc.Context(WIDTHS, w, precision="bf16")
    plan = drc.Plan(ctx, CLASSES, autotune=True)
    for k in range(len(CLASSES)):
        for li in range(2 * len(WIDTHS)):
            bn, _ = plan.describe(k, li)
            if li < 2 * len(WIDTHS) - 1:
                assert bn in (16, 32, 64, 128, 256) and bn > 0
            else:
                assert bn == 0  # the head
    counts = (57, 33)
    xs = [_maps(n, h, h, seed=60 + k) for k, (n, (h, _, _)) in enumerate(zip(counts, CLASSES))]
    outs, _ = _run_pass(plan, counts, xs, want_payload=False)
    for k, n in enumerate(counts):
        ref = oracle.forward(w, xs[k], WIDTHS)
        g = outs[k][:n].cpu().numpy()
        rms = np.sqrt(np.mean(ref * ref))
        assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-2
        assert np.max(np.abs(g - ref)) / rms < 0.1


def test_plan_autotuned_fp32_parity(drc):
    w = synth.he_weights(WIDTHS, seed=2, bias=True)
    ctx = drc.Context(WIDTHS, w, precision="fp32")
    plan = drc.Plan(ctx, CLASSES, autotune=True)
    counts = (21, 17)
    xs = [_maps(n, h, h, seed=80 + k) for k, (n, (h, _, _)) in enumerate(zip(counts, CLASSES))]
    outs, _ = _run_pass(plan, counts, xs, want_payload=False)
    for k, n in enumerate(counts):
        assert rel_err(outs[k][:n].cpu().numpy(), oracle.forward(w, xs[k], WIDTHS)) <= FP32_TOL


def test_plan_count_out_of_range_is_clamped_and_latched(drc):
    w = synth.he_weights(WIDTHS, seed=0)
    ctx = drc.Context(WIDTHS, w, precision="fp32")
    plan = drc.Plan(ctx, [(16, 16, 8)])
    x = _maps(8, 16, 16, seed=5)
    xin = torch.from_numpy(np.concatenate([x, x[:4]])).cuda()  # room for 12 maps
    out = torch.zeros((12, 3, 16, 16), device="cuda")
    plan.launch(torch.tensor([12], dtype=torch.int32, device="cuda"), [xin], [out])
    assert ctx.status() == drc.ERR_INVALID_ARG
    ref = ctx.denoise(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert torch.equal(out[:8], ref)
    assert torch.all(out[8:] == 0)
    assert ctx.status() == drc.OK


def test_plan_follows_new_weights(drc):
    w0 = synth.he_weights(WIDTHS, seed=0)
    w1 = synth.he_weights(WIDTHS, seed=9, bias=True)
    ctx = drc.Context(WIDTHS, w0, precision="fp32")
    plan = drc.Plan(ctx, [(32, 32, 16)])
    x = _maps(5, 32, 32, seed=7)
    ctx.set_weights(w1)
    outs, _ = _run_pass(plan, (5,), [x], want_payload=False)
    assert rel_err(outs[0][:5].cpu().numpy(), oracle.forward(w1, x, WIDTHS)) <= FP32_TOL


def test_plan_argument_errors(drc):
    w = synth.he_weights(WIDTHS, seed=0)
    ctx = drc.Context(WIDTHS, w, precision="fp32")
    with pytest.raises(drc.DrcError) as e:
        drc.Plan(ctx, [(12, 12, 4)])  # not a multiple of 2^3
    assert e.value.code == drc.ERR_INVALID_ARG
    with pytest.raises(drc.DrcError) as e:
        drc.Plan(ctx, [(16, 16, 0)])
    assert e.value.code == drc.ERR_INVALID_ARG
    plan = drc.Plan(ctx, [(16, 16, 4)])
    with pytest.raises(drc.DrcError) as e:  # host counts
        plan.launch(torch.tensor([1], dtype=torch.int32), [torch.zeros((4, 7, 16, 16), device="cuda")],
                    [torch.zeros((4, 3, 16, 16), device="cuda")])
    assert e.value.code == drc.ERR_INVALID_ARG
