"""The training-loop pieces of Sec. 4 through the C ABI against the FP64
oracle: map augmentation (drc_augment), the Adam step (drc_adam_step) and a
whole training step (augment, drc_backward, Adam, drc_set_weights)."""
import numpy as np
import pytest

import oracle
from paper_1910_02480_gb300 import synth
from parity import rel_err

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))  # the values the fp32 kernel is handed


@pytest.fixture(scope="module")
def drc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_02480_gb300 import build
    build.build()
    import paper_1910_02480_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(drc):
    return drc.Context([16], synth.he_weights([16]), precision="fp32")


@pytest.mark.parametrize("N,C,S", [(37, 7, 32), (5, 3, 64), (3, 7, 16), (2, 3, 80), (1, 1, 1)])
def test_augment_is_exact(drc, ctx, N, C, S):
    """A permutation of each plane: bit-exact.  64 x 64 is the largest plane
    staged in shared memory; 80 x 80 takes the direct gather.  Codes past 7
    use their low three bits."""
    rng = np.random.default_rng(N * 100 + S)
    x = rng.standard_normal((N, C, S, S)).astype(np.float32)
    codes = rng.integers(0, 16, size=N).astype(np.int32)
    codes[:min(N, 8)] = np.arange(min(N, 8))
    y = ctx.augment(torch.from_numpy(x).cuda(), torch.from_numpy(codes).cuda())
    torch.cuda.synchronize()
    ref = oracle.augment(x, codes & 7)
    np.testing.assert_array_equal(y.cpu().numpy(), ref.astype(np.float32))


def test_augment_argument_errors(drc, ctx):
    x = torch.zeros((2, 3, 8, 8), device="cuda")
    codes = torch.zeros(2, dtype=torch.int32, device="cuda")
    ctx.augment(x[:0], codes[:0])  # N = 0: nothing
    with pytest.raises(drc.DrcError):
        ctx.augment(torch.zeros((2, 3, 8, 4), device="cuda"), codes)
    with pytest.raises(drc.DrcError):
        ctx.augment(x, codes, out=x)  # in place
    with pytest.raises(drc.DrcError):
        ctx.augment(x, codes.cpu())


@pytest.mark.parametrize("n,offset,t", [(100003, 0, 1), (100003, 0, 7), (4099, 4, 3), (3, 0, 1)])
def test_adam_step_matches_oracle(drc, ctx, n, offset, t):
    """Four parameters per thread, the last n % 4 one at a time; offset 4
    starts the arrays one 16-byte step into their buffers.  fp32 against
    fp64: v to 1e-6 relative, m to its roundings' bound, w to two of its ulps
    plus its update's rounding and m's error carried through."""
    rng = np.random.default_rng(n + t)
    w = rng.standard_normal(n).astype(np.float32)
    g = (rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 1, size=n)).astype(np.float32)
    m = (rng.standard_normal(n) * 1e-2).astype(np.float32)
    v = (rng.uniform(0, 1e-3, size=n)).astype(np.float32)
    dev = [torch.from_numpy(np.concatenate([np.zeros(offset, np.float32), a])).cuda() for a in (w, g, m, v)]
    wd, gd, md, vd = [d[offset:] for d in dev]
    lr, b1, b2, eps = 6e-5, 0.9, 0.999, 1e-8
    ctx.adam_step(wd, gd, md, vd, t, lr, b1, b2, eps)
    torch.cuda.synchronize()
    wo, mo, vo = oracle.adam_step(w, g, m, v, t, F32(lr), F32(b1), F32(b2), F32(eps))
    # m's two terms may cancel: its three fp32 roundings are bounded by the
    # terms' sizes, not by the result's
    err_m = 3e-7 * (F32(b1) * np.abs(m) + (1 - F32(b1)) * np.abs(g))
    assert np.all(np.abs(md.cpu().numpy() - mo) <= err_m)
    np.testing.assert_allclose(vd.cpu().numpy(), vo, rtol=1e-6, atol=1e-30)
    # w: two of its ulps, the update's own rounding, and m's error carried
    # through the update lr m / (1 - b1^t) / (sqrt(v^) + eps)
    wg = wd.cpu().numpy().astype(np.float64)
    ulp = np.spacing(np.abs(wo).astype(np.float32)).astype(np.float64)
    vhat = vo / (1 - F32(b2) ** t)
    carried = F32(lr) * err_m / (1 - F32(b1) ** t) / (np.sqrt(vhat) + F32(eps))
    assert np.all(np.abs(wg - wo) <= 2 * ulp + 1e-5 * np.abs(wo - w) + carried)
    assert dev[0][:offset].abs().sum().item() == 0  # nothing written before the view


def test_adam_argument_errors(drc, ctx):
    z = torch.zeros(8, device="cuda")
    for kw in ({"t": 0}, {"t": 1, "lr": 0.0}, {"t": 1, "beta1": 1.0}, {"t": 1, "eps": -1.0}):
        with pytest.raises(drc.DrcError):
            ctx.adam_step(z, z.clone(), z.clone(), z.clone(), **kw)
    with pytest.raises(drc.DrcError):
        ctx.adam_step(z, z.cpu(), z.clone(), z.clone(), 1)
    with pytest.raises(drc.DrcError):  # device pointers are 16-byte aligned
        ctx.adam_step(z[1:], z.clone()[1:], z.clone()[1:], z.clone()[1:], 1)


def test_training_steps_match_oracle(drc):
    """Two steps at the paper's settings (widths 64/128/256, Adam lr 6e-5) on
    4 augmented 32 x 32 pairs, against the oracle's augment, L1 backward and
    Adam.

    Step 1 runs on biases shifted so that no pre-activation of its augmented
    input lies near a ReLU kink.  It moves each weight by about lr sign(g), so
    an element is matched where its oracle gradient is well clear of the fp32
    gradient's rounding (|g| > 1e-3 rms).  Step 2 runs on new weights and new
    codes, where a pre-activation may sit on a kink and rightly flip a few
    gradients, so its step vector is compared normwise.  Both steps check the
    loss and Adam's bound on the step size, and the context then denoises
    with the trained weights."""
    from parity import kink_free_biases, relu_margin
    widths = [64, 128, 256]
    rng = np.random.default_rng(5)
    g = synth.gbuffer(4, 1, seed=8)
    x, _ = synth.hemisphere_maps(g["pos"], g["nrm"], H=32, W=32, seed=9)
    x = np.ascontiguousarray(x, dtype=np.float32)
    target = (x[:, :3] + rng.uniform(0.01, 0.1, size=(4, 3, 32, 32))).astype(np.float32)
    steps = ((1, np.array([0, 5, 2, 7], dtype=np.int32)), (2, np.array([3, 1, 6, 4], dtype=np.int32)))
    xa1 = oracle.augment(x, steps[0][1]).astype(np.float32)
    w0 = kink_free_biases(synth.he_weights(widths, seed=0, bias=True), xa1, widths)
    assert relu_margin(w0, xa1, widths) > 1e-5
    ctx = drc.Context(widths, w0, precision="fp32")
    trainer = drc.Trainer(ctx, w0)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(target).cuda()
    wo = w0.astype(np.float64)
    mo = np.zeros_like(wo)
    vo = np.zeros_like(wo)
    lr = trainer.lr
    for t, cd in steps:
        w_prev = trainer.w.cpu().numpy().astype(np.float64)
        loss = trainer.step(xd, td, torch.from_numpy(cd).cuda())
        torch.cuda.synchronize()
        assert ctx.status() == drc.OK
        lo, dwo, _ = oracle.l1_backward(wo.astype(np.float32), oracle.augment(x, cd).astype(np.float32),
                                        oracle.augment(target, cd).astype(np.float32), widths)
        assert abs(loss.item() - lo) <= 1e-5 * abs(lo)
        w_before = wo
        wo, mo, vo = oracle.adam_step(wo, dwo, mo, vo, t, F32(lr), F32(0.9), F32(0.999), F32(1e-8))
        step_gpu = trainer.w.cpu().numpy().astype(np.float64) - w_prev
        step_orc = wo - w_before
        assert np.max(np.abs(step_gpu)) <= 3.17 * lr  # Adam's bound (1 - b1) / sqrt(1 - b2)
        if t == 1:
            sure = np.abs(dwo) > 1e-3 * np.sqrt(np.mean(dwo * dwo))
            assert sure.mean() > 0.8  # with 4 pairs some layers' gradients are small
            assert np.max(np.abs(step_gpu[sure] - step_orc[sure])) <= 2e-3 * lr
        else:
            assert np.linalg.norm(step_gpu - step_orc) <= 2e-2 * np.linalg.norm(step_orc)
    out = ctx.denoise(xd)
    torch.cuda.synchronize()
    ref = oracle.forward(trainer.w.cpu().numpy(), x, widths)
    assert rel_err(out.cpu().numpy(), ref) <= 1e-4
    ctx.close()
