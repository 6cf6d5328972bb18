#!/usr/bin/env python3
"""Throughput of the Deep Radiance Caching hot path on GB300.

One step = the whole hot path over one batch of synthetic input: denoise
4096 cache-point maps (7 x 32 x 32, encoder widths 64/128/256, FP32 path =
split-tf32 tensor-core products) with the per-map irradiance payload, then
interpolate a 1920 x 1080 G-buffer from the 64 x 64 caches (k = 16 nearest
by first-hit position, inverse-distance x normal-dot weights).  Metric:
cache-point maps denoised per second (whole job).

Flags: --gpus N --steps K --warmup W [--impl ours|reference]
       [--precision fp32|bf16] [--no-cpu-baseline]
Under torchrun every rank runs its own batch (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_MAPS, MAP_H, MAP_W = 4096, 32, 32
WIDTHS = [64, 128, 256]
IMG_W, IMG_H, GRID = 1920, 1080, 64
K_NN = 16
METRIC_NAME = "cache-point maps denoised/sec on 1 GB300"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) of the conv kernel's launches in one denoise call of
# the 4096-map workload: ncu dram__bytes_read.sum + dram__bytes_write.sum of a
# 2304-map denoise, scaled by 4096/2304; None where not taken, and reset to
# None whenever the kernel changes after the counters were taken.
TRAFFIC = {"fp32": 1611e6, "bf16": None}
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense ratio (tf32 : bf16)


def set_workload(maps, frame):
    """Smaller workloads for profiling runs; the defaults are the benchmark's."""
    global N_MAPS, IMG_W, IMG_H, GRID
    N_MAPS = int(maps)
    IMG_W, IMG_H = (int(v) for v in frame.lower().split("x"))
    GRID = int(round(N_MAPS ** 0.5))
    if GRID * GRID != N_MAPS:
        raise SystemExit("--maps must be a square number (a square cache grid)")


def valid_macs_per_layer(widths, H, W, cin=7, cout=3):
    """{layer name: multiply-accumulates per map}, counting in-bounds taps only.
    Names are the library's kernel labels (conv e1.., convT dS..d2, head)."""
    def conv_taps(n_in):  # per output index: taps u with 0 <= 2i+u-1 < n_in
        n_out = n_in // 2
        return sum(sum(1 for u in range(3) if 0 <= 2 * i + u - 1 < n_in) for i in range(n_out))

    def convT_taps(n_in):  # per input index: taps landing inside 0..2n_in-1
        return sum(sum(1 for u in range(3) if 0 <= 2 * i + u - 1 < 2 * n_in) for i in range(n_in))

    out = {}
    prev, h, w = cin, H, W
    for s, c in enumerate(widths, 1):
        out["conv e%d" % s] = prev * c * conv_taps(h) * conv_taps(w)
        prev, h, w = c, h // 2, w // 2
    S = len(widths)
    for s in range(S, 0, -1):
        ci = widths[s - 1]
        co = cout if s == 1 else widths[s - 2]
        hs, ws = H >> s, W >> s
        out["head" if s == 1 else "convT d%d" % s] = ci * co * convT_taps(hs) * convT_taps(ws)
    return out


def valid_macs_per_map(widths, H, W, cin=7, cout=3):
    return sum(valid_macs_per_layer(widths, H, W, cin, cout).values())


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def measure_precision(drc, torch, dev, prec, fp32_denoise_ms, autotune=True, steps=20, tile_cache=None):
    """Denoise-only throughput of another precision at the benchmark's size,
    its speedup over the FP32 path, and its error against the FP64 oracle on
    a sample of high-dynamic-range maps (lobes log-uniform in 1e-3..1e3)."""
    import oracle
    from paper_1910_02480_gb300 import synth
    w = synth.he_weights(WIDTHS, seed=0)
    g = synth.gbuffer(N_MAPS, 1, seed=12)
    x, _ = synth.hemisphere_maps(g["pos"], g["nrm"], H=MAP_H, W=MAP_W, seed=3)
    ctx = drc.Context(WIDTHS, w, precision=prec)
    lobe = synth.lobes(seed=1, log_uniform=True)
    cal_note = None
    if prec == "fp8":  # per-channel scales from a separate batch of the same field
        gc = synth.gbuffer(256, 1, seed=14)
        xc, _ = synth.hemisphere_maps(gc["pos"], gc["nrm"], H=MAP_H, W=MAP_W, lobe=lobe, seed=7)
        ctx.calibrate(torch.from_numpy(np.ascontiguousarray(xc, dtype=np.float32)).to(dev))
        cal_note = "256 maps of the HDR field (not the error sample), drc_calibrate"
    if autotune:
        ctx.autotune(N_MAPS, MAP_H, MAP_W, cache=tile_cache)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)
    out = torch.empty((N_MAPS, 3, MAP_H, MAP_W), device=dev)
    pay = torch.empty((N_MAPS, 3), device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(3):
        ctx.denoise(xd, out=out, payload=pay)
    ms = []
    torch.cuda.synchronize()
    ctx.read_timing()
    ctx.set_timing(True)
    for i in range(steps):
        flush.fill_(float(i))
        a, b = _events(torch)
        a.record()
        ctx.denoise(xd, out=out, payload=pay)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    ctx.set_timing(False)
    kt = ctx.read_timing()
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after %s timing" % prec)
    den = float(np.mean(ms))
    # the tensor-core conv kernel's roofline at this precision: valid-tap
    # FLOPs over its launches' device time; peaks: the measured bf16 burst,
    # and for e4m3 that times the nominal fp8 : bf16 ratio (4.5 / 2.25)
    layer_macs = valid_macs_per_layer(WIDTHS, MAP_H, MAP_W)
    conv_names = [n for n in layer_macs if n.startswith("conv")]
    conv_flops = 2.0 * sum(layer_macs[n] for n in conv_names) * N_MAPS
    conv_ms = sum(kt[n][1] for n in conv_names if n in kt) / steps
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else None
    bf16_peak = peaks["bf16_tflops"] if peaks else 1900.0
    peak = bf16_peak * (2.0 if prec == "fp8" else 1.0)
    achieved = conv_flops / (conv_ms * 1e-3) / 1e12 if conv_ms > 0 else None
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None, "kernel_ms_per_call": conv_ms,
            "kernel_ms_per_layer": {n: kt[n][1] / steps for n in conv_names if n in kt},
            "peak_source": ("of measured: bf16 burst %.1f TF/s" % bf16_peak if prec == "bf16" else
                            "of measured: bf16 burst %.1f TF/s x nominal e4m3/bf16 2" % bf16_peak)
            if peaks else "of fallback"}
    # error sample: 16 maps of the HDR field, log1p-encoded radiance in
    xs, _ = synth.hemisphere_maps(g["pos"][:16], g["nrm"][:16], H=MAP_H, W=MAP_W, lobe=lobe, seed=5)
    xs = np.ascontiguousarray(xs, dtype=np.float32)
    o, pa = ctx.denoise(torch.from_numpy(xs).to(dev), want_payload=True)
    torch.cuda.synchronize()
    ref = oracle.forward(w, xs, WIDTHS)
    refp = oracle.payload(np.expm1(ref))
    err = {}
    for name, gv, rv in (("out", o.cpu().numpy(), ref), ("payload", pa.cpu().numpy(), refp)):
        rms = float(np.sqrt(np.mean(rv * rv)))
        den_ = np.maximum(np.abs(rv), 0.1 * rms)
        err[name] = {"max_rel": float(np.max(np.abs(gv - rv) / den_)),
                     "normwise": float(np.linalg.norm(gv - rv) / np.linalg.norm(rv))}
    ctx.close()
    return {"denoise_ms": den, "denoise_maps_per_s": N_MAPS / (den * 1e-3), "roofline": roof,
            "speedup_vs_fp32_denoise": fp32_denoise_ms / den if fp32_denoise_ms else None, "error_vs_oracle": err,
            "error_sample": "16 maps 7x32x32, lobes log-uniform 1e-3..1e3, FP64 oracle",
            "calibration": cal_note}


def measure_uneven(drc, torch, dev, prec="bf16", reps=3):
    """Eight progressive passes with cache counts drawn in [200, 6000] and maps
    16x16 or 32x32 with probability 1/2 (widths 32/64/128): one plan launch
    per pass (autotuned tiles) against two drc_denoise calls per pass."""
    from paper_1910_02480_gb300 import synth
    widths = [32, 64, 128]
    w = synth.he_weights(widths, seed=0)
    counts, sizes = synth.pass_counts(seed=4)
    per = [(int(np.sum(sz == 32)), int(np.sum(sz == 16))) for sz in sizes]
    mx = int(max(counts))
    g = synth.gbuffer(mx, 1, seed=13)
    xs = {}
    for h in (32, 16):
        x, _ = synth.hemisphere_maps(g["pos"], g["nrm"], H=h, W=h, seed=6)
        xs[h] = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)
    outs = {h: torch.empty((mx, 3, h, h), device=dev) for h in (32, 16)}
    pays = {h: torch.empty((mx, 3), device=dev) for h in (32, 16)}
    ctx = drc.Context(widths, w, precision=prec)
    t0 = time.time()
    plan = drc.Plan(ctx, [(32, 32, mx), (16, 16, mx)], autotune=True)
    tune_s = time.time() - t0
    dcounts = [torch.tensor(pc, dtype=torch.int32, device=dev) for pc in per]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_plan():
        for dc in dcounts:
            plan.launch(dc, [xs[32], xs[16]], [outs[32], outs[16]], [pays[32], pays[16]])

    def run_calls():
        for n32, n16 in per:
            ctx.denoise(xs[32][:n32], out=outs[32][:n32], payload=pays[32][:n32])
            ctx.denoise(xs[16][:n16], out=outs[16][:n16], payload=pays[16][:n16])

    res = {}
    for name, fn in (("plan", run_plan), ("denoise_calls", run_calls)):
        fn()
        torch.cuda.synchronize()
        ms = []
        for i in range(reps):
            flush.fill_(float(i))
            a, b = _events(torch)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        res[name] = float(np.min(ms))
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after uneven batching")
    total = int(np.sum(counts))
    tiles = {"32x32": [plan.describe(0, li)[0] for li in range(2 * len(widths) - 1)],
             "16x16": [plan.describe(1, li)[0] for li in range(2 * len(widths) - 1)]}
    plan.close()
    ctx.close()
    return {"passes": len(counts), "maps": total, "counts": [int(c) for c in counts],
            "precision": prec, "widths": widths,
            "plan_ms": res["plan"], "plan_maps_per_s": total / (res["plan"] * 1e-3),
            "denoise_calls_ms": res["denoise_calls"],
            "denoise_calls_maps_per_s": total / (res["denoise_calls"] * 1e-3),
            "autotuned_tile_n": tiles, "autotune_s": tune_s}


def measure_training(drc, torch, dev, prec="bf16", batch=256, steps=10, recompute=True):
    """One training step = drc_backward on a batch of noisy / clean pairs of
    7 x 64 x 64 maps (clean = the analytic lobe field, noisy = Poisson(4)/4
    per texel, L1 on log radiance), widths 64/128/256/512: forward, loss and
    the whole reverse pass (weight, bias and input-side gradients).  With
    recompute the encoder's activations are checkpointed (the decoder
    overwrites them and the encoder runs again before its backward), as the
    training configuration specifies; without, every activation is kept."""
    from paper_1910_02480_gb300 import synth
    widths = [64, 128, 256, 512]
    H = W = 64
    w = synth.he_weights(widths, seed=0)
    g = synth.gbuffer(batch, 1, seed=15)
    x, clean = synth.hemisphere_maps(g["pos"], g["nrm"], H=H, W=W, seed=5, noise="poisson", spp=4)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)
    td = torch.from_numpy(np.ascontiguousarray(clean, dtype=np.float32)).to(dev)
    ctx = drc.Context(widths, w, precision=prec)
    flags = drc.BWD_L1_TARGET | (drc.BWD_RECOMPUTE_ENCODER if recompute else 0)
    for _ in range(3):
        ctx.backward(xd, td, flags=flags)
    torch.cuda.synchronize()
    ctx.read_timing()
    ctx.set_timing(True)
    a, b = _events(torch)
    a.record()
    for _ in range(steps):
        loss, _, _ = ctx.backward(xd, td, flags=flags)
    b.record()
    torch.cuda.synchronize()
    ctx.set_timing(False)
    kt = ctx.read_timing()
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after training steps")
    ms = a.elapsed_time(b) / steps
    macs = sum(valid_macs_per_layer(widths, H, W).values())
    flops_step = 2.0 * macs * batch * 3  # forward + data gradients + weight gradients (recompute not counted)
    by = {}
    for n, (cnt, t) in kt.items():
        key = n.split()[0] if n.split()[0] in ("conv", "convT", "dgrad", "wgrad", "bgrad") else n
        by[key] = by.get(key, 0.0) + t / steps
    ctx.close()
    return {"workload": "%d noisy/clean pairs 7x%dx%d, widths %s, L1 on log radiance, %s, %s" % (
                batch, H, W, "/".join(map(str, widths)), prec,
                "encoder activations checkpointed (recomputed)" if recompute else "all activations kept"),
            "ms_per_step": ms, "maps_per_s": batch / (ms * 1e-3), "loss": float(loss.item()),
            "approx_flops_per_step": flops_step, "achieved_tflops": flops_step / (ms * 1e-3) / 1e12,
            "kernel_ms_per_step": {k: round(v, 4) for k, v in sorted(by.items(), key=lambda kv: -kv[1])}}


def measure_training_paper(drc, torch, dev, batch=32, pool=512, steps=40):
    """The training loop at the paper's settings (Sec. 4): Adam at lr 6e-5 on
    mini-batches of 32 noisy / clean pairs of 7 x 32 x 32 maps, widths
    64/128/256 (base width 64, three downsizing steps), FP32.  Each step
    augments its pairs by one of the eight square symmetries each (seeded
    codes, an input of the step), takes the L1 loss and its gradient, and
    applies an Adam step whose weights the context then takes from device
    memory (drc_set_weights, no host round trip).  Steps cycle through a
    pool of 512 synthetic pairs."""
    from paper_1910_02480_gb300 import synth
    widths = [64, 128, 256]
    H = W = 32
    w = synth.he_weights(widths, seed=0)
    g = synth.gbuffer(pool, 1, seed=16)
    x, clean = synth.hemisphere_maps(g["pos"], g["nrm"], H=H, W=W, seed=6, noise="poisson", spp=4)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)
    td = torch.from_numpy(np.ascontiguousarray(clean, dtype=np.float32)).to(dev)
    codes = torch.from_numpy(np.random.default_rng(17).integers(0, 8, size=(steps + 3, batch)).astype(np.int32)).to(dev)
    ctx = drc.Context(widths, w, precision="fp32")
    tr = drc.Trainer(ctx, w)
    nb = pool // batch

    def step(k):
        b0 = (k % nb) * batch
        return tr.step(xd[b0:b0 + batch], td[b0:b0 + batch], codes[k])

    first = [float(step(k).item()) for k in range(3)]
    torch.cuda.synchronize()
    ctx.read_timing()
    ctx.set_timing(True)
    a, b = _events(torch)
    a.record()
    for k in range(3, 3 + steps):
        loss = step(k)
    b.record()
    torch.cuda.synchronize()
    ctx.set_timing(False)
    kt = ctx.read_timing()
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after training steps")
    ms = a.elapsed_time(b) / steps
    by = {}
    for n, (cnt, t) in kt.items():
        key = n.split()[0] if n.split()[0] in ("conv", "convT", "dgrad", "wgrad", "bgrad") else n
        by[key] = by.get(key, 0.0) + t / steps
    ctx.close()
    return {"workload": "Adam lr 6e-5, batches of %d augmented noisy/clean pairs 7x%dx%d, widths %s, L1 on log "
                        "radiance, fp32" % (batch, H, W, "/".join(map(str, widths))),
            "ms_per_step": ms, "pairs_per_s": batch / (ms * 1e-3), "loss_first_step": first[0],
            "loss_last_step": float(loss.item()), "steps": steps,
            "kernel_ms_per_step": {k: round(v, 4) for k, v in sorted(by.items(), key=lambda kv: -kv[1])}}


def measure_mapgen_indirect(drc, torch, dev, steps=10, S=8, D=3):
    """The steps around the denoiser at the benchmark's sizes: tracing the
    4096 caches' 7 x 32 x 32 input maps in the analytic room (D bounces,
    drc_gen_maps), and the indirect term of Eq. 3 at 1920 x 1080 from the
    k = 16 nearest caches' maps by multiple importance sampling with S
    samples per pixel (drc_indirect, emission and direct term composited).
    Both are bound by HBM: the map tracer reads its uniforms (n H W D 8 B)
    and writes the maps (n 7 H W 4 B); the estimator reads u (P S 16 B),
    the neighbour lists and weights (P k 8 B), normal, albedo, emission and
    direct light (P 48 B) and writes the image (P 12 B), besides gathering
    map texels from L2."""
    from paper_1910_02480_gb300 import synth
    g = synth.gbuffer(IMG_W, IMG_H, seed=2)
    c = synth.cache_grid(g, GRID, GRID)
    n, P, k = GRID * GRID, IMG_W * IMG_H, K_NN
    rng = np.random.default_rng(21)
    pos = np.float32(0.02 + 0.96 * c["pos"].astype(np.float64))
    alb = np.float32([[0.7, 0.2, 0.2], [0.2, 0.7, 0.2], [0.6, 0.6, 0.6], [0.6, 0.6, 0.5], [0.5, 0.5, 0.5],
                      [0.8, 0.8, 0.8]])
    scene = drc.make_scene(alb, np.full((6, 3), 0.05, np.float32), [0.3, 0.7, 0.35, 0.65, 8.0, 7.5, 6.0],
                           [[0.3, 0.3, 0.25, 0.15, 0.9, 0.8, 0.3], [0.7, 0.6, 0.3, 0.2, 0.3, 0.5, 0.9]])
    ctx = drc.Context(WIDTHS, synth.he_weights(WIDTHS, seed=0), precision="fp32")
    pd = torch.from_numpy(pos).to(dev)
    nd = torch.from_numpy(c["nrm"]).to(dev)
    ud = torch.from_numpy(rng.uniform(size=(n, MAP_H, MAP_W, D, 2)).astype(np.float32)).to(dev)
    maps = torch.empty((n, 7, MAP_H, MAP_W), device=dev)
    gd = {"width": IMG_W, "height": IMG_H, "pos": torch.from_numpy(g["pos"]).to(dev),
          "nrm": torch.from_numpy(g["nrm"]).to(dev)}
    cd = {"pos": torch.from_numpy(c["pos"]).to(dev), "nrm": nd, "pix": torch.from_numpy(c["pix"]).to(dev),
          "payload": torch.zeros((n, 3), device=dev)}
    nbr = torch.empty((P, k), dtype=torch.int32, device=dev)
    nw = torch.empty((P, k), dtype=torch.float32, device=dev)
    ctx.interpolate(cd, gd, k, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE,
                    synth.world_radius(n), nbr_out=nbr, nbr_w=nw)
    lin = torch.rand((n, 3, MAP_H, MAP_W), device=dev) * 2.0
    uu = torch.rand((P, S, 4), device=dev)
    albd = torch.rand((P, 3), device=dev) * 0.7 + 0.2
    emit = torch.zeros((P, 3), device=dev)
    direct = torch.rand((P, 3), device=dev)
    out = torch.empty((P, 3), device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ms = []
        for i in range(steps):
            flush.fill_(float(i))
            a, b = _events(torch)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.mean(ms))

    gen_ms = timed(lambda: ctx.gen_maps(scene, pd, nd, MAP_H, MAP_W, u=ud, out=maps))
    ind_ms = timed(lambda: ctx.indirect(lin, nd, gd["nrm"], IMG_W, IMG_H, nbr, nw, uu, albd, emit=emit,
                                        direct=direct, out=out))
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after map generation / indirect")
    peak = json.load(open(PEAKS_FILE))["hbm_gbs"] if os.path.exists(PEAKS_FILE) else 6800.0
    gen_bytes = n * MAP_H * MAP_W * (D * 8 + 7 * 4)
    ind_bytes = P * (S * 16 + k * 8 + 48 + 12)
    ctx.close()
    return {"gen_maps": {"workload": "%d caches, 7x%dx%d maps, %d bounces, room of 6 walls + ceiling light + 2 "
                                     "spheres" % (n, MAP_H, MAP_W, D),
                         "ms": gen_ms, "maps_per_s": n / (gen_ms * 1e-3),
                         "roofline": {"bound": "hbm", "achieved": gen_bytes / (gen_ms * 1e-3) / 1e9, "peak": peak,
                                      "unit": "GB/s", "frac": gen_bytes / (gen_ms * 1e-3) / 1e9 / peak,
                                      "algorithmic_bytes": gen_bytes}},
            "indirect": {"workload": "%dx%d pixels, k=%d, S=%d samples (MIS env/BRDF), emission + direct "
                                     "composited" % (IMG_W, IMG_H, k, S),
                         "ms": ind_ms, "pixels_per_s": P / (ind_ms * 1e-3),
                         "roofline": {"bound": "hbm", "achieved": ind_bytes / (ind_ms * 1e-3) / 1e9, "peak": peak,
                                      "unit": "GB/s", "frac": ind_bytes / (ind_ms * 1e-3) / 1e9 / peak,
                                      "algorithmic_bytes": ind_bytes}}}


def measure_progressive(drc, torch, dev, spacing0=64, passes=4, k=8, S=4, D=3):
    """Progressive refinement (Sec. 3.2) through every GPU step of the
    method, per pass on a 1920 x 1080 G-buffer: the pass's new image-plane
    sample points (drc_pass_points, grid spacing halving from 64 pixels),
    their 7 x 32 x 32 input maps traced in the analytic room (drc_gen_maps,
    D bounces), denoised by the benchmark network (log encode in, linear
    radiance out), the interpolation over every cache so far in the image
    plane (r = the pass's spacing) giving each pixel's k caches and weights,
    and the indirect term by multiple importance sampling (S samples)
    composited with a direct term (drc_indirect).  Times each pass on the
    device; the point lists are uploaded before the timed region."""
    from paper_1910_02480_gb300 import synth
    g = synth.gbuffer(IMG_W, IMG_H, seed=2)
    P = IMG_W * IMG_H
    pos_img = torch.from_numpy(np.float32(0.02 + 0.96 * g["pos"].astype(np.float64))).to(dev)
    nrm_img = torch.from_numpy(g["nrm"]).to(dev)
    gd = {"width": IMG_W, "height": IMG_H, "pos": pos_img, "nrm": nrm_img}
    alb = np.float32([[0.7, 0.2, 0.2], [0.2, 0.7, 0.2], [0.6, 0.6, 0.6], [0.6, 0.6, 0.5], [0.5, 0.5, 0.5],
                      [0.8, 0.8, 0.8]])
    scene = drc.make_scene(alb, np.full((6, 3), 0.05, np.float32), [0.3, 0.7, 0.35, 0.65, 8.0, 7.5, 6.0])
    ctx = drc.Context(WIDTHS, synth.he_weights(WIDTHS, seed=0), precision="fp32")
    pts = [torch.from_numpy(drc.pass_points(IMG_W, IMG_H, spacing0, t)).to(dev) for t in range(passes)]
    total = sum(int(p_.shape[0]) for p_ in pts)
    u_gen = torch.rand((total, MAP_H, MAP_W, D, 2), device=dev)
    u_ind = torch.rand((P, S, 4), device=dev)
    albd = torch.rand((P, 3), device=dev) * 0.7 + 0.2
    direct = torch.rand((P, 3), device=dev)
    maps7 = torch.empty((total, 7, MAP_H, MAP_W), device=dev)
    lin = torch.empty((total, 3, MAP_H, MAP_W), device=dev)
    pay = torch.zeros((total, 3), device=dev)  # the blend's payloads are not used: the MIS reads the maps
    nbr = torch.empty((P, k), dtype=torch.int32, device=dev)
    nw = torch.empty((P, k), dtype=torch.float32, device=dev)
    img = torch.empty((P, 3), device=dev)
    pix_all = torch.cat(pts).contiguous()
    idx_all = (pix_all[:, 1].long() * IMG_W + pix_all[:, 0].long())
    cpos_all = pos_img[idx_all].contiguous()
    cnrm_all = nrm_img[idx_all].contiguous()

    # per pass, 16-byte aligned copies of the new caches' points (a slice of an
    # [n, 3] array is not)
    cpos_new = [cpos_all[a0:a1].clone() for a0, a1 in
                [(sum(int(q.shape[0]) for q in pts[:t]), sum(int(q.shape[0]) for q in pts[:t + 1]))
                 for t in range(passes)]]
    cnrm_new = [cnrm_all[a0:a1].clone() for a0, a1 in
                [(sum(int(q.shape[0]) for q in pts[:t]), sum(int(q.shape[0]) for q in pts[:t + 1]))
                 for t in range(passes)]]

    def run_pass(t, n0, n1):
        ctx.gen_maps(scene, cpos_new[t], cnrm_new[t], MAP_H, MAP_W, u=u_gen[n0:n1], out=maps7[n0:n1])
        ctx.denoise(maps7[n0:n1], out=lin[n0:n1], flags=drc.F_ENCODE_INPUT | drc.F_DECODE_OUTPUT)
        cd = {"pos": cpos_all[:n1], "nrm": cnrm_all[:n1], "pix": pix_all[:n1], "payload": pay[:n1]}
        ctx.interpolate(cd, gd, k, drc.METRIC_IMAGE, drc.WP_INVERSE, drc.INTERP_IRRADIANCE,
                        float(spacing0 >> t), nbr_out=nbr, nbr_w=nw)
        ctx.indirect(lin[:n1], cnrm_all[:n1], nrm_img, IMG_W, IMG_H, nbr, nw, u_ind, albd, direct=direct, out=img)

    bounds, n0 = [], 0
    for p_ in pts:
        bounds.append((n0, n0 + int(p_.shape[0])))
        n0 += int(p_.shape[0])
    for t, (a0, a1) in enumerate(bounds):  # warm-up of every pass shape
        run_pass(t, a0, a1)
    torch.cuda.synchronize()
    per = []
    for t, (a0, a1) in enumerate(bounds):
        ev = _events(torch)
        ev[0].record()
        run_pass(t, a0, a1)
        ev[1].record()
        torch.cuda.synchronize()
        per.append(ev[0].elapsed_time(ev[1]))
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after the progressive passes")
    ctx.close()
    return {"workload": "%dx%d, grid spacing %d halving over %d passes, 7x%dx%d maps (%d bounces), k=%d IMAGE "
                        "metric, S=%d MIS samples, direct term composited" % (IMG_W, IMG_H, spacing0, passes,
                                                                             MAP_H, MAP_W, D, k, S),
            "new_caches_per_pass": [b - a for a, b in bounds], "caches_total": total,
            "ms_per_pass": [round(v, 4) for v in per], "ms_total": float(sum(per))}


def unet_flops_per_map(base=64, levels=3, H=32, W=32, cin=7, cout=3):
    """Valid multiply-adds x 2 of the paper-form U-Net on one H x W map: a
    stride-1 3x3 layer with zero padding meets (3H - 2)(3W - 2) in-map taps
    per channel pair; the 1x1 head H W."""
    flops = 0.0
    for lvl in range(levels + 1):
        h, w, c = H >> lvl, W >> lvl, base << lvl
        ci = cin if lvl == 0 else base << (lvl - 1)
        flops += 2.0 * (3 * h - 2) * (3 * w - 2) * (ci * c + c * c)
    for lvl in range(levels - 1, -1, -1):
        h, w, c = H >> lvl, W >> lvl, base << lvl
        flops += 2.0 * (3 * h - 2) * (3 * w - 2) * (3 * c * c + c * c)
    return flops + 2.0 * H * W * base * cout


def unet_layer_flops(base=64, levels=3, H=32, W=32, cin=7):
    """Valid FLOPs per map of each 3x3 layer of the paper-form U-Net, keyed by
    the name the library traces its launch under ("unet conv i", i in
    execution order: two per encoder level, two per decoder level)."""
    out, i = {}, 0
    for lvl in range(levels + 1):
        h, w, c = H >> lvl, W >> lvl, base << lvl
        ci = cin if lvl == 0 else base << (lvl - 1)
        for a, b in ((ci, c), (c, c)):
            out["unet conv %d" % i] = 2.0 * (3 * h - 2) * (3 * w - 2) * a * b
            i += 1
    for lvl in range(levels - 1, -1, -1):
        h, w, c = H >> lvl, W >> lvl, base << lvl
        for a, b in ((3 * c, c), (c, c)):
            out["unet conv %d" % i] = 2.0 * (3 * h - 2) * (3 * w - 2) * a * b
            i += 1
    return out


def measure_unet(drc, torch, dev, N=4096, steps=5, warmup=3):
    """The paper's own network form (Sec. 3.3: a U-Net, base 64, three
    downsizing steps, 7.8 M parameters) in FP32 on 4096 synthetic 7 x 32 x 32
    maps: its 3x3 layers on the tensor cores (split-tf32 implicit GEMMs of the
    conv kernel family).  One step is the whole forward call: BN folding and
    weight packing, input staging, 14 convolutions, pooling, upsampling, the
    head.  Activations (about 12 GB) are far larger than L2."""
    from paper_1910_02480_gb300 import synth
    g = synth.gbuffer(N, 1, seed=18)
    x, _ = synth.hemisphere_maps(g["pos"], g["nrm"], H=32, W=32, seed=19)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)
    ctx = drc.Context([16], synth.he_weights([16]), precision="fp32")
    net = drc.UNet(ctx, synth.unet_params(64, 3, seed=0), 64, 3)
    out = torch.empty((N, 3, 32, 32), device=dev)
    for _ in range(warmup):
        net.forward(xd, out=out)
    torch.cuda.synchronize()
    ctx.read_timing()
    ctx.set_timing(True)
    ms = []
    for _ in range(steps):
        a, b = _events(torch)
        a.record()
        net.forward(xd, out=out)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    ctx.set_timing(False)
    kt = ctx.read_timing()
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after the U-Net")
    ms = float(np.mean(ms))
    lf = unet_layer_flops()
    conv_flops = sum(lf.values()) * N
    conv_ms = sum(kt[n][1] for n in lf if n in kt) / steps
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else None
    bf16 = peaks["bf16_tflops"] if peaks else 1900.0
    peak = bf16 * TF32_PER_BF16 / 3.0
    achieved = conv_flops / (conv_ms * 1e-3) / 1e12 if conv_ms > 0 else None
    per_layer = {}
    for n, f in lf.items():
        if n in kt and kt[n][1] > 0:
            lms = kt[n][1] / steps
            per_layer[n] = {"ms": lms, "frac": f * N / (lms * 1e-3) / 1e12 / peak}
    others = {n: v[1] / steps for n, v in kt.items() if n not in lf}
    ctx.close()
    return {"workload": "%d maps 7x32x32, U-Net base 64, 3 levels (7.8 M parameters), fp32 split-tf32 tensor cores"
                        % N,
            "tensor_cores": drc.unet_tensor_cores(64, 3, 32, 32),
            "ms": ms, "maps_per_s": N / (ms * 1e-3), "flops_per_map": unet_flops_per_map(),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if achieved else None, "kernel": "conv_tc_kernel (14 launches)",
                         "kernel_ms_per_call": conv_ms,
                         "peak_source": ("of measured: bf16 burst %.1f TF/s x nominal tf32/bf16 %.3f / 3 products"
                                         % (bf16, TF32_PER_BF16)) if peaks else "of fallback"},
            "per_layer": per_layer, "other_kernels_ms": others}


def make_inputs(seed_offset=0):
    from paper_1910_02480_gb300 import synth
    g = synth.gbuffer(IMG_W, IMG_H, seed=2 + seed_offset)
    c = synth.cache_grid(g, GRID, GRID)
    x, _ = synth.hemisphere_maps(c["pos"], c["nrm"], H=MAP_H, W=MAP_W, seed=3 + seed_offset)
    w = synth.he_weights(WIDTHS, seed=0)
    return w, x, g, c


def cpu_baseline(w, x, g, c, budget_s=12.0, one_thread=False):
    """The FP64 oracle on a bounded sample of the step, scaled to maps/s."""
    import oracle
    from paper_1910_02480_gb300 import synth
    r = synth.world_radius(GRID * GRID)
    t0 = time.perf_counter()
    n_f = 8
    oracle.forward(w, x[:n_f], WIDTHS)
    t_f = time.perf_counter() - t0
    per_map = t_f / n_f
    n_f2 = int(max(8, min(N_MAPS, 0.5 * budget_s / max(per_map, 1e-6))))
    t0 = time.perf_counter()
    ref = oracle.forward(w, x[:n_f2], WIDTHS)
    per_map = (time.perf_counter() - t0) / n_f2
    pay = oracle.payload(np.expm1(ref)).astype(np.float32)
    cc = dict(c)
    cc["payload"] = np.zeros((GRID * GRID, 3), np.float32)
    cc["payload"][:n_f2] = pay
    P = IMG_W * IMG_H
    t0 = time.perf_counter()
    oracle.interpolate(cc, g, K_NN, oracle.METRIC_WORLD, oracle.WP_INVERSE, oracle.INTERP_IRRADIANCE, r,
                       p_range=(0, 2048))
    per_px = (time.perf_counter() - t0) / 2048
    n_p = int(max(2048, min(P, 0.5 * budget_s / max(per_px, 1e-9))))
    t0 = time.perf_counter()
    oracle.interpolate(cc, g, K_NN, oracle.METRIC_WORLD, oracle.WP_INVERSE, oracle.INTERP_IRRADIANCE, r,
                       p_range=(0, n_p))
    per_px = (time.perf_counter() - t0) / n_p
    step_s = per_map * N_MAPS + per_px * P
    cores = oracle.get_threads()
    out = {"value": N_MAPS / step_s, "unit": "maps/s", "cores": cores, "kind": "oracle",
           "sample": "%d of %d maps denoised + %d of %d pixels interpolated (FP64 C oracle, OpenMP), "
                     "scaled to one full step" % (n_f2, N_MAPS, n_p, P),
           "step_s": step_s, "cpu_model": cpu_model()}
    if one_thread:
        # the same on one thread, on a smaller sample (about a tenth of the budget)
        oracle.set_threads(1)
        try:
            m1 = max(2, min(n_f2, int(0.05 * budget_s / max(per_map * cores, 1e-6))))
            t0 = time.perf_counter()
            oracle.forward(w, x[:m1], WIDTHS)
            pm1 = (time.perf_counter() - t0) / m1
            p1 = max(256, min(n_p, int(0.05 * budget_s / max(per_px * cores, 1e-9))))
            t0 = time.perf_counter()
            oracle.interpolate(cc, g, K_NN, oracle.METRIC_WORLD, oracle.WP_INVERSE, oracle.INTERP_IRRADIANCE, r,
                               p_range=(0, p1))
            pp1 = (time.perf_counter() - t0) / p1
        finally:
            oracle.set_threads(cores)
        out["one_thread"] = {"value": N_MAPS / (pm1 * N_MAPS + pp1 * P), "unit": "maps/s",
                             "sample": "%d maps + %d pixels on 1 thread, scaled to one full step" % (m1, p1)}
    return out


def cpu_model():
    """The host CPU's model string (lscpu, else /proc/cpuinfo, else the platform)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        for key in ("model name", "Model name", "CPU part"):
            for line in info.splitlines():
                if line.startswith(key):
                    return line.split(":", 1)[1].strip() + ("" if key != "CPU part" else " (CPU part)")
    except OSError:
        pass
    return platform.processor() or platform.machine()


def max_over_ranks(value, dist, device):
    """The slowest rank's figure (step times are reduced with MAX); the
    value itself on one rank."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, maps_per_rank, ms_per_step):
    """Whole-job throughput: every rank's maps over the slowest rank's step."""
    return world * maps_per_rank / (ms_per_step * 1e-3)


def run_reference(args, rank):
    """--impl reference: the oracle as it stands, timed per step on a bounded
    sample of the same workload."""
    if rank != 0:
        return
    w, x, g, c = make_inputs()
    base = None
    for _ in range(args.warmup):
        base = cpu_baseline(w, x, g, c, budget_s=4.0)
    times = []
    for _ in range(args.steps):
        base = cpu_baseline(w, x, g, c, budget_s=4.0)
        times.append(base["step_s"])
    step = float(np.mean(times))
    val = N_MAPS / step
    line = {"impl": "reference", "metric": METRIC_NAME, "value": val, "unit": "maps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "4096 maps 7x32x32, widths 64/128/256 + 1920x1080 interpolation, k=16 WORLD",
                       "sampled": True},
            "cpu_baseline": {"value": val, "unit": "maps/s", "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": val, "unit": "maps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the precision and uneven-batching lines")
    ap.add_argument("--no-autotune", action="store_true", help="default tile widths instead of drc_autotune")
    ap.add_argument("--tile-cache", default=None, metavar="PATH",
                    help="drc_autotune_cached file: reuse the tiles a previous run chose for this shape (profiling "
                         "runs replay the plain run's choice instead of timing under the profiler)")
    ap.add_argument("--maps", type=int, default=N_MAPS, help="maps per step (profiling of smaller cases)")
    ap.add_argument("--frame", default="%dx%d" % (IMG_W, IMG_H), help="G-buffer WxH (profiling)")
    ap.add_argument("--precision-only", default=None, choices=["bf16", "fp8"],
                    help="only the BF16 or FP8 denoise line (precision_variants) at --maps, --steps timed calls "
                         "(profiling of those conv kernels)")
    ap.add_argument("--unet-only", type=int, default=0, metavar="N",
                    help="only the paper-form U-Net on N maps (profiling): one JSON line, --steps timed forwards")
    args = ap.parse_args()
    set_workload(args.maps, args.frame)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_1910_02480_gb300 as drc
    from paper_1910_02480_gb300 import build, synth
    build.build()
    torch.cuda.set_device(local)
    if args.unet_only > 0:
        print(json.dumps(measure_unet(drc, torch, torch.device("cuda", local), N=args.unet_only,
                                      steps=max(1, args.steps), warmup=max(1, args.warmup))))
        return
    if args.precision_only:
        r = measure_precision(drc, torch, torch.device("cuda", local), args.precision_only, None,
                              autotune=not args.no_autotune, steps=max(1, args.steps), tile_cache=args.tile_cache)
        print(json.dumps(dict(r, precision=args.precision_only, maps=N_MAPS)))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w, x, g, c = make_inputs(seed_offset=rank)
    dev = torch.device("cuda", local)
    ctx = drc.Context(WIDTHS, w, precision=args.precision, max_maps=N_MAPS, max_hw=MAP_H * MAP_W)
    if not args.no_autotune:  # setup: per-layer tile choice for this batch shape
        ctx.autotune(N_MAPS, MAP_H, MAP_W, cache=args.tile_cache)
    tiles = [ctx.describe_layer(li) for li in range(2 * len(WIDTHS))]
    xd = torch.from_numpy(x).to(dev)
    gd = {"width": IMG_W, "height": IMG_H, "pos": torch.from_numpy(g["pos"]).to(dev),
          "nrm": torch.from_numpy(g["nrm"]).to(dev)}
    cd = {"pos": torch.from_numpy(c["pos"]).to(dev), "nrm": torch.from_numpy(c["nrm"]).to(dev),
          "pix": torch.from_numpy(c["pix"]).to(dev)}
    out = torch.empty((N_MAPS, 3, MAP_H, MAP_W), device=dev)
    pay = torch.empty((N_MAPS, 3), device=dev)
    rgb = torch.empty((IMG_W * IMG_H, 3), device=dev)
    cd["payload"] = pay
    r = synth.world_radius(GRID * GRID)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def step():
        ctx.denoise(xd, out=out, payload=pay)
        ctx.interpolate(cd, gd, K_NN, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, r, out=rgb)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after warm-up")

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ctx.read_timing()  # drop anything recorded before the timed region
    ctx.set_timing(True)  # per-kernel CUDA events on the launching stream
    launches0 = ctx.launch_count()
    for i in range(args.steps):
        flush.fill_(float(i))  # evict the previous step's data from L2 (outside the timed events)
        e0, e1, e2 = ev[i]
        e0.record(stream)
        ctx.denoise(xd, out=out, payload=pay)
        e1.record(stream)
        ctx.interpolate(cd, gd, K_NN, drc.METRIC_WORLD, drc.WP_INVERSE, drc.INTERP_IRRADIANCE, r, out=rgb)
        e2.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = ctx.launch_count() - launches0
    ctx.set_timing(False)
    ktimes = ctx.read_timing()
    step_ms = [a.elapsed_time(c_) for a, _, c_ in ev]
    den_ms = [a.elapsed_time(b) for a, b, _ in ev]
    itp_ms = [b.elapsed_time(c_) for _, b, c_ in ev]
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after timed region")
    ms = max_over_ranks(float(np.mean(step_ms)), dist, dev)
    value = job_value(world, N_MAPS, ms)

    # end to end through the public API with host buffers: drc_frame_host
    # copies the pinned maps and G-buffer in and the image out inside every
    # call, overlapping the copies with the compute (chunked map uploads; the
    # next frame's uploads under this frame's interpolation).  The timed
    # region is n_e2e back-to-back frames between two device synchronisations,
    # on the host clock, so every copy of every frame lies inside it; each
    # frame's inputs (167 MB) exceed L2.
    xh = torch.from_numpy(x).pin_memory()
    gh = {"width": IMG_W, "height": IMG_H, "pos": torch.from_numpy(g["pos"]).pin_memory(),
          "nrm": torch.from_numpy(g["nrm"]).pin_memory()}
    rgb_h = torch.empty((IMG_W * IMG_H, 3), dtype=torch.float32).pin_memory()
    cdev = {"pos": cd["pos"], "nrm": cd["nrm"], "pix": cd["pix"]}

    def frame():
        ctx.frame_host(xh, cdev, gh, K_NN, drc.METRIC_WORLD, drc.WP_INVERSE, r, rgb_host=rgb_h)

    for _ in range(2):  # staging allocation, copy stream
        frame()
    torch.cuda.synchronize()
    n_e2e = max(3, min(args.steps, 20))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        frame()
    torch.cuda.synchronize()
    e2e_step = (time.perf_counter() - t0) * 1e3 / n_e2e
    if ctx.status() != drc.OK:
        raise RuntimeError("device status after the end-to-end frames")
    e2e_step = max_over_ranks(e2e_step, dist, dev)
    h2d = x.nbytes + g["pos"].nbytes + g["nrm"].nbytes
    d2h = IMG_W * IMG_H * 3 * 4

    layer_macs = valid_macs_per_layer(WIDTHS, MAP_H, MAP_W)
    den = float(np.mean(den_ms)) * 1e-3
    # the tensor-core conv kernel: its launches' device time (library events on
    # the launching stream, over the timed region) against their valid FLOPs
    conv_names = [n for n in layer_macs if n.startswith("conv")]
    conv_flops = 2.0 * sum(layer_macs[n] for n in conv_names) * N_MAPS
    conv_ms = sum(ktimes[n][1] for n in conv_names if n in ktimes) / args.steps
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else None
    if args.precision == "fp32":
        bf16 = peaks["bf16_tflops"] if peaks else 1900.0
        peak = bf16 * TF32_PER_BF16 / 3.0
        peak_note = ("of measured: bf16 burst %.1f TF/s x nominal tf32/bf16 %.3f / 3 products" % (bf16, TF32_PER_BF16)
                     if peaks else "of fallback: 1.9 PF/s bf16 x tf32/bf16 / 3")
    else:
        peak = peaks["bf16_tflops"] if peaks else 1900.0
        peak_note = "of measured: bf16 burst" if peaks else "of fallback: bf16"
    achieved = conv_flops / (conv_ms * 1e-3) / 1e12 if conv_ms > 0 else None
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None,
                "traffic": TRAFFIC.get(args.precision) if N_MAPS == 4096 else None,
                "kernel": "conv_tc_kernel (%d launches per denoise: %s)" % (len(conv_names), ", ".join(conv_names)),
                "peak_source": peak_note,
                "algorithmic_flops_per_call": conv_flops,
                "kernel_ms_per_call": conv_ms}
    kernels = {n: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps}
               for n, v in ktimes.items()}
    q = ktimes.get("interp query")
    if q:
        kernels["interp query"]["io_gb_per_s"] = IMG_W * IMG_H * 36 / (q[1] / q[0] * 1e-3) / 1e9
    line = {"metric": METRIC_NAME, "value": value, "unit": "maps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16", "data": "synthetic",
            "config": {"workload": "%d maps 7x32x32, encoder 64/128/256 (FP32 production size) + "
                                   "%dx%d interpolation, k=16, WORLD metric, IRRADIANCE" % (N_MAPS, IMG_W, IMG_H),
                       "precision": args.precision, "l2": "flushed between timed steps (256 MB write)",
                       "conv_tiles": {n: {"tile_n": t[0], "a_path": t[1]} for n, t in zip(
                           [k for k in valid_macs_per_layer(WIDTHS, MAP_H, MAP_W)], tiles)},
                       "parallelism": "replica per GPU" if world > 1 else "1 GPU"},
            "denoise_ms": den * 1e3, "interp_ms": float(np.mean(itp_ms)),
            "interp_pixels_per_s": IMG_W * IMG_H / (float(np.mean(itp_ms)) * 1e-3),
            "roofline": roofline,
            "e2e": {"value": job_value(world, N_MAPS, e2e_step), "unit": "maps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "kernels": kernels,
            "clocks": clk}
    if rank == 0 and world == 1 and not args.no_extras and N_MAPS == 4096:
        # secondary lines: one that fails is reported in place, the headline stands
        def extra(name, fn):
            try:
                line[name] = fn()
            except Exception as exc:  # noqa: BLE001
                line[name] = {"error": "%s: %s" % (type(exc).__name__, exc)}

        extra("precision_variants",
              lambda: {p: measure_precision(drc, torch, dev, p, den * 1e3, not args.no_autotune)
                       for p in ("bf16", "fp8") if p != args.precision})
        extra("uneven_batching", lambda: measure_uneven(drc, torch, dev))
        extra("training", lambda: measure_training(drc, torch, dev, recompute=True))
        extra("training_keep_activations", lambda: measure_training(drc, torch, dev, recompute=False))
        extra("training_paper_settings", lambda: measure_training_paper(drc, torch, dev))
        extra("paper_form_unet", lambda: measure_unet(drc, torch, dev))
        extra("map_generation_and_indirect", lambda: measure_mapgen_indirect(drc, torch, dev))
        extra("progressive_passes", lambda: measure_progressive(drc, torch, dev))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        b = cpu_baseline(w, x, g, c, one_thread=True)
        b.pop("step_s", None)
        line["cpu_baseline"] = b
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
