#!/usr/bin/env python
"""Benchmark of the tokenizer hot path on B300: encode + FSQ + drop mask + decode.

One step = one pass of the whole hot path over one synthetic 720p clip
(1 x 3 x 17 x 720 x 1280, default tokenizer: channels 128/256/512, 2 residual
blocks per level, 4x temporal / 8x8 spatial, FSQ [8,8,8,5,5,5]):
  tok_encode (tcgen05 convs, GroupNorm+SiLU, FSQ fused in the last conv)
  -> tok_drop_mask (Philox Bernoulli drop, zero fill, packet row masks)
  -> tok_decode (tcgen05 convs, depth-to-space fused in the up convs).
Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on
a bounded sample of the same workload instead.

Multi-GPU: replicas (each rank its own clip, no data-path collective); value
is the clips of all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("tokenizer encode+decode frames/s at 720p (BF16 vs plain FP32), fwd+bwd step ms, "
          "p99 chunk ms")
WORKLOAD = ("tokenizer encode + FSQ + token drop (15%) + decode of a 1x3x17x720x1280 clip; channels "
            "128/256/512, 2 causal res-blocks per level, 4x8x8 compression, FSQ [8,8,8,5,5,5], BF16 "
            "tcgen05 convs with FP32 accumulation")
LEVELS = (8, 8, 8, 5, 5, 5)
STEM_CH = 128  # channels of the first level (the stem's output)
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}


# DRAM bytes (read + write) of the 33 conv_tc_kernel launches of one 1x3x17x720x1280 encode
# + decode: the ncu dram__bytes_read.sum + dram__bytes_write.sum of the same launches on a
# 5-frame 720p clip, each launch scaled by its tensors' sizes at 17 and at 5 frames.
# Algorithmic: every layer's input read once, its residual read once, its output written
# once. Re-measure when the conv kernel changes.
CONV_DRAM_BYTES_PER_STEP = 29.66e9
CONV_ALGORITHMIC_BYTES_PER_STEP = 31.56e9
CONV_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the 33 conv_tc_kernel launches of a "
                       "1x3x5x720x1280 encode + decode, each scaled to the 17-frame launch by its tensor sizes")
# The stem (stem_tc_kernel: pixels -> 128 channels, im2col rows formed on chip, GroupNorm
# statistics in its epilogue): its DRAM bytes of the 5-frame capture times 17/5, and its
# algorithmic bytes (the BF16 pixels read once, its output written once).
STEM_DRAM_BYTES_PER_STEP = 0.940e9
STEM_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the stem launch of a 1x3x5x720x1280 "
                       "encode (32.3 + 243.3 MB), times 17/5")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return FALLBACK_PEAKS, "fallback"


# ----------------------------------------------------------------- clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    def __init__(self, gpu_id: str | None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [q.strip() for q in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- our arm

def gpu_arm(args):
    import torch

    import paper_2602_03529_b300 as P
    from paper_2602_03529_b300 import replicas as R
    import synthetic as S

    R.init()
    rank, local, world = R.world()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, T, H, W = 1, args.T, args.H, args.W
    tk = P.Tokenizer("bf16")
    params = S.weights_for(tk.param_spec(), seed=0)
    tk.set_params(params)
    tk.reserve(N, T, H, W)
    Tq, Hq, Wq = tk.latent_shape(T, H, W)
    x_host = S.to_bf16_f32(S.blurred_noise_clip(1000 + rank, N, T, H, W))
    x = torch.from_numpy(x_host).to(dev, torch.bfloat16)
    z = torch.empty((N, Tq, Hq, Wq, len(LEVELS)), device=dev)
    idx = torch.empty((N, Tq, Hq, Wq), device=dev, dtype=torch.int32)
    idx_d = torch.empty_like(idx)
    kb = torch.empty((N, Tq, Hq, (Wq + 31) // 32), device=dev, dtype=torch.int32)
    xh = torch.empty((N, T, H, W, 3), device=dev)
    flush = torch.empty(256 << 20, device=dev, dtype=torch.uint8)  # > L2 (126 MB)
    rate = 0.15

    def step(i, xin=None, out=None):
        tk.encode(x if xin is None else xin, z, idx)
        P.drop_mask(idx, rate, seed=12345, stream_id=rank, chunk_id=i, levels=LEVELS, out=idx_d, keep_bits=kb)
        tk.decode(idx_d, H, W, out=xh if out is None else out)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    assert tk.status() == 0, "device-side error during warm-up"

    # ---------------- timed region: device-resident inputs, L2 flushed per step
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    R.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(uuid) if rank == 0 else None
    tk.profile(True)
    tk.profile_read()
    l0 = tk.launch_count()
    evs = []
    for i in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step(args.warmup + i)
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    R.barrier()
    clocks = sampler.stop() if sampler else None
    launches = tk.launch_count() - l0 + args.steps  # + one drop-mask kernel per step
    recs = tk.profile_records()
    prof = tk.profile_read()
    tk.profile(False)
    assert tk.status() == 0, "device-side error in the timed region"
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    total_ms = R.max_over_ranks(total_ms)
    frames = world * N * T * args.steps
    value = frames / (total_ms / 1e3)

    # ---------------- end to end: pinned host clips in, decoded frames out, as a pipeline:
    # the upload of clip i+1 and the download of clip i-1 run on their own copy streams
    # while clip i is coded (double buffers on both sides; every clip's copies are timed)
    xpin = [torch.from_numpy(x_host).to(torch.bfloat16).pin_memory() for _ in range(2)]
    xhpin = [torch.empty((N, T, H, W, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    xdev = [torch.empty_like(x) for _ in range(2)]
    xhdev = [torch.empty_like(xh) for _ in range(2)]
    up, down, comp = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.current_stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(4, min(args.steps, 8))
    R.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        bb = i % 2
        with torch.cuda.stream(up):
            if i >= 2:
                up.wait_event(ev_done[bb])  # clip i-2 no longer reads this input buffer
            xdev[bb].copy_(xpin[bb], non_blocking=True)
            ev_in[bb].record(up)
        comp.wait_event(ev_in[bb])
        if i >= 2:
            comp.wait_event(ev_out[bb])  # clip i-2's frames have left this output buffer
        step(10_000 + i, xin=xdev[bb], out=xhdev[bb])
        ev_done[bb].record(comp)
        with torch.cuda.stream(down):
            down.wait_event(ev_done[bb])
            xhpin[bb].copy_(xhdev[bb], non_blocking=True)
            ev_out[bb].record(down)
    torch.cuda.synchronize()
    e2e_s = R.max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * N * T * e2e_steps / e2e_s, "unit": "frames/s", "steps": e2e_steps,
           "pipelined": "upload of clip i+1 and download of clip i-1 overlap the coding of clip i",
           "h2d_bytes_per_step": xpin[0].numel() * 2, "d2h_bytes_per_step": xhpin[0].numel() * 4}

    # ---------------- the plain FP32 CUDA-core path (denominator of the 5x target)
    fp32 = None
    if not args.no_fp32:
        tf = P.Tokenizer("fp32")
        tf.set_params(params)
        tf.reserve(N, T, H, W)
        xf = torch.from_numpy(x_host).to(dev)
        zf = torch.empty_like(z)

        def fstep(i):
            tf.encode(xf, zf, idx)
            P.drop_mask(idx, rate, seed=12345, stream_id=rank, chunk_id=i, levels=LEVELS, out=idx_d,
                        keep_bits=kb)
            tf.decode(idx_d, H, W, out=xh)

        fstep(0)
        torch.cuda.synchronize()
        ks = max(1, min(2, args.steps))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(ks):
            fstep(1 + i)
        e1.record()
        torch.cuda.synchronize()
        fms = R.max_over_ranks(e0.elapsed_time(e1))
        fp32 = {"value": world * N * T * ks / (fms / 1e3), "unit": "frames/s", "ms_per_step": fms / ks}
        assert tf.status() == 0
        tf.close()

    peaks, peak_src = load_peaks()
    # the stem is its own kernel (stem_tc_kernel); the conv roofline covers conv_tc_kernel
    stem = [r for r in recs if r["cls"] == 0 and r["name"] == "enc.stem"]
    stem_ms, stem_flop = sum(r["ms"] for r in stem), sum(r["work"] for r in stem)
    conv_ms, conv_flop = prof["conv_ms"] - stem_ms, prof["conv_flop"] - stem_flop
    conv_tflops = conv_flop / (conv_ms / 1e3) / 1e12 if conv_ms > 0 else 0.0
    stem_alg = N * T * H * W * 3 * 2 + N * T * (H // 2) * (W // 2) * STEM_CH * 2  # stride (1, 2, 2)
    stem_gbs = stem_alg * len(stem) / (stem_ms / 1e3) / 1e9 if stem_ms > 0 else 0.0
    peak = float(peaks["bf16_tflops_sustained"])
    roofline = {
        "kernel": "conv_tc_kernel (tcgen05 implicit-GEMM causal conv, all launches)",
        "bound": "tensor", "achieved": conv_tflops, "peak": peak, "unit": "TFLOP/s",
        "frac": conv_tflops / peak,
        "peak_source": f"{peak_src} bf16_tflops_sustained (kernel inside a long step)",
        "frac_of_burst_peak": conv_tflops / float(peaks["bf16_tflops"]),
        "traffic": CONV_DRAM_BYTES_PER_STEP, "traffic_unit": "bytes per step (33 launches)",
        "traffic_algorithmic": CONV_ALGORITHMIC_BYTES_PER_STEP, "traffic_source": CONV_TRAFFIC_SOURCE,
        "flop_per_step": conv_flop / args.steps,
        "launches_per_step": (prof["conv_launches"] - len(stem)) / args.steps,
        "conv_ms_per_step": conv_ms / args.steps,
        "conv_share_of_step": conv_ms / max(total_ms, 1e-9),
        "stem": {"kernel": "stem_tc_kernel (pixels -> 128 channels, stride (1,2,2), im2col rows formed in "
                           "shared memory, bias and GroupNorm statistics in the epilogue)",
                 "bound": "hbm", "ms_per_step": stem_ms / args.steps,
                 "algorithmic_bytes": stem_alg, "achieved_gbs": stem_gbs, "peak_gbs": float(peaks["hbm_gbs"]),
                 "frac": stem_gbs / float(peaks["hbm_gbs"]), "traffic": STEM_DRAM_BYTES_PER_STEP,
                 "traffic_source": STEM_TRAFFIC_SOURCE,
                 "note": "bound by instruction issue in its epilogue (about 8300 warp instructions per "
                         "128-voxel tile, 61% issue active under ncu), not by HBM"},
        "groupnorm": {"ms_per_step": prof["gn_ms"] / args.steps,
                      "achieved_gbs": prof["gn_bytes"] / (prof["gn_ms"] / 1e3) / 1e9 if prof["gn_ms"] else 0.0,
                      "peak_gbs": float(peaks["hbm_gbs"])},
        "other_ms_per_step": prof["other_ms"] / args.steps,
    }
    out = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "T": T, "H": H, "W": W, "latent": [Tq, Hq, Wq],
                   "parallelism": f"replicas x{world}", "drop_rate": rate,
                   "l2": "256 MB buffer written before every timed step (L2 is 126 MB); activations are ~1 GB each"},
        "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "fp32_path": fp32, "speedup_vs_fp32": (value / fp32["value"]) if fp32 else None,
    }
    out["residuals"] = residuals(x, xh, roofline["groupnorm"]["peak_gbs"])
    tk.close()
    if not args.no_train:
        out["training"] = training(args, params)
    if not args.no_group:
        out["grouped"] = grouped(args, params, roofline["peak"])
    out["selection"] = selection(args, roofline["groupnorm"]["peak_gbs"])
    out["gop_smoothing"] = gop_smoothing(roofline["groupnorm"]["peak_gbs"])
    out["token_kernels"] = token_kernels(roofline["groupnorm"]["peak_gbs"])
    out["cudnn_reference"] = cudnn_reference(roofline["peak"])
    if not args.no_rsa:
        tk8 = P.Tokenizer("bf16", t_stem=2)
        p8 = S.weights_for(tk8.param_spec(), seed=0)
        tk8.close()
        out["rsa_8x8x8"] = rsa_8x8x8(p8, roofline["groupnorm"]["peak_gbs"])
    if not args.no_serve:
        out["serving"] = serving(args, params, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    R.barrier()
    R.finalize()
    return out if rank == 0 else None


# ------------------------------------------------------------- training

def training(args, params, N=2, T=17, H=256, W=256, steps=5, warmup=2):
    """Joint training step (forward with drop + MSE + hand-written backward + SGD) of the
    default tokenizer on a 2x3x17x256x256 BF16 batch, in both memory modes: per-residual-
    block recomputation (the default; block interiors rebuilt in the backward) and keeping
    the interiors from the forward."""
    import torch

    import paper_2602_03529_b300 as P
    from paper_2602_03529_b300.train import Trainer
    import synthetic as S

    x = torch.from_numpy(S.blurred_noise_clip(7, N, T, H, W)).to("cuda", torch.bfloat16)
    out = {"workload": f"fwd+bwd step, batch {N}x3x{T}x{H}x{W}, BF16, MSE, STE, drop 10%, SGD with the weight "
                       "re-pack", "steps": steps, "warmup": warmup}
    for mode, rc in (("recompute", True), ("keep", False)):
        tk = P.Tokenizer("bf16")
        tk.set_params(params)
        tr = Trainer(tk, N, T, H, W, recompute=rc)
        for i in range(warmup):
            tr.step(x, 0.1, 1, i, lr=1e-5)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        for i in range(steps):
            e = ev[i]
            e[0].record()
            tr.forward(x, 0.1, 1, 100 + i)
            e[1].record()
            tr.backward()
            e[2].record()
            tr.sgd(1e-5)
            e[3].record()
        torch.cuda.synchronize()
        assert tk.status() == 0, "device-side error in the training step"
        fwd = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
        bwd = sum(e[1].elapsed_time(e[2]) for e in ev) / steps
        upd = sum(e[2].elapsed_time(e[3]) for e in ev) / steps
        out[mode] = {"step_ms": fwd + bwd + upd, "fwd_ms": fwd, "bwd_ms": bwd, "sgd_ms": upd,
                     "loss": float(tr.loss.item()), "workspace_bytes": tr.workspace_bytes}
        tk.close()
    out["step_ms"] = out["recompute"]["step_ms"]  # the default mode
    return out


# ------------------------------------------------------------- grouped

GROUP_RES = [(360, 640), (480, 854), (720, 1280), (1080, 1920)]


def grouped(args, params, peak_tflops, steps=3, warmup=2, T=17):
    """One grouped forward (encode + decode) over four 17-frame clips at 360p, 480p,
    720p and 1080p: every conv of a layer is one tensor-core launch over the four
    clips. Timed beside the same four clips run one after another."""
    import torch

    import paper_2602_03529_b300 as P
    import synthetic as S

    tk = P.Tokenizer("bf16")
    tk.set_params(params)
    shapes = [(1, T, h, w) for h, w in GROUP_RES]
    tk.reserve_batch(shapes)
    xs = [torch.from_numpy(S.to_bf16_f32(S.moving_rects_clip(i, T, h, w)[None])).to("cuda", torch.bfloat16)
          for i, (h, w) in enumerate(GROUP_RES)]
    flush = torch.empty(256 << 20, device="cuda", dtype=torch.uint8)

    def batch():
        _, ids = tk.encode_batch(xs, want_z=False)
        return tk.decode_batch(ids, GROUP_RES)

    def single():
        for x, (h, w) in zip(xs, GROUP_RES):
            _, idx = tk.encode(x, want_z=False)
            tk.decode(idx, h, w)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / steps

    l0 = tk.launch_count()
    batch()
    launches = tk.launch_count() - l0
    batch_ms = timed(batch)
    single_ms = timed(single)
    tk.profile(True)
    tk.profile_read()
    batch()
    torch.cuda.synchronize()
    prof = tk.profile_read()
    tk.profile(False)
    assert tk.status() == 0, "device-side error in the grouped forward"
    tk.close()
    frames = T * len(GROUP_RES)
    conv_tf = prof["conv_flop"] / (prof["conv_ms"] / 1e3) / 1e12 if prof["conv_ms"] > 0 else None
    return {"workload": "encode + decode of 4 clips x 17 frames at 360x640, 480x854, 720x1280, 1080x1920 "
                        "(moving rectangles over smooth noise), BF16, one grouped launch per layer",
            "ms": batch_ms, "frames_per_s": frames / (batch_ms / 1e3), "launches": launches,
            "conv_tflop": prof["conv_flop"] / 1e12, "conv_ms": prof["conv_ms"],
            "conv_tflops": conv_tf, "conv_frac": (conv_tf / peak_tflops) if conv_tf else None,
            "peak_tflops": peak_tflops, "sequential_ms": single_ms,
            "speedup_vs_sequential": single_ms / batch_ms, "steps": steps, "warmup": warmup}


# ------------------------------------------------------------- token selection

def selection(args, hbm_gbs, streams=256, Tp=4, Hq=90, Wq=160, rate=0.25, steps=10, warmup=3):
    """Similarity-based token selection (Eq. 3) over the P latents of a batch of 720p chunks
    (256 streams x 4 P latent frames x 90 x 160 tokens against each stream's I latent: inputs,
    outputs and keys exceed L2).
    Algorithmic bytes = P indices read + I indices read + indices written + keep bits written."""
    import numpy as np
    import torch

    import paper_2602_03529_b300 as P

    rng = np.random.default_rng(5)
    ii = rng.integers(0, 64000, (streams, 1, Hq, Wq))
    ip = np.where(rng.random((streams, Tp, Hq, Wq)) < 0.5, np.repeat(ii, Tp, axis=1),
                  rng.integers(0, 64000, (streams, Tp, Hq, Wq)))
    dp = torch.from_numpy(ip.astype(np.int32)).cuda()
    di = torch.from_numpy(ii.astype(np.int32)).cuda()
    out = torch.empty_like(dp)
    kb = torch.empty((streams, Tp, Hq, (Wq + 31) // 32), device="cuda", dtype=torch.int32)
    need = P._lib.tok_similarity_workspace_bytes(streams, Tp, Hq, Wq)
    ws = torch.empty(need, device="cuda", dtype=torch.uint8)

    def run():
        P._lib.tok_similarity_mask(dp.data_ptr(), di.data_ptr(), streams, Tp, Hq, Wq, list(LEVELS), rate,
                                   out.data_ptr(), kb.data_ptr(), None, ws.data_ptr(), need, None)

    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ntok = streams * Tp * Hq * Wq
    nbytes = ntok * 4 + streams * Hq * Wq * 4 + ntok * 4 + kb.numel() * 4
    return {"workload": f"{streams} streams x {Tp} P latent frames x {Hq}x{Wq} tokens (720p chunks), "
                        f"drop rate {rate}", "tokens": ntok, "ms": ms, "tokens_per_s": ntok / (ms / 1e3),
            "achieved_gbs": nbytes / (ms / 1e3) / 1e9, "peak_gbs": hbm_gbs,
            "frac": nbytes / (ms / 1e3) / 1e9 / hbm_gbs, "algorithmic_bytes": nbytes,
            "note": "2 launches: code and similarity tables, then one 1024-thread block per latent frame "
                    "(integer-form cosines, 2048-bucket histogram, threshold bucket resolved as one value, "
                    "a candidate radix select or a whole-frame radix select, tie cut by position, drop and "
                    "keep bits); bound by instruction issue (about 8.7 warp instructions per token), not by "
                    "HBM"}


# ------------------------------------------------------------- a library reference point

def cudnn_reference(peak_tflops, steps=10, warmup=3):
    """A labelled reference point, not part of the timed step: torch's conv3d (cuDNN)
    in BF16 on the level-0 layer of the 720p step (17 x 360 x 640, 128 -> 128 channels,
    3x3x3; zero-padded in time instead of causal, the same FLOPs), channels-last, beside
    this library's tok_conv3d on the same layer (replicate-causal)."""
    import torch
    import torch.nn.functional as F

    import paper_2602_03529_b300 as P

    T, H, W, C = 17, 360, 640, 128
    g = torch.Generator(device="cuda").manual_seed(4)
    x = torch.randn((1, T, H, W, C), device="cuda", generator=g).to(torch.bfloat16)
    w = torch.randn((C, 3, 3, 3, C), device="cuda", generator=g) * 0.02
    b = torch.zeros(C, device="cuda")
    flop = 2.0 * T * H * W * C * 27 * C
    xt = x.permute(0, 4, 1, 2, 3).contiguous(memory_format=torch.channels_last_3d)
    wt = w.permute(0, 4, 1, 2, 3).to(torch.bfloat16).contiguous(memory_format=torch.channels_last_3d)

    def timed(fn, reps=steps):
        for _ in range(min(warmup, reps)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_cudnn = timed(lambda: F.conv3d(xt, wt, padding=1))
    ms_ours = timed(lambda: P.conv3d(x, w, b, (1, 1, 1), "replicate"))
    # plain FP32 on the CUDA cores on both sides (no TF32): cuDNN against this library's FP32 path
    x32, xt32, wt32 = x.float(), xt.float(), wt.float()
    tf32 = torch.backends.cudnn.allow_tf32
    torch.backends.cudnn.allow_tf32 = False
    try:
        ms_cudnn32 = timed(lambda: F.conv3d(xt32, wt32, padding=1), reps=3)
    finally:
        torch.backends.cudnn.allow_tf32 = tf32
    ms_ours32 = timed(lambda: P.conv3d(x32, w, b, (1, 1, 1), "replicate"), reps=3)
    return {"workload": "level-0 conv of the 720p step: 1x17x360x640, 128 -> 128 channels, 3x3x3, BF16",
            "tflop": flop / 1e12, "cudnn_ms": ms_cudnn, "cudnn_tflops": flop / (ms_cudnn / 1e3) / 1e12,
            "ours_ms": ms_ours, "ours_tflops": flop / (ms_ours / 1e3) / 1e12, "peak_tflops": peak_tflops,
            "fp32": {"cudnn_ms": ms_cudnn32, "cudnn_tflops": flop / (ms_cudnn32 / 1e3) / 1e12, "ours_ms": ms_ours32,
                     "ours_tflops": flop / (ms_ours32 / 1e3) / 1e12,
                     "note": "plain FP32 (cuDNN with TF32 off; ours: the CUDA-core FP32 path)"},
            "note": "torch.nn.functional.conv3d (cuDNN), channels_last_3d, symmetric zero padding; ours: tok_conv3d "
                    "(weight packing included in every call)"}


# ------------------------------------------------------------- FSQ and drop mask alone

def token_kernels(hbm_gbs, steps=10, warmup=3):
    """The FSQ (K3) and drop-mask (K4) kernels stand-alone at working sets above 1 GB:
    tok_quantize over 2^26 latent vectors of 6 fp32 channels (24 B in + 4 B out per
    token: 1.88 GB), tok_drop_mask over 2048 streams x 4 latent frames x 90 x 160 tokens
    of 720p chunks at rate 0.15 (4 B in + 4 B out per token + 4 B per 32-token row word:
    0.96 GB). Device-resident inputs; every launch streams more than 8x L2."""
    import torch

    import paper_2602_03529_b300 as P

    g = torch.Generator(device="cuda").manual_seed(11)
    ntok = 1 << 26
    z = torch.randn((ntok, len(LEVELS)), device="cuda", generator=g)
    idx = torch.empty(ntok, device="cuda", dtype=torch.int32)

    def q():
        P._lib.tok_quantize(z.data_ptr(), ntok, list(LEVELS), idx.data_ptr(), None, None)

    shape = (2048, 4, 90, 160)
    tok = torch.randint(0, 64000, shape, device="cuda", dtype=torch.int32, generator=g)
    out = torch.empty_like(tok)
    kb = torch.empty(shape[:3] + ((shape[3] + 31) // 32,), device="cuda", dtype=torch.int32)

    def d(i=[0]):
        i[0] += 1
        P.drop_mask(tok, 0.15, seed=5, stream_id=0, chunk_id=i[0], levels=LEVELS, out=out, keep_bits=kb)

    res = {"workload": "tok_quantize: 2^26 tokens x 6 fp32 channels; tok_drop_mask: 2048 x 4 x 90 x 160 tokens, "
                       "rate 0.15", "peak_gbs": hbm_gbs}
    for name, fn, nbytes, n in (("quantize", q, ntok * (4 * len(LEVELS) + 4), ntok),
                                ("drop_mask", d, tok.numel() * 8 + kb.numel() * 4, tok.numel())):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        gbs = nbytes / (ms / 1e3) / 1e9
        res[name] = {"tokens": n, "ms": ms, "algorithmic_bytes": nbytes, "achieved_gbs": gbs, "frac": gbs / hbm_gbs,
                     "tokens_per_s": n / (ms / 1e3)}
    return res


# ------------------------------------------------------------- pixel residuals

def residuals(x, xh, hbm_gbs, window=4, theta=0.05, steps=10, warmup=3):
    """Pixel residual path (Eq. 4) on the 720p clip and its reconstruction from the timed
    step: window means of x - x_hat with theta zeroing, the sparse form, and the
    receiver-side add. HBM-bound; algorithmic bytes per stage as listed."""
    import torch

    import paper_2602_03529_b300 as P

    N, T, H, W, C = x.shape
    r = P.residual(x, xh, window, theta)
    pos, val, offs = P.residual_sparse(r)
    xr = xh.clone()
    for _ in range(warmup):
        r = P.residual(x, xh, window, theta)
        pos, val, offs = P.residual_sparse(r)
        P.residual_apply(xr, window, pos, val, offs)
    torch.cuda.synchronize()
    # each stage `steps` times back to back between two events, so that the host's
    # launch latency overlaps the device work instead of being timed with it
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    for _ in range(steps):
        r = P.residual(x, xh, window, theta)
    ev[1].record()
    for _ in range(steps):
        pos, val, offs = P.residual_sparse(r)
    ev[2].record()
    for _ in range(steps):
        P.residual_apply(xr, window, pos, val, offs)
    ev[3].record()
    torch.cuda.synchronize()
    t = [ev[i].elapsed_time(ev[i + 1]) / steps for i in range(3)]
    nnz = int(offs[-1].item())
    E = H * W * C
    nwin = (T + window - 1) // window
    b_mean = N * T * E * (x.element_size() + 4) + N * nwin * E * 4
    b_sparse = 2 * N * nwin * E * 4 + nnz * 8
    b_apply = nnz * 8 + 2 * nnz * window * 4
    return {"workload": f"{N}x{T}x{H}x{W}x{C} clip and its reconstruction, {window}-frame windows, "
                        f"theta {theta}", "nonzeros": nnz, "density": nnz / (N * nwin * E),
            "mean_ms": t[0], "mean_gbs": b_mean / (t[0] / 1e3) / 1e9, "mean_frac": b_mean / (t[0] / 1e3) / 1e9 / hbm_gbs,
            "sparse_ms": t[1], "sparse_gbs": b_sparse / (t[1] / 1e3) / 1e9,
            "apply_ms": t[2], "apply_gbs": b_apply / (t[2] / 1e3) / 1e9 if t[2] > 0 else None,
            "peak_gbs": hbm_gbs}


# ------------------------------------------------------------- GoP boundary smoothing

def gop_smoothing(hbm_gbs, N=8, T=9, H=720, W=1280, n=4, steps=10, warmup=3):
    """Eq. 2 blending and the Eq. 1 boundary loss with its gradient on 8 consecutive 9-frame
    720p GoP reconstructions (fp32 frames). HBM-bound: blend reads n previous + T current
    frames and writes T frames; the loss reads 2n frames, the gradient pass 2n frames and
    writes T frames."""
    import torch

    import paper_2602_03529_b300 as P

    g = torch.Generator(device="cuda").manual_seed(3)
    prev = torch.rand((N, T, H, W, 3), device="cuda", generator=g) * 2 - 1
    curr = torch.rand((N, T, H, W, 3), device="cuda", generator=g) * 2 - 1
    out = torch.empty_like(curr)
    for _ in range(warmup):
        P.gop_blend(prev, curr, n, out=out)
        P.temporal_loss(curr, prev, n)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    for _ in range(steps):
        P.gop_blend(prev, curr, n, out=out)
    ev[1].record()
    for _ in range(steps):
        P.temporal_loss(curr, prev, n)
    ev[2].record()
    torch.cuda.synchronize()
    tb, tl = ev[0].elapsed_time(ev[1]) / steps, ev[1].elapsed_time(ev[2]) / steps
    fb = H * W * 3 * 4
    bb = N * fb * (n + 2 * T)
    bl = N * fb * (2 * n + 2 * n + T)
    return {"workload": f"{N} GoPs x {T} frames at {H}x{W}, n = {n} boundary frames", "blend_ms": tb,
            "blend_gbs": bb / (tb / 1e3) / 1e9, "blend_frac": bb / (tb / 1e3) / 1e9 / hbm_gbs,
            "loss_and_grad_ms": tl, "loss_and_grad_gbs": bl / (tl / 1e3) / 1e9, "peak_gbs": hbm_gbs}


# ------------------------------------------------------------- resolution control + 8x8x8

def rsa_8x8x8(params8, hbm_gbs, N=4, T=17, steps=3, warmup=2):
    """Sec. 5 resolution control feeding the paper's 8x temporal / 8x8 spatial tokenizer
    (Sec. 4.1): N clips of T 1080p uint8 frames are downsampled 3x (640x360) or 2x (960x540)
    to bf16 in [-1, 1], encoded, 15% of tokens dropped, and decoded at the reduced size
    (the learned super-resolution stage is not part of this path). Encoder and decoder
    frames/s are reported apart, as in the paper's scaling table; the downsample kernel
    against HBM (it reads the 1080p frames once and writes the small bf16 frames)."""
    import numpy as np
    import torch

    import paper_2602_03529_b300 as P

    tk = P.Tokenizer("bf16", t_stem=2)
    tk.set_params(params8)
    rng = np.random.default_rng(8)
    x8 = torch.from_numpy(rng.integers(0, 256, (N, T, 1080, 1920, 3), dtype=np.uint8)).cuda()
    flush = torch.empty(256 << 20, device="cuda", dtype=torch.uint8)
    out = {"workload": f"{N} clips x {T} frames of 1080p uint8 -> s x s area downsample -> 8x8x8 tokenizer "
                       "(channels 128/256/512, 2 blocks per level, FSQ [8,8,8,5,5,5]), 15% drop",
           "peak_gbs": hbm_gbs}
    for s in (3, 2):
        H, W = 1080 // s, 1920 // s
        tk.reserve(N, T, H, W)
        Tq, Hq, Wq = tk.latent_shape(T, H, W)
        xs = torch.empty((N, T, H, W, 3), device="cuda", dtype=torch.bfloat16)
        z = torch.empty((N, Tq, Hq, Wq, len(LEVELS)), device="cuda")
        idx = torch.empty((N, Tq, Hq, Wq), device="cuda", dtype=torch.int32)
        idx_d = torch.empty_like(idx)
        xh = torch.empty((N, T, H, W, 3), device="cuda")
        for i in range(warmup):
            P.downsample(x8, s, torch.bfloat16, out=xs)
            tk.encode(xs, z, idx)
            P.drop_mask(idx, 0.15, seed=5, stream_id=0, chunk_id=i, levels=LEVELS, out=idx_d)
            tk.decode(idx_d, H, W, out=xh)
        torch.cuda.synchronize()
        t_ds = t_enc = t_dec = 0.0
        for i in range(steps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record()
            P.downsample(x8, s, torch.bfloat16, out=xs)
            ev[1].record()
            tk.encode(xs, z, idx)
            P.drop_mask(idx, 0.15, seed=5, stream_id=0, chunk_id=100 + i, levels=LEVELS, out=idx_d)
            ev[2].record()
            tk.decode(idx_d, H, W, out=xh)
            ev[3].record()
            torch.cuda.synchronize()
            t_ds += ev[0].elapsed_time(ev[1])
            t_enc += ev[1].elapsed_time(ev[2])
            t_dec += ev[2].elapsed_time(ev[3])
        assert tk.status() == 0
        frames = N * T * steps
        ds_bytes = N * T * (1080 * 1920 * 3 + H * W * 3 * 2)
        out[f"{s}x"] = {"H": H, "W": W, "latent": [Tq, Hq, Wq],
                        "encoder_fps": frames / ((t_ds + t_enc) / 1e3), "decoder_fps": frames / (t_dec / 1e3),
                        "codec_fps": frames / ((t_ds + t_enc + t_dec) / 1e3),
                        "downsample_ms": t_ds / steps, "downsample_gbs": ds_bytes / (t_ds / steps / 1e3) / 1e9,
                        "downsample_frac": ds_bytes / (t_ds / steps / 1e3) / 1e9 / hbm_gbs}
    tk.close()
    return out


# ------------------------------------------------------------- serving

SERVE_RES = [(480, 854), (720, 1280), (1080, 1920)]


def serving(args, params, rank, world):
    """Streaming loop: Poisson-arriving streams of mixed 480p/720p/1080p at 30 fps, causal
    4-frame chunks with on-device conv caches, per-chunk token drop U[0, 30%], BF16."""
    import numpy as np
    import torch

    import synthetic as S
    from paper_2602_03529_b300 import replicas as R
    from paper_2602_03529_b300.serve import GpuExecutor, MemoryPool, Server, StreamSpec

    n = args.serve_streams
    rng = np.random.default_rng(1)
    starts = S.poisson_arrivals(1, n, args.serve_horizon, start_rate_hz=n / args.serve_horizon)
    specs = [StreamSpec(i, *SERVE_RES[int(rng.integers(3))], start=float(starts[i]), n_chunks=args.serve_chunks)
             for i in range(n)]
    mine = [specs[i] for i in R.shard(n, rank, world)]
    clips = {(r, sd): torch.from_numpy(S.moving_rects_clip(100 + sd, 9, *r)).to("cuda", torch.bfloat16)
             for r in SERVE_RES for sd in (0, 1)}

    def content(spec):
        return torch.roll(clips[((spec.H, spec.W), spec.sid % 2)], shifts=spec.sid % 9, dims=0)

    mb = args.serve_batch
    ex = GpuExecutor(args.serve_lanes, params, None, content_fn=content, max_batch=mb, priorities=True,
                     resolutions=SERVE_RES)

    # chunk time of each resolution alone on the urgent lane (steady state: the median of
    # 8 chunks after a first one), with a margin for sharing the GPU with background lanes
    alone = ex.calibrate(reps=8, resolutions=SERVE_RES)

    def service_time(spec):
        return args.serve_margin * alone[(spec.H, spec.W)]

    # admission: memory from the device's free bytes (conv caches + buffers per stream),
    # compute by the streams' measured chunk time per second against the load bound
    mem_budget = ex.memory_budget()
    pool = MemoryPool(ex, mem_budget)
    # warm-up: every lane, every resolution, batches of every size
    warm = [StreamSpec(10_000 + i, *SERVE_RES[i % 3], start=0.0, n_chunks=2) for i in range(12)]
    Server(ex, args.serve_lanes, pool, 1e30, stall_timeout=5.0, max_batch=mb).run(warm, horizon=1.0)
    torch.cuda.synchronize()
    rep = Server(ex, args.serve_lanes, pool, 0.0, target_latency=0.033, stall_timeout=1.0,
                 service_time=service_time, max_batch=mb, align_phases=not args.serve_no_align,
                 load=args.serve_load).run(mine, horizon=args.serve_horizon)
    torch.cuda.synchronize()
    assert all(s == 0 for s in ex.status()), "device-side error while serving"
    slots_opened = {f"{h}x{w}": sum(1 for x in ex.slots.get((h, w), []) if x is not None) for h, w in SERVE_RES}
    stream_gb = {f"{h}x{w}": ex.stream_bytes((h, w)) / 1e9 for h, w in SERVE_RES}
    ex.close()
    rep.pop("admission_wait_s", None)  # per-stream detail; the p50 stays
    rep.update({"lanes": args.serve_lanes, "max_batch": mb, "phase_aligned": not args.serve_no_align,
                "urgent": {f"{h}x{w}": service_time(StreamSpec(0, h, w, 0.0, 1)) <= 0.033 for h, w in SERVE_RES},
                "service_ms": {f"{h}x{w}": 1e3 * service_time(StreamSpec(0, h, w, 0.0, 1)) for h, w in SERVE_RES},
                "chunk_alone_ms": {f"{h}x{w}": 1e3 * alone[(h, w)] for h, w in SERVE_RES},
                "service_margin": args.serve_margin,
                "admission": {"memory_budget_gb": mem_budget / 1e9, "stream_gb": stream_gb,
                              "slots_opened": slots_opened, "memory_allocated_gb": pool.allocated / 1e9,
                              "compute": "sum over admitted streams of chunk service time x 7.5 chunks/s "
                                         f"<= {args.serve_load}"},
                "load_factor": args.serve_load,
                "stream_chunks": args.serve_chunks, "arrival_horizon_s": args.serve_horizon,
                "drop_rate": "U[0, 0.30] per chunk", "target_ms": 33.0})
    return rep


# -------------------------------------------------------- the oracle (CPU)

def oracle_sample(T, H, W, seed=0):
    """Encode + drop + decode of one T x H x W clip by the FP64 oracle; returns seconds."""
    import synthetic as S
    from oracle import Arch, Oracle, ops, param_spec
    a = Arch()
    p = {k: S.to_bf16_f32(v) for k, v in S.weights_for(param_spec(a), seed=0).items()}
    x = S.to_bf16_f32(S.blurred_noise_clip(seed, 1, T, H, W))
    o = Oracle(a, p)
    t0 = time.perf_counter()
    idx, _, _ = o.encode(x)
    dropped = ops.drop_mask(*idx.shape, 0.15, 12345, 0, seed)
    o.decode(ops.apply_drop(idx, dropped, a.levels), H, W)
    return time.perf_counter() - t0


def cpu_baseline(args, T=5, H=128, W=192):
    from oracle import ops
    s = oracle_sample(T, H, W)
    eq = T * H * W / (args.H * args.W)  # 720p-frame equivalents (work scales with pixels)
    return {"value": eq / s, "unit": "frames/s (720p-equivalent)", "cores": ops.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle encode+drop+decode of a 1x3x{T}x{H}x{W} crop of the same workload "
                      f"({s:.1f} s); work scales with pixel count, so frames/s = {eq:.4f} 720p frames / time"}


def reference_arm(args):
    from paper_2602_03529_b300 import replicas as R
    rank, _, world = R.world()
    if rank != 0:
        return None
    from oracle import ops
    T, H, W = 5, 64, 96
    for i in range(args.warmup):
        oracle_sample(T, H, W, seed=i)
    secs = [oracle_sample(T, H, W, seed=100 + i) for i in range(args.steps)]
    total = sum(secs)
    eq = T * H * W / (args.H * args.W) * args.steps
    value = eq / total
    sample = (f"FP64 oracle encode+drop+decode of a 1x3x{T}x{H}x{W} crop per step "
              "(720p-frame equivalents by pixel count)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": 1, "T": args.T, "H": args.H, "W": args.W, "sample": [T, H, W]},
            "cpu_baseline": {"value": value, "unit": "frames/s", "kind": "oracle", "cores": ops.num_threads(),
                             "sample": sample},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}

# ------------------------------------------------------------- profiling workloads
# `python bench.py --case NAME [--N --T --H --W --s]` runs one fixed workload once
# and exits (no JSON line); the ncu captures kept with the measurements name these
# commands. Inputs come from the seeded generators; weights are He-normal from seed 0.

def case_clip(N, T, H, W):
    """One encode + decode of a seeded blurred-noise clip, BF16."""
    import torch

    import paper_2602_03529_b300 as P
    import synthetic as S

    tk = P.Tokenizer("bf16")
    tk.set_params(S.weights_for(tk.param_spec(), seed=0))
    tk.reserve(N, T, H, W)
    x = torch.from_numpy(S.to_bf16_f32(S.blurred_noise_clip(1, N, T, H, W))).to("cuda", torch.bfloat16)
    _, idx = tk.encode(x, want_z=False)
    tk.decode(idx, H, W)
    torch.cuda.synchronize()
    if tk.status() != 0:
        sys.exit(f"device status {tk.status()}")
    print("clip ok", N, T, H, W, f"{tk.workspace_bytes(N, T, H, W) / 1e9:.2f} GB workspace")


def case_train(N, T, H, W, keep=False):
    """One training step (forward with 10% drop, MSE, backward, SGD), then one more
    forward + backward; block interiors rebuilt in the backward (the default), or kept."""
    import torch

    import paper_2602_03529_b300 as P
    from paper_2602_03529_b300.train import Trainer
    import synthetic as S

    tk = P.Tokenizer("bf16")
    tk.set_params(S.weights_for(tk.param_spec(), seed=0))
    tr = Trainer(tk, N, T, H, W, recompute=not keep)
    x = torch.from_numpy(S.blurred_noise_clip(7, N, T, H, W)).to("cuda", torch.bfloat16)
    tr.step(x, 0.1, 1, 0, 1e-5)
    tr.forward(x, 0.1, 1, 1)
    tr.backward()
    torch.cuda.synchronize()
    if tk.status() != 0:
        sys.exit(f"device status {tk.status()}")
    print("train ok", N, T, H, W)


def case_downsample(N, T, H, W, s):
    """Three s x s area downsamples of seeded uint8 frames to bf16 (the resolution
    control of the 1080p encoder input)."""
    import numpy as np
    import torch

    import paper_2602_03529_b300 as P

    x = torch.from_numpy(np.random.default_rng(8).integers(0, 256, (N, T, H, W, 3), dtype=np.uint8)).cuda()
    y = P.downsample(x, s, torch.bfloat16)
    for _ in range(2):
        P.downsample(x, s, torch.bfloat16, out=y)
    torch.cuda.synchronize()
    print("downsample ok", tuple(y.shape))


def case_select(N, T, H, W):
    """Token selection over N streams x T P latent frames of H x W tokens (half of the P
    tokens equal to the I token at their position), drop rate 0.25, three times."""
    import numpy as np
    import torch

    import paper_2602_03529_b300 as P

    rng = np.random.default_rng(5)
    ii = rng.integers(0, 64000, (N, 1, H, W))
    ip = np.where(rng.random((N, T, H, W)) < 0.5, np.repeat(ii, T, axis=1), rng.integers(0, 64000, (N, T, H, W)))
    dp = torch.from_numpy(ip.astype(np.int32)).cuda()
    di = torch.from_numpy(ii.astype(np.int32)).cuda()
    for _ in range(3):
        out, kb, _ = P.similarity_mask(dp, di, 0.25)
    torch.cuda.synchronize()
    print("select ok", tuple(out.shape), int((out == 32036).sum()))


def case_tokens(N, T, H, W):
    """tok_quantize over 2^26 latent vectors of 6 fp32 channels and tok_drop_mask over
    N streams x T latent frames of H x W tokens at rate 0.15, three times each."""
    import torch

    import paper_2602_03529_b300 as P

    g = torch.Generator(device="cuda").manual_seed(11)
    ntok = 1 << 26
    z = torch.randn((ntok, len(LEVELS)), device="cuda", generator=g)
    idx = torch.empty(ntok, device="cuda", dtype=torch.int32)
    tok = torch.randint(0, 64000, (N, T, H, W), device="cuda", generator=g, dtype=torch.int32)
    out = torch.empty_like(tok)
    kb = torch.empty((N, T, H, (W + 31) // 32), device="cuda", dtype=torch.int32)
    for _ in range(3):
        P._lib.tok_quantize(z.data_ptr(), ntok, list(LEVELS), idx.data_ptr(), None, None)
    for i in range(3):
        P.drop_mask(tok, 0.15, seed=5, stream_id=0, chunk_id=i, levels=LEVELS, out=out, keep_bits=kb)
    torch.cuda.synchronize()
    print("tokens ok", int(idx[:4].sum()), int((out == 32036).sum()))


def case_residual_gop(N, T, H, W):
    """The pixel residual path (Eq. 4: window means, sparse form, receiver add) on a
    clip of N x T frames of H x W and a reconstruction of it, then the GoP blend (Eq. 2)
    and boundary loss (Eq. 1) on 4 GoPs of 9 frames at H x W, three times each."""
    import torch

    import paper_2602_03529_b300 as P

    g = torch.Generator(device="cuda").manual_seed(13)
    x = (torch.rand((N, T, H, W, 3), device="cuda", generator=g) * 2 - 1).to(torch.bfloat16)
    xh = x.float() + 0.1 * torch.randn((N, T, H, W, 3), device="cuda", generator=g)
    xr = xh.clone()
    for _ in range(3):
        r = P.residual(x, xh, 4, 0.05)
        pos, val, offs = P.residual_sparse(r)
        P.residual_apply(xr, 4, pos, val, offs)
    prev = torch.rand((4, 9, H, W, 3), device="cuda", generator=g) * 2 - 1
    curr = torch.rand((4, 9, H, W, 3), device="cuda", generator=g) * 2 - 1
    out = torch.empty_like(curr)
    for _ in range(3):
        P.gop_blend(prev, curr, 4, out=out)
        P.temporal_loss(curr, prev, 4)
    torch.cuda.synchronize()
    print("residual-gop ok", int(offs[-1].item()))


def case_chunk(N, T, H, W, chunks=6):
    """One stream of H x W (N and T unused): chunk 0, then `chunks` 4-frame chunks,
    encode + decode each; prints per chunk the event-timed milliseconds and the
    library's per-class kernel time (conv, GroupNorm, other), then, for the last
    chunk, every launch with its time."""
    import torch

    import paper_2602_03529_b300 as P
    import synthetic as S

    tk = P.Tokenizer("bf16")
    tk.set_params(S.weights_for(tk.param_spec(), seed=0))
    x = torch.from_numpy(S.moving_rects_clip(3, 1 + 4 * chunks, H, W)[None]).to("cuda", torch.bfloat16)
    vid = tk.stream_open(H, W)
    tk.profile(True)
    for k in range(chunks + 1):
        a, b = (0, 1) if k == 0 else (4 * k - 3, 4 * k + 1)
        xc = x[:, a:b].contiguous()
        torch.cuda.synchronize()
        tk.profile_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, idx = tk.encode(xc, video=vid, want_z=False)
        tk.decode(idx, H, W, video=vid, first_chunk=(k == 0))
        e1.record()
        torch.cuda.synchronize()
        recs = tk.profile_records()
        prof = tk.profile_read()
        print(f"chunk {k}: {e0.elapsed_time(e1):.3f} ms, conv {prof['conv_ms']:.3f} ms "
              f"({prof['conv_flop'] / 1e12:.2f} TFLOP), gn {prof['gn_ms']:.3f} ms, other {prof['other_ms']:.3f} ms, "
              f"launches {len(recs)}")
    for r in recs:
        print(f"  {r['name']:<24} cls {r['cls']} {r['ms']:.4f} ms")
    tk.stream_close(vid)
    if tk.status() != 0:
        sys.exit(f"device status {tk.status()}")


CASE_SHAPES = {"clip": (1, 5, 720, 1280), "train": (2, 17, 256, 256), "train-keep": (2, 17, 256, 256),
               "downsample": (4, 17, 1080, 1920), "select": (256, 4, 90, 160), "chunk": (1, 5, 1080, 1920),
               "tokens": (2048, 4, 90, 160), "residual-gop": (1, 17, 720, 1280)}


def run_case(args):
    shape = [v if v is not None else d for v, d in zip((args.N, args.T_case, args.H_case, args.W_case),
                                                       CASE_SHAPES[args.case])]
    if args.case == "clip":
        case_clip(*shape)
    elif args.case == "train":
        case_train(*shape)
    elif args.case == "train-keep":
        case_train(*shape, keep=True)
    elif args.case == "downsample":
        case_downsample(*shape, args.s)
    elif args.case == "chunk":
        case_chunk(*shape)
    elif args.case == "residual-gop":
        case_residual_gop(*shape)
    elif args.case == "tokens":
        case_tokens(*shape)
    else:
        case_select(*shape)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--T", type=int, default=17)
    ap.add_argument("--H", type=int, default=720)
    ap.add_argument("--W", type=int, default=1280)
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-group", action="store_true")
    ap.add_argument("--no-rsa", action="store_true", help="skip the downsample + 8x8x8 tokenizer section")
    ap.add_argument("--serve-streams", type=int, default=64)
    ap.add_argument("--serve-horizon", type=float, default=20.0)
    ap.add_argument("--serve-chunks", type=int, default=16)
    ap.add_argument("--serve-lanes", type=int, default=2)
    ap.add_argument("--serve-load", type=float, default=0.75,
                    help="admitted streams' GPU time per second (measured chunk times) at most this")
    ap.add_argument("--serve-batch", type=int, default=4)
    ap.add_argument("--serve-margin", type=float, default=1.10,
                    help="service estimate = margin x measured chunk time alone (urgent iff <= 33 ms)")
    ap.add_argument("--serve-no-align", action="store_true")
    ap.add_argument("--case", choices=sorted(CASE_SHAPES), help="run one fixed profiling workload and exit")
    ap.add_argument("--N", type=int, help="--case: batch")
    ap.add_argument("--case-T", dest="T_case", type=int, help="--case: frames")
    ap.add_argument("--case-H", dest="H_case", type=int, help="--case: height")
    ap.add_argument("--case-W", dest="W_case", type=int, help="--case: width")
    ap.add_argument("--s", type=int, default=3, help="--case downsample: factor")
    args = ap.parse_args()
    if args.case:
        run_case(args)
        return
    out = reference_arm(args) if args.impl == "reference" else gpu_arm(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
