#!/usr/bin/env python
"""Throughput benchmark: escape-time rendering on B300 (paper Sec. 2/3).

One step = the throughput sweep: 16 renders of 4096x4096 pixels (Julia over
[-1.6,1.6]^2 for C in {0.285+0.01i, -0.7269+0.1889i, -0.4+0.6i} and the
Mandelbrot plane over [-2.5,1]x[-1.75,1.75], limits 100 and 1000, binary32 and
binary64), uint16 counts + RGBA8 from a 256-entry palette, all 16 frames as
one batch plan through the C ABI (one jl_batch_launch, a captured CUDA graph,
per step).  The metric is pixel-iterations per second
(sum of escape counts / time) and the fraction of the binary32 / binary64
issue peak measured on the same GPU by jl_probe_peak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): each rank renders its own full sweep (weak scaling, no
collective on the data path); rank 0 prints one JSON line.  --impl reference
times the CPU oracle on the host cores on a fixed row sample of the same
workload (every ORACLE_ROW_STRIDE-th row of every frame), the same sample as
the JSON line's cpu_baseline.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pixel-iterations/sec (Giter/s) and % FP32/FP64 peak; C-values screened/sec at hist-L1<=0.05"
UNIT = "Giter/s"
WORKLOAD = ("throughput sweep: 16 renders of 4096x4096 (Julia [-1.6,1.6]^2, C in {0.285+0.01i, "
            "-0.7269+0.1889i, -0.4+0.6i}; Mandelbrot [-2.5,1]x[-1.75,1.75]) x limit {100,1000} x "
            "{binary32, binary64}; uint16 counts + RGBA8")
OPS_PER_ITER = 8  # 3 multiplies + 5 adds per escape-time step (no FMA)
CERT_OPS = 9      # binary32 arithmetic of one step of the certified binary32 pass
CERT2_OPS = 62    # binary32 arithmetic of one step of the double-float pass
# The oracle's sample of the sweep: every 8th row of each frame (512 rows of
# 4096, interleaved over the host threads), about a second of all-core work.
ORACLE_ROW_STRIDE = 8


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--size", type=int, default=4096)
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-survey", action="store_true", help="skip the surrogate screening workload")
    p.add_argument("--survey-epochs", type=int, default=300)
    p.add_argument("--no-extra", action="store_true", help="skip the path-animation and deep-zoom sections")
    p.add_argument("--tune-save", default=None, help="write the autotuned launch shapes to this file")
    p.add_argument("--tune-load", default=None,
                   help="load launch shapes from this file instead of autotuning (e.g. to replay a plain run's "
                        "choices under a profiler, whose per-launch overhead would distort the tuning)")
    return p.parse_args()


FLOP_PER_C = 2 * (64 * 256 + 256 * 256 + 256 * 101)  # forward of the surrogate network
# one training sample: the forward, the three weight-gradient products
# (dW1, dW2, dW3: the forward's size again) and the two error products
# dH2 = dZ W3 (101 x 256) and dH1 = dZ2 W2 (256 x 256)
FLOP_TRAIN_PER_SAMPLE = 2 * FLOP_PER_C + 2 * (101 * 256 + 256 * 256)


def run_survey(args, K, W):
    """Surrogate screening workload: 65,536 training C rendered 128x128 over
    [-2,2]^2 (limit 100) as histogram targets, training on the device, then
    1,048,576 candidate C screened by predicted-histogram entropy with the top
    1% re-rendered as the judge; plain batched rendering of every candidate
    is timed beside it."""
    import torch

    from paper_1611_03079_b300 import surrogate as sg, workloads as wl
    ctr = torch.from_numpy(wl.survey_train()).cuda()
    held = torch.from_numpy(wl.survey_heldout()).cuda()
    cand = torch.from_numpy(wl.survey_candidates()).cuda()
    n, k = cand.shape[0], cand.shape[0] // 100
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    # targets
    tplan = sg.HistogramPlan(ctr.cpu().numpy())
    e0, e1 = ev(), ev()
    e0.record()
    T = tplan.launch()
    e1.record()
    torch.cuda.synchronize()
    t_targets = e0.elapsed_time(e1) * 1e-3
    Th = sg.render_histograms(held.cpu().numpy())
    # training
    m = sg.Surrogate(wl.fourier_matrix(), wl.mlp_init())
    order = torch.from_numpy(sg.Surrogate.epoch_order(ctr.shape[0], args.survey_epochs, 1)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    curve = m.train(ctr, T, args.survey_epochs, batch=1024, lr=2e-3, lr_final=1e-5, order=order)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    train_steps = args.survey_epochs * (ctr.shape[0] // 1024)
    P, _ = m.forward(held)
    held_l1 = float(sg.hist_l1(P, Th).mean())
    # plain batched rendering of every candidate (the method without the network)
    plan = sg.HistogramPlan(cand.cpu().numpy())
    for _ in range(max(W, 1)):
        plan.launch()
    e0, e1 = ev(), ev()
    e0.record()
    for _ in range(K):
        Tc = plan.launch()
    e1.record()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) * 1e-3 / K
    # screening (fused forward + top-k), timed alone and as the forward only;
    # the same outputs every call (the library replays one CUDA graph)
    sout = (torch.empty(k, dtype=torch.int32, device="cuda"), torch.empty(k, dtype=torch.float32, device="cuda"),
            torch.empty(n, dtype=torch.float32, device="cuda"))
    for _ in range(max(W, 2)):
        idx, val, S = m.survey(cand, k, out=sout)
    e0, e1 = ev(), ev()
    e0.record()
    for _ in range(K):
        idx, val, S = m.survey(cand, k, out=sout)
    e1.record()
    torch.cuda.synchronize()
    t_survey = e0.elapsed_time(e1) * 1e-3 / K
    e0, e1 = ev(), ev()
    e0.record()
    for _ in range(K):
        m.forward(cand, probs=False, score=True)
    e1.record()
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1) * 1e-3 / K
    # judge: predicted vs rendered histograms of the selected C
    Pk, _ = m.forward(cand[idx.long()].contiguous())
    l1 = sg.hist_l1(Pk, Tc[idx.long()].contiguous())
    ent = -(torch.where(Tc > 0, Tc * torch.log(Tc), torch.zeros_like(Tc))).sum(1)
    res = {"candidates": n, "k": k, "screened_per_s": n / t_survey, "plain_render_per_s": n / t_plain,
           "speedup_vs_plain_render": t_plain / t_survey, "survey_ms": t_survey * 1e3, "forward_ms": t_fwd * 1e3,
           "plain_render_ms": t_plain * 1e3, "judge_l1_mean": float(l1.mean()),
           "judge_l1_p95": float(l1.quantile(0.95)), "judge_l1_max": float(l1.max()),
           "l1_target_met": bool(float(l1.mean()) <= 0.05), "heldout_l1_mean": held_l1,
           "targets_ms": t_targets * 1e3, "train_s": t_train, "train_epochs": args.survey_epochs,
           "final_loss": float(curve[-1]),
           "true_entropy_selected": float(ent[idx.long()].mean()), "true_entropy_all": float(ent.mean()),
           "roofline_forward": {"bound": "tensor", "kernel": "fused_forward_kernel",
                                "achieved": FLOP_PER_C * n / t_fwd / 1e12, "unit": "TFLOP/s",
                                "algorithmic_unit": "%d FLOP per C (bf16 products)" % FLOP_PER_C},
           "roofline_training": {"bound": "tensor", "kernels": "train_step_kernel + adam_kernel per step",
                                 "achieved": FLOP_TRAIN_PER_SAMPLE * 1024 * train_steps / t_train / 1e12,
                                 "unit": "TFLOP/s", "steps": train_steps, "us_per_step": t_train / train_steps * 1e6,
                                 "launches_per_step": 2,
                                 "algorithmic_unit": "%d FLOP per training sample (bf16 products), batch 1024"
                                                     % FLOP_TRAIN_PER_SAMPLE,
                                 "timing": "host wall clock of jl_train over all epochs (the per-epoch sample "
                                           "permutations are drawn and copied to the device before it; the loss "
                                           "read-back is inside)"}}
    tplan.close()
    plan.close()
    m.close()
    return res


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, ".bench_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed region starts once the sampler is running (its first line is written)
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
    return world, rank, local


def cpu_sample(frames, stride=ORACLE_ROW_STRIDE, threads=None):
    """The oracle (as it stands) on every stride-th row of every frame, rows
    interleaved over the host threads.  Returns (Giter/s, threads,
    description, iterations, seconds)."""
    import numpy as np
    import oracle
    threads = threads or min(os.cpu_count() or 1, 64)
    t0 = time.perf_counter()
    iters = rows = 0
    for f in frames:
        n_rows = len(range(stride // 2, f["H"], stride))
        k = oracle.render_strided(f["c"], f["rect"], f["W"], f["H"], stride // 2, stride, n_rows,
                                  f["max_iter"], f["mode"], f["precision"], threads=threads)
        iters += int(k.astype(np.int64).sum())
        rows += n_rows
    secs = time.perf_counter() - t0
    desc = ("every %d-th row of each of the %d sweep frames (%d rows, %.3g G iterations), %d threads"
            % (stride, len(frames), rows, iters / 1e9, threads))
    return iters / secs / 1e9, threads, desc, iters, secs


def run_single_frame(K, W, peak32):
    """The small configuration (one 512x512 Julia frame, C = -0.8+0.156i,
    [-2,2]^2, binary32, limit 100, uint8 counts + RGBA8): the latency of one
    render call, and the sustained rate of 1,024 such frames as one batch plan."""
    import torch

    import paper_1611_03079_b300 as jl
    from paper_1611_03079_b300 import workloads as wl
    f = wl.single_frame()
    out = jl.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], count_type="u8")
    torch.cuda.synchronize()
    iters = float(out["counts"].double().sum())
    for _ in range(W):
        jl.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], count_type="u8", out=out)
    reps = 50 * K
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        jl.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], count_type="u8", out=out)
    e1.record()
    torch.cuda.synchronize()
    t1 = e0.elapsed_time(e1) * 1e-3 / reps
    nb = 1024
    b = jl.Batch([dict(f) for _ in range(nb)], tune=True)
    for _ in range(W):
        b.launch()
    e0.record()
    for _ in range(K):
        b.launch()
    e1.record()
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) * 1e-3 / K
    b.close()
    return {"W": f["W"], "H": f["H"], "max_iter": f["max_iter"], "mean_count": iters / (f["W"] * f["H"]),
            "one_render_ms": t1 * 1e3, "one_render_giter_s": iters / t1 / 1e9,
            "one_render_frac": 8 * iters / t1 / peak32,
            "batch_frames": nb, "batch_ms": tb * 1e3, "batch_giter_s": nb * iters / tb / 1e9,
            "batch_frac": 8 * nb * iters / tb / peak32,
            "note": "one render is launch-bound (a few microseconds of work); the batch is the sustained rate"}


def run_path_animation(K, W):
    """720-frame path animation (C(t) = 0.7885 exp(it), three resolutions,
    limit 100, RGBA8) as one batch plan: one CUDA-graph launch per step."""
    import torch

    import paper_1611_03079_b300 as jl
    from paper_1611_03079_b300 import workloads as wl
    frames = wl.path_animation()
    # iteration count from the histogram bins of a separate plan (not timed)
    hframes = [dict(f, hist=True, rgba=False) for f in frames]
    hb = jl.Batch(hframes)
    hb.launch()
    torch.cuda.synchronize()
    bins = torch.arange(101, dtype=torch.float64, device="cuda")
    iters = sum(float((hb.hist(i).double() * bins).sum()) * f["W"] * f["H"] for i, f in enumerate(frames))
    hb.close()
    # the plan picks its kernel by timing candidates on these frames (autotuned
    # for this workload, whatever the limit-100 bucket of the sweep chose)
    b = jl.Batch(frames, palette=wl.random_palette(7), tune=True)
    for _ in range(W):
        b.launch()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        b.launch()
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3 / K
    pix = sum(f["W"] * f["H"] for f in frames)
    res = {"frames": len(frames), "pixels": pix, "iterations": iters, "ms": t * 1e3, "frames_per_s": len(frames) / t,
           "giter_s": iters / t / 1e9, "gpixel_s": pix / t / 1e9, "graph_launches_per_step": 1,
           "status": b.status()}
    b.close()
    return res


def run_deep_zoom(K, W):
    """64 deep-zoom frames (1920x1080, limit 2000, precision chosen per frame)
    as one batch plan; plus the binary32-vs-binary64 count mismatch rate of
    every frame (forced renders of both)."""
    import numpy as np
    import torch

    import paper_1611_03079_b300 as jl
    from paper_1611_03079_b300 import workloads as wl
    frames = wl.deep_zoom()
    for f in frames:
        f["rgba"] = False
    b = jl.Batch(frames)
    for _ in range(W):
        b.launch()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        b.launch()
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3 / K
    iters = sum(float((b.counts(i).to(torch.int32) & 0xFFFF).sum()) for i in range(len(frames)))
    precs = b.precisions()
    rates = []
    for f in frames:
        c = {}
        for p in (0, 1):
            r = jl.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=p, count_type="u16", rgba=False)
            c[p] = r["counts"].view(torch.int16)
        rates.append(float((c[0] != c[1]).float().mean()))
    res = {"frames": len(frames), "ms": t * 1e3, "giter_s": iters / t / 1e9, "iterations": iters,
           "fp64_frames": int(sum(precs)), "fp32_frames": int(len(precs) - sum(precs)),
           "mismatch_rate_fp32_vs_fp64": {"per_frame": [round(x, 6) for x in rates],
                                          "auto_fp32_frames_max": max([r for r, p in zip(rates, precs) if p == 0],
                                                                      default=0.0),
                                          "auto_fp64_frames_mean": float(np.mean([r for r, p in zip(rates, precs)
                                                                                  if p == 1] or [0.0]))}}
    b.close()
    return res


def run_fig1_sweep():
    """Fig. 1 of the paper on this machine: square images of 10 .. 10,000
    pixels per side (Julia C = -0.8+0.156i over [-2,2]^2, limit 100,
    binary32; display excluded), GPU (jl_render, CUDA events, best of 3)
    against the sequential CPU oracle (one host thread) and the oracle on all
    host cores."""
    import torch

    import oracle
    import paper_1611_03079_b300 as jl
    rows = []
    for n in (10, 32, 100, 316, 1000, 3162, 10000):
        out = None
        best = float("inf")
        for r in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = jl.render(complex(-0.8, 0.156), (-2.0, 2.0, -2.0, 2.0), n, n, 100, precision="fp32",
                            count_type="u16", rgba=True, out=out)
            e1.record()
            torch.cuda.synchronize()
            if r:
                best = min(best, e0.elapsed_time(e1))
        t0 = time.perf_counter()
        oracle.render(complex(-0.8, 0.156), (-2.0, 2.0, -2.0, 2.0), n, n, 100, threads=1)
        t1 = time.perf_counter()
        oracle.render(complex(-0.8, 0.156), (-2.0, 2.0, -2.0, 2.0), n, n, 100)
        t2 = time.perf_counter()
        rows.append({"side": n, "gpu_ms": best, "cpu_1thread_ms": (t1 - t0) * 1e3,
                     "cpu_all_cores_ms": (t2 - t1) * 1e3})
    return rows


def map_ops_per_iteration(m):
    """Algorithmic IEEE operations of one step of a generic map (escape test
    included; a division counts as one operation although the hardware
    sequence is longer).  Z^2 + C gives 8, as for the quadratic path."""
    if m["kind"] == "power":
        d = int(m["degree"])
        top = d.bit_length() - 1
        return 3 + 3 + 5 * (top - 1) + 6 * (bin(d).count("1") - 1) + 2
    nd, nq = len(m["num"]) - 1, len(m["den"]) - 1
    # test 3; Horner 8 per degree (complex product 6, coefficient 2);
    # quotient 11 (|Q|^2 3, two numerators 3 + 3, two divisions); + C 2
    return 3 + 8 * (nd + nq) + 11 + 2


def run_generic_maps(K, W, peaks):
    """Generic maps (Sec. 2 other functions, Fig. 4): Multibrot parameter
    planes d = 3, 4, 5, 8, Fig. 4's map as printed, and the d = 3 plane in
    binary64, each 4096 x 4096 (uint16 counts + RGBA8) through jl_render_map;
    CUDA events around K renders after W warm-ups (queued behind a GPU sleep so
    that they run back to back), median of three such windows.  The oracle is timed on a
    64-row band of each frame on all host cores for context."""
    import numpy as np
    import torch

    import oracle
    import paper_1611_03079_b300 as jl
    from paper_1611_03079_b300 import workloads as wl
    rows = []
    for f in wl.map_sweep(4096):
        prec = "fp64" if f["precision"] else "fp32"
        mode = "mandelbrot" if f["mode"] else "julia"
        out = None
        for _ in range(W):
            out = jl.render_map(f["map"], f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=prec,
                                mode=mode, out=out)
        # median of three windows of K renders.  A render is a few hundred
        # microseconds of device work, about as long as the Python call that
        # launches it, so each window's renders are queued behind a fixed-length
        # GPU sleep and then run back to back: the events time the device.
        windows = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda._sleep(int(4e6 * K))
            e0.record()
            for _ in range(K):
                out = jl.render_map(f["map"], f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=prec,
                                    mode=mode, out=out)
            e1.record()
            torch.cuda.synchronize()
            windows.append(e0.elapsed_time(e1) / K)
        ms = statistics.median(windows)
        iters = int((out["counts"].view(torch.int16).to(torch.int32) & 0xFFFF).to(torch.int64).sum().item())
        ops = map_ops_per_iteration(f["map"])
        achieved = iters * ops / (ms * 1e-3)
        # oracle on a central band of 64 rows
        xmin, xmax, ymin, ymax = f["rect"]
        dy = (ymax - ymin) / f["H"]
        j0 = f["H"] // 2 - 32
        band = (xmin, xmax, ymin + j0 * dy, ymin + (j0 + 64) * dy)
        t0 = time.perf_counter()
        ref = oracle.render_map(f["map"], f["c"], band, f["W"], 64, f["max_iter"], f["mode"], f["precision"])
        cpu_s = time.perf_counter() - t0
        name = ("d=%d parameter plane" % f["map"]["degree"]) if f["map"]["kind"] == "power" else \
            "Fig. 4 map as printed, Julia C=%s" % f["c"]
        rows.append({"map": name, "precision": "binary64" if f["precision"] else "binary32",
                     "W": f["W"], "H": f["H"], "max_iter": f["max_iter"], "ms": ms, "iterations": iters,
                     "giter_s": iters / (ms * 1e-3) / 1e9, "ops_per_iteration": ops,
                     "achieved_gops": achieved / 1e9, "peak_gops": peaks[f["precision"]] / 1e9,
                     "frac": achieved / peaks[f["precision"]],
                     "cpu_band_giter_s": float(ref.astype(np.int64).sum()) / cpu_s / 1e9,
                     "cpu_cores": os.cpu_count()})
    return rows


def run_reference(args):
    world, rank, _ = dist_setup("gloo")
    if rank != 0:
        return
    from paper_1611_03079_b300 import workloads as wl
    frames = wl.throughput_sweep(args.size)
    for _ in range(args.warmup):
        cpu_sample(frames)
    vals = []
    t_all = time.perf_counter()
    desc = cores = None
    for _ in range(args.steps):
        v, cores, desc, _, _ = cpu_sample(frames)
        vals.append(v)
    wall = time.perf_counter() - t_all
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "impl": "CPU oracle (plain C, -O2 -ffp-contract=off)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_1611_03079_b300 as jl
    from paper_1611_03079_b300 import _lib, workloads as wl

    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = _lib.lib()
    stream = torch.cuda.current_stream()

    frames = wl.throughput_sweep(args.size)
    pal = wl.random_palette(7)
    # binary32 / binary64 issue peaks on this GPU (outside the timed region)
    import ctypes
    # The binary32 denominator is the larger of the scalar FMUL/FADD rate and
    # the packed add/mul.rn.f32x2 rate (separately rounded operations either way).
    probes = {}
    for kind, iters in ((0, 200000), (1, 4000), (2, 200000)):
        ops = ctypes.c_double(0)
        secs = ctypes.c_double(0)
        _lib.check(L.jl_probe_peak(kind, iters, ctypes.byref(ops), ctypes.byref(secs), stream.cuda_stream))
        probes[kind] = ops.value
    peaks = {0: max(probes[0], probes[2]), 1: probes[1]}

    # launch-shape autotuning (one-off, before any timing): per precision and
    # limit bucket, calibrated on the sweep frames themselves
    tuned = {}
    if args.tune_load:
        jl.tune_load(args.tune_load)
    for prec in (0, 1):
        for mi in (100, 1000):
            if args.tune_load:
                r = jl.tune_get("fp64" if prec else "fp32", mi)
            else:
                calib = [f for f in frames if f["precision"] == prec and f["max_iter"] == mi]
                r = jl.autotune("fp64" if prec else "fp32", mi, calib=calib, reps=1)
            tuned["%s limit %d" % ("binary64" if prec else "binary32", mi)] = {
                k: r[k] for k in ("ppt", "unroll", "threads", "ms", "candidates")}
    if args.tune_save:
        jl.tune_save(args.tune_save)

    # The sweep as one batch plan: one CUDA-graph launch per step renders all
    # 16 frames (coordinate tables, binary32 and binary64 persistent kernels on
    # concurrent branches).  Separate plans of the binary32 and of the binary64
    # frames give the per-precision breakdown.
    for f in frames:
        f["count_type"], f["rgba"] = "u16", True
    # The plan also times candidate kernels on its own launch (the tuner's
    # single-frame calibration can misjudge a concurrent multi-frame launch);
    # the per-precision plans use the kernels it chose.
    plan = jl.Batch(frames, palette=pal, tune=True)
    sub = {p: [i for i in range(len(frames)) if frames[i]["precision"] == p] for p in (0, 1)}
    chosen = {"fp32": plan.variant(0), "fp64": plan.variant(1)}
    W_ = max(args.warmup, 3)
    for _ in range(W_):
        plan.launch()
    torch.cuda.synchronize()
    iters = [int((plan.counts(i).to(torch.int32) & 0xFFFF).to(torch.int64).sum().item()) for i in range(len(frames))]

    n = len(frames)
    K = args.steps
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    t_start.record(stream)
    for s in range(K):
        plan.launch(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    total_ms = t_start.elapsed_time(t_end)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    total_iters = sum(iters)
    value = world * K * total_iters / (total_ms * 1e-3) / 1e9

    # per-precision breakdown and rooflines (ALU bound): each precision's frames
    # as a plan of their own, with timing events recorded inside its graph
    # around each kernel (binary64: the certified binary32 pass, then the
    # binary64 kernel on the pixels it left)
    by_prec, kern = {}, {}
    for prec in (0, 1):
        sp = jl.Batch([frames[i] for i in sub[prec]], palette=pal, variants=chosen, phases=True)
        for _ in range(2):
            sp.launch(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            sp.launch(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3 / K
        ph = []
        for _ in range(K):
            sp.launch(stream)
            torch.cuda.synchronize()
            ph.append(sp.phase_ms())
        ph = [statistics.mean(v[k] for v in ph) for k in range(4)]
        it = sum(iters[i] for i in sub[prec])
        px = sum(frames[i]["W"] * frames[i]["H"] for i in sub[prec])
        ops = OPS_PER_ITER * it / t
        by_prec[prec] = {"giter_s": it / t / 1e9, "time_ms": t * 1e3, "iterations": it,
                         "achieved_gops": ops / 1e9, "peak_gops": peaks[prec] / 1e9, "frac": ops / peaks[prec],
                         "frames": len(sub[prec]), "kernel_ms": ph}
        if prec == 0:
            kern["escape_compact_kernel" if chosen["fp32"][0] == 0 and chosen["fp32"][1] > 0 else
                 "escape_kernel<float>"] = dict(ms=ph[0], ops=OPS_PER_ITER * it, peak=peaks[0], prec="binary32",
                                                bytes=6 * px, unit_note="8 binary32 lane ops per iteration")
        elif ph[1] > 0:
            l32, l64, it_df, it64, st32, st_df = sp.cert_stats(stream)
            by_prec[prec]["frac_note"] = (
                "8 binary64 ops per iteration over the binary64 issue rate; above 1 because the certified "
                "binary32 and double-float passes settle %.1f %% of these iterations on the binary32 pipe "
                "(bit-exact binary64 counts); per-kernel fractions in roofline / roofline_other_kernels"
                % (100.0 * (it - it64) / max(it, 1)))
            by_prec[prec].update({"cert_listed_binary32_pass": l32, "cert_listed_to_binary64": l64,
                                  "iterations_settled_double_float": it_df, "iterations_binary64": it64,
                                  "tests_binary32_pass": st32, "tests_double_float_pass": st_df})
            kern["cert_kernel"] = dict(
                ms=ph[1], ops=CERT_OPS * st32, peak=peaks[0], prec="binary32",
                bytes=6 * (px - l32) + 8 * l32,
                unit_note="%d binary32 lane ops per test the certified binary32 pass decides (%d tests: every "
                          "binary64 pixel's tests up to its escape, its limit or its unsettled test): the orbit "
                          "step y*y, fma(x,x,y2), fma(-y,y,cr), fma(x,x,.), x+x, fma(2x,y,ci) and the bound update "
                          "fma(2s',E), fma(E,.,EC), fma(2.5u,r,.); the test's fma(r,.,.) is formed once per block "
                          "of 6 steps where |C32| lies outside [1.9975, 2.0025] (every sweep pixel) and is not "
                          "counted, nor are the approximate square root (XU pipe) and the compare; it settles %d "
                          "of the %d binary64 iterations" % (CERT_OPS, st32, it - it_df - it64, it))
            if ph[2] > 0:
                kern["cert2_kernel"] = dict(
                    ms=ph[2], ops=CERT2_OPS * st_df, peak=peaks[0], prec="binary32",
                    bytes=8 * l32 + 6 * (l32 - l64) + 8 * l64,
                    unit_note="%d binary32 lane ops per test the double-float pass decides (%d tests of the %d "
                              "pixels the binary32 pass lists): the test on the high parts (7), the float-pair "
                              "step with exact product splits (6), three TwoSums (18), the low parts (14), two "
                              "renormalising TwoSums (12) and the bound (5); it settles %d iterations"
                              % (CERT2_OPS, st_df, l32, it_df))
            kern["escape_kernel<double> (list)"] = dict(
                ms=ph[3], ops=OPS_PER_ITER * it64, peak=peaks[1], prec="binary64", bytes=14 * l64,
                unit_note="8 binary64 lane ops per iteration of the listed pixels; the kernel issues 6 of them "
                          "on the FP64 pipe: x+x is an exponent increment on the integer pipe and the escape "
                          "test is estimated in binary32 (exact binary64 replay near the threshold)")
        else:
            kern["escape_kernel<double>"] = dict(ms=ph[3], ops=OPS_PER_ITER * it, peak=peaks[1], prec="binary64",
                                                 bytes=6 * px, unit_note="8 binary64 lane ops per iteration")
        sp.close()
    for k, v in kern.items():
        v["achieved"] = v["ops"] / (v["ms"] * 1e-3) / 1e9
        v["frac"] = v["achieved"] * 1e9 / v["peak"]
    dom_k = max(kern, key=lambda k: kern[k]["ms"])
    d = kern[dom_k]
    # DRAM bytes (read + write) per launch of each kernel, from one ncu capture
    # of the same plan launch (profiles/escape_kernel_sweep4096.md)
    traffic = {"cert_kernel": 65916160 + 786704384, "cert2_kernel": 82806784 + 149423360,
               "escape_kernel<double> (list)": 7740672 + 4626432,
               "escape_compact_kernel": 30964992 + 780568320} if args.size == 4096 else {}
    roofline = {"bound": "alu", "kernel": dom_k, "precision": d["prec"],
                "achieved": d["achieved"], "peak": d["peak"] / 1e9, "unit": "Gop/s", "frac": d["frac"],
                "traffic": traffic.get(dom_k),
                "traffic_note": "bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture "
                                "of this plan launch, profiles/escape_kernel_sweep4096.md); algorithmic bytes per "
                                "launch: %d (uint16 count + RGBA8 per pixel it stores, 8 B per list entry)"
                                % d["bytes"],
                "peak_source": "measured on this GPU by jl_probe_peak (independent multiply/add chains, no FMA; "
                               "binary32: the larger of scalar FMUL/FADD, %.0f G lane-ops/s, and packed "
                               "add/mul.f32x2, %.0f)" % (probes[0] / 1e9, probes[2] / 1e9),
                "algorithmic_unit": d["unit_note"] + " (x*x, y*y, x+x, (x+x)*y, +ci, x2-y2, +cr, x2+y2)",
                "ms_per_launch": d["ms"],
                "timing": "CUDA events recorded inside the graph around this kernel, plan of the %s sweep "
                          "frames alone, mean of %d synchronised launches" % (d["prec"], K)}
    roofline_other = [{"kernel": k, "precision": v["prec"], "achieved": v["achieved"], "peak": v["peak"] / 1e9,
                       "unit": "Gop/s", "frac": v["frac"], "ms_per_launch": v["ms"], "traffic": traffic.get(k),
                       "algorithmic_unit": v["unit_note"]} for k, v in kern.items() if k != dom_k]

    e2e = None
    if not args.no_e2e and rank == 0:
        # the public host-output path: jl_render_frames_to_host renders the 16
        # frames into pinned host memory, copies overlapped with rendering
        hf = jl.HostFrames([dict(f, count_type="u16", rgba=True) for f in frames], palette=pal, depth=0)
        hf.render(stream)  # warm-up
        times = []
        for _ in range(max(K, 1)):
            t0 = time.perf_counter()
            hf.render(stream)
            times.append(time.perf_counter() - t0)
        e2e_s = statistics.median(times)
        ok = all(np.array_equal(hf.counts(i), plan.counts(i).cpu().numpy().view(np.uint16)) and
                 np.array_equal(hf.rgba(i), plan.rgba(i).cpu().numpy()) for i in range(len(frames)))
        e2e = {"value": total_iters / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": 96 * n,
               "d2h_bytes_per_step": int(hf.d2h_bytes), "ms_per_step": e2e_s * 1e3, "steps": len(times),
               "outputs_match_device_plan": bool(ok),
               "launches_per_step": hf.launches(),
               "note": "host plan (jl_host_plan_run): per step, each frame's coordinate tables are computed "
                       "from its description (step A1), then the 16 frames render on 4 internal render "
                       "streams into one device slot each (the last frame as 4 row bands) and are copied to "
                       "pinned host memory (counts + RGBA8) on 2 copy streams as each frame (band) finishes; "
                       "host wall clock per call (median of steps), the call returns after the last copy; "
                       "h2d = the 16 frame descriptions (96 B each), which reach the device as kernel "
                       "parameters of the coordinate and escape launches (no separate copy); the host "
                       "outputs equal the device plan's byte for byte"}

    cpu = None
    if not args.no_cpu and rank == 0:
        # the reference arm itself, in a fresh process (the same code and
        # sample; in this process torch's host threads would compete with
        # the oracle's for the cores)
        env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", "3",
                              "--warmup", "1", "--size", str(args.size)], capture_output=True, text=True, env=env,
                             check=True).stdout
        ref = json.loads(out.strip().splitlines()[-1])
        cpu = dict(ref["cpu_baseline"])
        cpu["sample"] += "; mean of 3 timed runs after 1 warm-up, in a separate process (bench.py --impl reference)"

    # binary32-vs-binary64 count mismatch of the sweep frames (same frame, both precisions)
    mismatch = {}
    for i in range(n):
        f = frames[i]
        if f["precision"] != 0:
            continue
        j = next(jj for jj in range(n) if frames[jj]["precision"] == 1 and frames[jj]["c"] == f["c"] and
                 frames[jj]["max_iter"] == f["max_iter"] and frames[jj]["mode"] == f["mode"])
        key = "%s %s limit %d" % ("mandelbrot" if f["mode"] else "julia", f["c"], f["max_iter"])
        a16, b16 = plan.counts(i), plan.counts(j)
        mismatch[key] = float((a16 != b16).float().mean())

    extra = {}
    if not args.no_extra and rank == 0:
        extra["single_frame_512"] = run_single_frame(K, max(args.warmup, 3), peaks[0])
        extra["path_animation"] = run_path_animation(K, max(args.warmup, 3))
        extra["deep_zoom"] = run_deep_zoom(1, 1)
        extra["fig1_size_sweep"] = run_fig1_sweep()
        extra["generic_maps"] = run_generic_maps(K, max(args.warmup, 3), peaks)

    survey = None
    if not args.no_survey and rank == 0:
        survey = run_survey(args, K, max(args.warmup, 3))
        try:
            peaks_file = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
            pk = float(peaks_file["bf16_tflops"])
            src = "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
        except (OSError, KeyError, ValueError):
            pk, src = 1800.0, "fallback 1.8 PFLOP/s"
        survey["roofline_forward"].update({"peak": pk, "frac": survey["roofline_forward"]["achieved"] / pk,
                                           "peak_source": src})
        try:
            pks = float(peaks_file["bf16_tflops_sustained"])
            srcs = "measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
        except (NameError, KeyError, ValueError):
            pks, srcs = 1400.0, "fallback 1.4 PFLOP/s sustained"
        survey["roofline_training"].update({"peak": pks, "frac": survey["roofline_training"]["achieved"] / pks,
                                            "peak_source": srcs})

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": max(args.warmup, 3), "ms_per_step": total_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "frames_per_step": n, "pixels_per_step": sum(
                    f["W"] * f["H"] for f in frames), "iterations_per_step": total_iters,
                    "l2": "outputs are 1.6 GB per step, larger than the 126 MB L2; no flush needed",
                    "parallelism": "replicas" if world > 1 else "single GPU"},
                "survey_summary": None if survey is None else {
                    k: survey[k] for k in ("screened_per_s", "speedup_vs_plain_render", "judge_l1_mean",
                                           "l1_target_met", "heldout_l1_mean", "train_s")},
                "roofline_training": None if survey is None else survey["roofline_training"],
                "roofline": roofline, "roofline_other_kernels": roofline_other,
                "by_precision": {("binary64" if p else "binary32"): by_prec[p] for p in (0, 1)},
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": (6 if chosen["fp64"][0] > 0 else 4) * K,
                "gpu_launches_note": "one CUDA-graph launch per step holding %d kernels of this library "
                                     "(coordinate tables of each precision group, the binary32 escape kernel%s)"
                                     % (6 if chosen["fp64"][0] > 0 else 4,
                                        ", the certified binary32 and double-float passes of the binary64 frames "
                                        "and the binary64 kernel on the pixels they list" if chosen["fp64"][0] > 0
                                        else ", the binary64 escape kernel"),
                "autotuned_variants": tuned,
                "plan_variants": {k: list(v) for k, v in chosen.items()},
                "survey": survey,
                "mismatch_rate_fp32_vs_fp64_sweep": mismatch,
                **extra,
                "peaks_gops": {"binary32": peaks[0] / 1e9, "binary64": peaks[1] / 1e9,
                               "binary32_scalar_fmul_fadd": probes[0] / 1e9,
                               "binary32_packed_add_mul": probes[2] / 1e9}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
