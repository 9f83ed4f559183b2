"""Command-line renderer (through the C ABI).

  python -m paper_1611_03079_b300.cli --workload sweep --index 13 --size 2048 --repeat 3
  python -m paper_1611_03079_b300.cli --c -0.8+0.156j --rect -2 2 -2 2 --W 512 --H 512 --out f.npy
  python -m paper_1611_03079_b300.cli --workload forward --n 1048576 --repeat 3
  python -m paper_1611_03079_b300.cli --workload sweep-plan --precision fp64 --repeat 3
  python -m paper_1611_03079_b300.cli --workload train --epochs 2

Renders one frame `repeat` times on cuda:0 and prints the kernel-bracketed
time and pixel-iterations per second; optionally saves counts (.npy).  Also
used as the small, self-contained command that profiles are taken on.
"""
import argparse
import json

import numpy as np


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--workload", choices=["sweep", "sweep-plan", "single", "path", "forward", "train"], default=None)
    p.add_argument("--epochs", type=int, default=2, help="train workload: epochs over 65,536 seeded C values")
    p.add_argument("--n", type=int, default=1 << 20, help="forward workload: number of C values screened")
    p.add_argument("--frames", type=int, default=72, help="path workload: first N frames as one batch plan")
    p.add_argument("--index", type=int, default=0)
    p.add_argument("--size", type=int, default=4096)
    p.add_argument("--c", type=complex, default=complex(-0.8, 0.156))
    p.add_argument("--rect", type=float, nargs=4, default=[-2.0, 2.0, -2.0, 2.0])
    p.add_argument("--W", type=int, default=512)
    p.add_argument("--H", type=int, default=512)
    p.add_argument("--max-iter", type=int, default=100)
    p.add_argument("--precision", default="fp32")
    p.add_argument("--mode", default="julia")
    p.add_argument("--repeat", type=int, default=1)
    p.add_argument("--variant", type=int, nargs="+", default=None, help="ppt unroll threads ctas_per_sm")
    p.add_argument("--out", default=None)
    p.add_argument("--probe", action="store_true", help="print the issue-rate probes and exit")
    a = p.parse_args(argv)
    if a.probe:
        return probe()

    import torch

    import paper_1611_03079_b300 as jl
    from paper_1611_03079_b300 import workloads as wl

    if a.workload == "path":
        return path(a)
    if a.workload == "forward":
        return forward(a)
    if a.workload == "sweep-plan":
        return sweep_plan(a)
    if a.workload == "train":
        return train(a)
    if a.workload == "sweep":
        f = wl.throughput_sweep(a.size)[a.index]
    elif a.workload == "single":
        f = wl.single_frame()
    else:
        f = dict(c=a.c, rect=tuple(a.rect), W=a.W, H=a.H, max_iter=a.max_iter,
                 precision={"fp32": 0, "fp64": 1, "auto": 2}[a.precision],
                 mode={"julia": 0, "mandelbrot": 1}[a.mode])
    torch.cuda.set_device(0)
    out = None
    times = []
    for _ in range(a.repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = jl.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=f["precision"],
                        mode=f["mode"], count_type="u16", rgba=True, out=out, variant=a.variant)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    iters = int(out["counts"].to(torch.int64).sum().item())
    best = min(times)
    print(json.dumps({"frame": {k: (str(v) if k == "c" else v) for k, v in f.items()}, "ms": times,
                      "best_ms": best, "giter_s": iters / (best * 1e-3) / 1e9, "iterations": iters}))
    if a.out:
        np.save(a.out, out["counts"].view(torch.int16).cpu().numpy().view(np.uint16))


def sweep_plan(a):
    """The throughput-sweep frames of one precision (--precision fp32 / fp64)
    as one batch plan with uint16 counts and RGBA8, launched `repeat` times:
    the launch whose kernel the benchmark's roofline reports."""
    import torch

    import paper_1611_03079_b300 as jl
    from paper_1611_03079_b300 import workloads as wl
    torch.cuda.set_device(0)
    prec = {"fp32": 0, "fp64": 1}[a.precision]
    frames = [dict(f, count_type="u16", rgba=True) for f in wl.throughput_sweep(a.size) if f["precision"] == prec]
    variants = {a.precision: tuple(a.variant)} if a.variant else None
    b = jl.Batch(frames, palette=wl.random_palette(7), variants=variants)
    times = []
    for _ in range(a.repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.launch()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    iters = sum(int((b.counts(i).to(torch.int32) & 0xFFFF).to(torch.int64).sum().item()) for i in range(len(frames)))
    pix = sum(f["W"] * f["H"] for f in frames)
    print(json.dumps({"frames": len(frames), "pixels": pix, "output_bytes": 6 * pix, "iterations": iters,
                      "ms": times, "best_ms": min(times), "giter_s": iters / (min(times) * 1e-3) / 1e9,
                      "variant": list(b.variant(prec)), "status": b.status(),
                      "cert_stats": list(b.cert_stats())}))
    b.close()


def path(a):
    """First N frames of the path animation as one batch plan, launched
    `repeat` times (RGBA8 only)."""
    import torch

    import paper_1611_03079_b300 as jl
    from paper_1611_03079_b300 import workloads as wl
    torch.cuda.set_device(0)
    frames = wl.path_animation()[:a.frames]
    variants = {"fp32": tuple(a.variant[:3])} if a.variant else None
    b = jl.Batch(frames, variants=variants)
    times = []
    for _ in range(a.repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.launch()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    pix = sum(f["W"] * f["H"] for f in frames)
    print(json.dumps({"frames": len(frames), "pixels": pix, "ms": times, "gpixel_s": pix / (min(times) * 1e-3) / 1e9,
                      "status": b.status()}))
    b.close()


def forward(a):
    """The fused surrogate forward (entropy scores only) over n seeded C
    values, with a seeded random-init network, `repeat` times."""
    import torch

    from paper_1611_03079_b300 import surrogate, workloads as wl
    torch.cuda.set_device(0)
    model = surrogate.Surrogate(wl.fourier_matrix(), wl.mlp_init())
    c = torch.from_numpy(wl.survey_candidates(a.n)).cuda()
    times = []
    for _ in range(a.repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, score = model.forward(c, probs=False, score=True)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    flop = 215552.0 * a.n
    best = min(times)
    print(json.dumps({"n": a.n, "ms": times, "best_ms": best, "tflop_s": flop / (best * 1e-3) / 1e12,
                      "mean_score": float(score.mean().item())}))
    model.close()


def train(a):
    """Surrogate training (batch 1024, Adam) on the 65,536 seeded training C
    values with seeded random target histograms (the products and kernels of
    a training step, without rendering the targets), `epochs` epochs."""
    import time

    import torch

    from paper_1611_03079_b300 import surrogate, workloads as wl
    torch.cuda.set_device(0)
    c = torch.from_numpy(wl.survey_train()).cuda()
    g = torch.Generator(device="cpu").manual_seed(5)
    t = torch.rand((c.shape[0], 101), generator=g).cuda()
    t = t / t.sum(1, keepdim=True)
    model = surrogate.Surrogate(wl.fourier_matrix(), wl.mlp_init())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    curve = model.train(c, t, a.epochs, batch=1024, lr=2e-3, lr_final=1e-5, order_seed=1)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    steps = a.epochs * (c.shape[0] // 1024)
    print(json.dumps({"epochs": a.epochs, "steps": steps, "s": secs, "ms_per_step": secs / steps * 1e3,
                      "final_loss": float(curve[-1])}))
    model.close()


def probe():
    import ctypes

    import torch

    from paper_1611_03079_b300 import _lib
    torch.cuda.set_device(0)
    L = _lib.lib()
    names = {0: "binary32 fmul+fadd", 1: "binary64 dmul+dadd", 2: "binary32x2 packed add / mul chains"}
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    res = {}
    for kind, iters in ((0, 200000), (1, 4000), (2, 200000)):
        ops, secs = ctypes.c_double(0), ctypes.c_double(0)
        _lib.check(L.jl_probe_peak(kind, iters, ctypes.byref(ops), ctypes.byref(secs), None))
        res[names[kind]] = {"G_lane_ops_s": ops.value / 1e9, "ms": secs.value * 1e3,
                            "lane_ops_per_clk_per_sm_at_2032MHz": ops.value / (sms * 2.032e9)}
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
