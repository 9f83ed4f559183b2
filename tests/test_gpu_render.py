"""GPU parity of jl_render against the CPU oracle: escape counts bit-exact in
the same working precision, RGBA8 and histograms byte/bit-exact (Sec. 2
escape time and colour levels; Sec. 3 Mandelbrot mode and deep zoom).

All calls go through the C ABI (libjl.so via the ctypes binding)."""
import numpy as np
import pytest

import oracle
import paper_1611_03079_b300 as jl
from paper_1611_03079_b300 import workloads as wl

pytestmark = pytest.mark.gpu

PAL = wl.random_palette(7)


def gpu_render(f, variant=None, count_type=None, rgba=True, hist=False, palette=PAL):
    import torch
    ct = count_type or f.get("count_type") or "u16"
    out = jl.render(f.get("c"), f["rect"], f["W"], f["H"], f["max_iter"], precision=f["precision"],
                    mode=f["mode"], count_type=ct, rgba=rgba, hist=hist, palette=palette, variant=variant)
    torch.cuda.synchronize()
    res = {}
    if "counts" in out:
        res["counts"] = out["counts"].cpu().numpy().astype(np.uint16) if ct == "u8" else \
            out["counts"].view(torch.int16).cpu().numpy().view(np.uint16)
    if "rgba" in out:
        res["rgba"] = out["rgba"].cpu().numpy()
    if "hist" in out:
        res["hist"] = out["hist"].cpu().numpy()
    return res


def oracle_render(f, prec=None):
    p = f["precision"] if prec is None else prec
    if p == wl.AUTO:
        p = oracle.precision_for_view(f["rect"], f["W"], f["H"])
    return oracle.render(f.get("c"), f["rect"], f["W"], f["H"], f["max_iter"], f["mode"], p)


def check_frame(f, variant=None, hist=True):
    g = gpu_render(f, variant=variant, hist=hist)
    k = oracle_render(f)
    mism = int((g["counts"] != k).sum())
    assert mism == 0, "%d count mismatches (of %d) for %s variant=%s" % (mism, k.size, f, variant)
    assert (g["rgba"] == oracle.colour(k, f["max_iter"], PAL)).all()
    if hist:
        assert (g["hist"] == oracle.hist(k, f["max_iter"])).all()
    return k


def test_single_frame_workload(cuda):
    """512x512 Julia C = -0.8+0.156i, binary32, limit 100, uint8 counts."""
    f = wl.single_frame()
    g = gpu_render(f, count_type="u8", hist=True)
    k = oracle_render(f)
    assert (g["counts"] == k).all()
    assert (g["rgba"] == oracle.colour(k, 100, PAL)).all()
    assert (g["hist"] == oracle.hist(k, 100)).all()


@pytest.mark.parametrize("seed", range(6))
def test_random_views(cuda, seed):
    """Ragged sizes (1..97 per side, several chunks per row and a ragged tail),
    both modes, both precisions, limits from 1 to 300."""
    for f in wl.random_views(12, seed=100 + seed):
        check_frame(f)


@pytest.mark.parametrize("prec", [0, 1])
def test_every_variant(cuda, prec):
    import ctypes
    L = jl._lib.lib()
    n = L.jl_variant_list(prec, None, 0)
    buf = (ctypes.c_int32 * (2 * n))()
    L.jl_variant_list(prec, buf, n)
    frames = [dict(c=complex(-0.7269, 0.1889), rect=(-1.6, 1.6, -1.6, 1.6), W=333, H=211, max_iter=1000,
                   mode=0, precision=prec),
              dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=300, H=301, max_iter=300, mode=1, precision=prec)]
    for i in range(n):
        for threads in (128, 256):
            v = (buf[2 * i], buf[2 * i + 1], threads, 0)
            for f in frames:
                check_frame(f, variant=v, hist=False)


EDGE = [
    dict(c=0.3 + 0.5j, rect=(-2, 2, -2, 2), W=1, H=1, max_iter=100, mode=0, precision=0),
    dict(c=0.3 + 0.5j, rect=(-2, 2, -2, 2), W=1, H=777, max_iter=100, mode=0, precision=0),
    dict(c=0.3 + 0.5j, rect=(-2, 2, -2, 2), W=1031, H=1, max_iter=100, mode=0, precision=1),
    dict(c=-0.8 + 0.156j, rect=(-2, 2, -2, 2), W=64, H=64, max_iter=1, mode=0, precision=0),
    dict(c=-0.8 + 0.156j, rect=(-2, 2, -2, 2), W=64, H=64, max_iter=2, mode=1, precision=1),
    dict(c=-0.8 + 0.156j, rect=(-2, 2, -2, 2), W=64, H=64, max_iter=7, mode=0, precision=0),
    dict(c=0j, rect=(5, 6, 5, 6), W=40, H=30, max_iter=100, mode=0, precision=0),            # all count 0
    dict(c=0j, rect=(-0.1, 0.1, -0.1, 0.1), W=40, H=30, max_iter=500, mode=0, precision=0),  # all inside
    dict(c=-2 + 0j, rect=(-2.0, 2.0, -0.25, 0.25), W=1001, H=1, max_iter=300, mode=0, precision=0),
    dict(c=-2 + 0j, rect=(1.5, 2.5, -0.5, 0.5), W=1, H=1, max_iter=50, mode=0, precision=1),   # |Z|^2 == 4
    dict(c=2.5 + 0.1j, rect=(-2, 2, -2, 2), W=200, H=150, max_iter=100, mode=0, precision=0),  # |C| > 2
    dict(c=-1.9999 + 0j, rect=(-2, 2, -1, 1), W=300, H=150, max_iter=400, mode=0, precision=0),
    dict(c=None, rect=(-2.05, -1.95, -0.05, 0.05), W=257, H=129, max_iter=2000, mode=1, precision=0),
    dict(c=None, rect=(1.2, 2.2, 0.9, 1.9), W=256, H=256, max_iter=300, mode=1, precision=1),  # |C| ~ 2 band
    dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=700, H=700, max_iter=255, mode=1, precision=0),
    dict(c=0.285 + 0.01j, rect=(-1.6, 1.6, -1.6, 1.6), W=97, H=53, max_iter=65535, mode=0, precision=0),
    dict(c=-0.7269 + 0.1889j, rect=(-1.6, 1.6, -1.6, 1.6), W=300, H=300, max_iter=5000, mode=0, precision=1),
]


@pytest.mark.parametrize("idx", range(len(EDGE)))
def test_edge_cases(cuda, idx):
    check_frame(EDGE[idx])


def test_u8_counts_and_uint16_agree(cuda):
    f = dict(c=-0.4 + 0.6j, rect=(-1.6, 1.6, -1.6, 1.6), W=500, H=400, max_iter=255, mode=0, precision=0)
    a = gpu_render(f, count_type="u8")
    b = gpu_render(f, count_type="u16")
    assert (a["counts"] == b["counts"]).all()
    assert (a["counts"] == oracle_render(f)).all()


def test_auto_precision_deep_view(cuda):
    """AUTO picks binary64 for a 1e-9-wide view and the counts match the
    binary64 oracle."""
    z = wl.julia_boundary_points(complex(-0.7269, 0.1889), 1, seed=5)[0]
    w = 1e-9
    f = dict(c=complex(-0.7269, 0.1889), rect=(z.real - w / 2, z.real + w / 2, z.imag - w / 4, z.imag + w / 4),
             W=320, H=160, max_iter=2000, mode=0, precision=wl.AUTO)
    assert jl.select_precision(f["rect"], 320, 160) == jl.JL_FP64
    k = check_frame(f)
    assert (k == oracle_render(f, prec=oracle.FP64)).all()


def test_hist_global_bins(cuda):
    """max_iter + 1 > 4096 bins: histogram accumulated in global memory."""
    f = dict(c=-0.7269 + 0.1889j, rect=(-1.6, 1.6, -1.6, 1.6), W=256, H=256, max_iter=6000, mode=0, precision=0)
    check_frame(f, hist=True)


def test_render_to_host_matches(cuda):
    f = dict(c=-0.7269 + 0.1889j, rect=(-1.6, 1.6, -1.6, 1.6), W=640, H=480, max_iter=1000, mode=0,
             precision=0)
    h = jl.render_to_host(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=0, mode=0,
                          count_type="u16", rgba=True, hist=True, palette=PAL)
    g = gpu_render(f, hist=True)
    assert (h["counts"] == g["counts"]).all()
    assert (h["rgba"] == g["rgba"]).all()
    assert (h["hist"] == g["hist"]).all()


def test_deterministic(cuda):
    f = dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=1024, H=1024, max_iter=1000, mode=1, precision=0)
    a = gpu_render(f, hist=True)
    b = gpu_render(f, hist=True)
    for key in a:
        assert (a[key] == b[key]).all()


@pytest.fixture(scope="module")
def sweep_batch():
    """The 16 sweep frames (4096 x 4096) as one batch plan, exactly as
    bench.py launches them."""
    import torch
    frames = wl.throughput_sweep()
    for f in frames:
        f["count_type"], f["rgba"], f["hist"] = "u16", True, True
    b = jl.Batch(frames, palette=PAL)
    b.launch()
    torch.cuda.synchronize()
    yield frames, b
    b.close()


@pytest.mark.slow
@pytest.mark.parametrize("idx", range(16))
def test_throughput_sweep_full_size_sampled(cuda, sweep_batch, idx):
    """The 4096x4096 sweep frames in the benchmark's launch configuration (one
    batch plan): sampled rows (64 spread rows including the first and last)
    checked against the oracle row by row, plus full-frame invariants:
    180-degree symmetry of binary32 Julia frames (their grids are exactly
    antisymmetric), row symmetry of Mandelbrot frames, and histograms that
    recover the bin counts of the whole frame."""
    frames, b = sweep_batch
    f = frames[idx]
    c = b.counts(idx).cpu().numpy().view(np.uint16)
    rgba = b.rgba(idx).cpu().numpy()
    rows = sorted(set([0, f["H"] - 1] + list(range(37, f["H"], 64))))
    k = oracle.render_rows(f["c"], f["rect"], f["W"], f["H"], rows, f["max_iter"], f["mode"], f["precision"])
    assert (c[rows] == k).all()
    assert (rgba[rows] == oracle.colour(k, f["max_iter"], PAL)).all()
    if f["precision"] == 0:
        if f["mode"] == 0:
            assert (c == c[::-1, ::-1]).all()
        else:
            assert (c == c[::-1, :]).all()
    h = b.hist(idx).cpu().numpy().astype(np.float64)
    assert abs(h.sum() - 1.0) < 1e-4
    assert (np.rint(h * f["W"] * f["H"]) == np.bincount(c.ravel(), minlength=f["max_iter"] + 1)).all()


@pytest.mark.slow
def test_throughput_sweep_bench_outputs(cuda, sweep_batch):
    """The sweep as bench.py renders it (uint16 counts and RGBA8, no
    histograms, so the tile kernels take their store path without per-frame
    tests; a tuned plan, which times its candidate kernels on these frames
    and keeps the fastest) gives the same bytes as the plan above, whose
    counts are checked against the oracle."""
    import torch
    frames, b = sweep_batch
    bf = [dict(f, hist=False) for f in frames]
    b2 = jl.Batch(bf, palette=PAL, tune=True)
    b2.launch()
    torch.cuda.synchronize()
    for i in range(len(frames)):
        assert torch.equal(b2.counts(i), b.counts(i)), i
        assert torch.equal(b2.rgba(i), b.rgba(i)), i
    b2.close()


def test_integer_doubling_is_exact(cuda):
    """The binary64 kernels form x + x on the integer pipes; it must equal
    IEEE x + x bit for bit (zero, subnormals, carries into the exponent,
    overflow to infinity, infinities; NaN stays NaN)."""
    import torch
    rng = np.random.default_rng(0)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072009e-308, 2.2250738585072014e-308,
                        1.1125369292536007e-308, 8.98846567431158e307, 8.988465674311579e307,
                        1.7976931348623157e308, -1.7976931348623157e308, np.inf, -np.inf, 1.0, -2.0, 1e-310,
                        4.0, 2.0 - 2 ** -52])
    vals = np.concatenate([special, rng.standard_normal(4000) * 10.0 ** rng.uniform(-310, 308, 4000),
                           np.frombuffer(rng.bytes(8 * 4000), dtype=np.float64)])
    vals = vals[~np.isnan(vals)]
    x = torch.from_numpy(vals).cuda()
    y = torch.empty_like(x)
    jl._lib.check(jl._lib.lib().jl_selftest_double(x.data_ptr(), y.data_ptr(), x.numel(), None))
    torch.cuda.synchronize()
    with np.errstate(over="ignore"):
        ref = vals + vals
    assert (y.cpu().numpy().view(np.uint64) == ref.view(np.uint64)).all()
    z = torch.tensor([float("nan")], dtype=torch.float64, device="cuda")
    w = torch.empty_like(z)
    jl._lib.check(jl._lib.lib().jl_selftest_double(z.data_ptr(), w.data_ptr(), 1, None))
    torch.cuda.synchronize()
    assert torch.isnan(w).all()


@pytest.mark.parametrize("T", [8, 16])
def test_compact_kernel_frames(cuda, T):
    """The compacting tile kernel (binary32; stragglers parked in per-warp
    rings and resumed in full batches): bit-exact counts, colours and
    histograms on frames where many pixels are parked and resumed several
    times (limits up to 65535), on the edge cases and on ragged views."""
    v = (0, T, 256, 0)
    heavy = [dict(c=complex(-0.7269, 0.1889), rect=(-1.6, 1.6, -1.6, 1.6), W=517, H=389, max_iter=1000, mode=0,
                  precision=0),
             dict(c=complex(-0.4, 0.6), rect=(-1.6, 1.6, -1.6, 1.6), W=256, H=256, max_iter=5000, mode=0,
                  precision=0),
             dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=401, H=333, max_iter=1000, mode=1, precision=0),
             dict(c=None, rect=(-0.7530, -0.7490, 0.0990, 0.1030), W=64, H=40, max_iter=65535, mode=1,
                  precision=0)]
    for f in heavy:
        check_frame(f, variant=v, hist=f["max_iter"] <= 5000)
    for f in EDGE:
        if f["precision"] == 0:
            check_frame(f, variant=v)
    for f in wl.random_views(12, seed=300 + T):
        f = dict(f)
        f["precision"] = 0
        check_frame(f, variant=v)


# Julia frames with |C|^2 >= 3.99: the monotone-escape argument behind the
# blocked test does not cover them, so the binary64 kernels take their exact
# step-by-step branch for every pixel (and the binary32 kernels theirs).
UNSAFE_C = [
    dict(c=2.5 + 0.1j, rect=(-2.0, 2.0, -1.5, 1.5), W=480, H=360, max_iter=100),
    dict(c=-1.9999 + 0j, rect=(-2.0, 2.0, -1.0, 1.0), W=640, H=321, max_iter=1000),
    dict(c=-2 + 0j, rect=(-2.1, 2.1, -0.5, 0.5), W=640, H=161, max_iter=1000),
    dict(c=-2 + 0j, rect=(-2.0, 2.0, -0.25, 0.25), W=1001, H=1, max_iter=2000),     # the segment [-2, 2]
    dict(c=1.414 + 1.414j, rect=(-2.0, 2.0, -2.0, 2.0), W=512, H=512, max_iter=200),  # |C|^2 = 3.998792
    dict(c=-2.0001 + 0j, rect=(-2.1, 2.1, -1.0, 1.0), W=400, H=200, max_iter=5000),
    dict(c=2j, rect=(-1.6, 1.6, -1.6, 1.6), W=333, H=297, max_iter=1000),           # |C| = 2 exactly
]


@pytest.mark.parametrize("idx", range(len(UNSAFE_C)))
@pytest.mark.parametrize("prec", [1, 0])
def test_unsafe_band_full_views(cuda, idx, prec):
    """Full views of Julia sets with |C|^2 >= 3.99 in every kernel variant of
    the precision, bit-exact against the oracle (counts and colours; the
    histogram for the default variant)."""
    import ctypes
    f = dict(UNSAFE_C[idx], mode=0, precision=prec)
    k = oracle_render(f)
    L = jl._lib.lib()
    n = L.jl_variant_list(prec, None, 0)
    buf = (ctypes.c_int32 * (2 * n))()
    L.jl_variant_list(prec, buf, n)
    variants = [None] + [(buf[2 * i], buf[2 * i + 1], t, 0) for i in range(n) for t in (128, 256)]
    for v in variants:
        g = gpu_render(f, variant=v, hist=v is None)
        mism = int((g["counts"] != k).sum())
        assert mism == 0, "%d count mismatches (of %d), variant %s" % (mism, k.size, v)
        assert (g["rgba"] == oracle.colour(k, f["max_iter"], PAL)).all()
        if v is None:
            assert (g["hist"] == oracle.hist(k, f["max_iter"])).all()


@pytest.mark.parametrize("side", [10, 32, 100, 316, 1000, 3162, 10000])
def test_fig1_size_sweep_frames(cuda, side):
    """The square frames of the Fig. 1 size sweep (Julia C = -0.8+0.156i over
    [-2,2]^2, limit 100, binary32, uint16 + RGBA8) in the launch the bench
    times: whole frames up to 1000 per side; above that 32 rows (the first,
    the last, the middle and 29 seeded ones) against the oracle, plus the
    histogram of the whole frame against the GPU counts' own histogram."""
    f = dict(c=-0.8 + 0.156j, rect=(-2.0, 2.0, -2.0, 2.0), W=side, H=side, max_iter=100, mode=0, precision=0)
    if side <= 1000:
        check_frame(f)
        return
    g = gpu_render(f, hist=True)
    rng = np.random.default_rng(side)
    rows = np.unique(np.concatenate([[0, side - 1, side // 2], rng.choice(side, 29, replace=False)]))
    k = oracle.render_rows(f["c"], f["rect"], side, side, rows, 100, 0, 0)
    mism = int((g["counts"][rows] != k).sum())
    assert mism == 0, "%d mismatches in %d sampled rows" % (mism, rows.size)
    assert (g["rgba"][rows] == oracle.colour(k, 100, PAL)).all()
    assert (g["hist"] == oracle.hist(g["counts"], 100)).all()
    # 180-degree rotation symmetry of the whole frame (the grid's coordinates
    # are exact negatives of each other when the side is even)
    if side % 2 == 0:
        assert (g["counts"] == g["counts"][::-1, ::-1]).all()
