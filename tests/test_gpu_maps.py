"""Generic maps on the GPU (jl_render_map) against the CPU oracle: escape
counts bit for bit, colours and histograms exactly, for Z <- Z^d + C
(d = 2..16, compile-time and run-time degrees) and Z <- P(Z)/Q(Z) + C
(Fig. 4's map as printed and seeded rational maps), both precisions, both
modes, ragged sizes that span several 32 x 32 tiles, and the degenerate
cases (1 x 1 frames, a limit of 1, Q = 0)."""
import numpy as np
import pytest

import oracle
import paper_1611_03079_b300 as jl
from paper_1611_03079_b300 import workloads as wl

pytestmark = pytest.mark.gpu

PREC = {0: "fp32", 1: "fp64"}
MODE = {0: "julia", 1: "mandelbrot"}


def gpu_counts(m, c, rect, W, H, mi, mode, prec, **kw):
    import torch
    out = jl.render_map(m, c, rect, W, H, mi, precision=PREC[prec], mode=MODE[mode], rgba=False, **kw)
    torch.cuda.synchronize()
    return out["counts"].view(torch.int16).cpu().numpy().view(np.uint16)


def check(m, c, rect, W, H, mi, mode, prec):
    got = gpu_counts(m, c, rect, W, H, mi, mode, prec)
    ref = oracle.render_map(m, c, rect, W, H, mi, mode, prec)
    bad = np.argwhere(got != ref)
    assert bad.size == 0, (m["kind"], m.get("degree"), prec, mode, bad[:5], got[tuple(bad[0])], ref[tuple(bad[0])])
    return ref


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d", [2, 3, 4, 5, 6, 7, 8, 9, 12, 16])
def test_power_maps(cuda, prec, d):
    # Multi-Julia (C near the boundary of the connectedness locus) and the
    # parameter plane; 333 x 197 leaves ragged tiles in both directions
    ref = check(wl.power_map(d), complex(-0.55, 0.48), (-1.5, 1.5, -1.3, 1.3), 333, 197, 300, 0, prec)
    assert 0 < ref.mean() < 300
    check(wl.power_map(d), 0j, (-1.6, 1.6, -1.6, 1.6), 211, 203, 200, 1, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_power2_matches_quadratic_path(cuda, prec):
    import torch
    c, rect = complex(-0.7269, 0.1889), (-1.6, 1.6, -1.6, 1.6)
    a = gpu_counts(wl.power_map(2), c, rect, 640, 360, 500, 0, prec)
    b = jl.render(c, rect, 640, 360, 500, precision=PREC[prec], rgba=False)["counts"]
    torch.cuda.synchronize()
    assert (a == b.view(torch.int16).cpu().numpy().view(np.uint16)).all()


@pytest.mark.parametrize("prec", [0, 1])
def test_fig4_map_as_printed(cuda, prec):
    ref = check(wl.fig4_map(), wl.FIG4_C, (-1.6, 1.6, -1.6, 1.6), 301, 257, 100, 0, prec)
    assert ref.max() >= 2


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("prec", [0, 1])
def test_random_rational_maps(cuda, seed, prec):
    rng = np.random.default_rng(seed)
    nd, nq = int(rng.integers(0, 9)), int(rng.integers(0, 9))
    m = wl.random_rational_map(seed, num_degree=max(nd, 2), den_degree=nq)
    check(m, complex(*rng.uniform(-0.5, 0.5, 2)), (-2.0, 2.0, -1.5, 1.5), 150, 113, 250, 0, prec)
    check(dict(m, z0=complex(*rng.uniform(-0.5, 0.5, 2))), 0j, (-2.0, 2.0, -2.0, 2.0), 97, 131, 150, 1, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_degree_extremes_and_degenerate_cases(cuda, prec):
    rect = (-2.0, 2.0, -2.0, 2.0)
    # constant P over degree-8 Q, degree-8 P over constant Q
    check(wl.rational_map([0.4 + 0.1j], [1, 0, 0, 0, 0, 0, 0, 0, 0.5]), 0.1j, rect, 64, 40, 120, 0, prec)
    check(wl.rational_map([0, 0, 0, 0, 0, 0, 0, 0.3, 1], [2]), -0.2, rect, 40, 64, 120, 0, prec)
    # Q = 0: NaN after the first update -> count 1 inside the bailout disc
    ref = check(wl.rational_map([1, 1], [0]), 0.3, rect, 50, 50, 40, 0, prec)
    assert set(np.unique(ref)) <= {0, 1}
    # 1 x 1, 1 x N, N x 1 frames and a limit of 1
    for W, H in ((1, 1), (1, 77), (77, 1)):
        check(wl.power_map(3), 0.2 + 0.3j, (-1.0, 1.0, -1.0, 1.0), W, H, 50, 0, prec)
    check(wl.power_map(5), 0.2 + 0.3j, (-1.5, 1.5, -1.5, 1.5), 65, 33, 1, 0, prec)
    # a large bailout
    check(dict(wl.power_map(4), bailout=1e6), -0.3j, (-1.5, 1.5, -1.5, 1.5), 70, 70, 90, 0, prec)


def test_outputs_u8_rgba_hist(cuda):
    import torch
    m, c, rect, W, H, mi = wl.power_map(3), complex(0.4, 0.2), (-1.4, 1.4, -1.2, 1.2), 257, 129, 200
    pal = wl.random_palette(3)
    out = jl.render_map(m, c, rect, W, H, mi, count_type="u8", rgba=True, hist=True, palette=pal)
    torch.cuda.synchronize()
    ref = oracle.render_map(m, c, rect, W, H, mi, 0, 0)
    assert (out["counts"].cpu().numpy() == ref).all()
    ref_rgba = oracle.colour(ref, mi, pal)
    assert (out["rgba"].cpu().numpy() == ref_rgba).all()
    assert (out["hist"].cpu().numpy() == oracle.hist(ref, mi)).all()
    # global-memory histogram path (limit above the shared-memory bins)
    mi2 = 5000
    out2 = jl.render_map(m, c, rect, 97, 61, mi2, count_type="u16", rgba=False, hist=True)
    torch.cuda.synchronize()
    ref2 = oracle.render_map(m, c, rect, 97, 61, mi2, 0, 0)
    assert (out2["hist"].cpu().numpy() == oracle.hist(ref2, mi2)).all()


def test_auto_precision_on_a_deep_view(cuda):
    m = wl.power_map(3)
    cx, cy, w = -0.2, 0.75, 1e-9
    rect = (cx - w, cx + w, cy - w, cy + w)
    assert jl.select_precision(rect, 160, 160) == 1
    got = gpu_counts(m, 0j, rect, 160, 160, 400, 1, 1)
    import torch
    auto = jl.render_map(m, 0j, rect, 160, 160, 400, precision="auto", mode="mandelbrot", rgba=False)["counts"]
    torch.cuda.synchronize()
    assert (auto.view(torch.int16).cpu().numpy().view(np.uint16) == got).all()
    assert (got == oracle.render_map(m, 0j, rect, 160, 160, 400, 1, 1)).all()


@pytest.mark.parametrize("fi", range(6))
def test_benchmark_frames_sampled(cuda, fi):
    """The 4096 x 4096 benchmark frames: 20,000 sampled pixels against the
    oracle one by one, and the count histogram sums to W*H."""
    import torch
    f = wl.map_sweep(4096)[fi]
    out = jl.render_map(f["map"], f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=PREC[f["precision"]],
                        mode=MODE[f["mode"]], rgba=False, hist=True)
    torch.cuda.synchronize()
    counts = out["counts"].view(torch.int16).cpu().numpy().view(np.uint16)
    rng = np.random.default_rng(fi)
    xmin, xmax, ymin, ymax = f["rect"]
    dx, dy = (xmax - xmin) / f["W"], (ymax - ymin) / f["H"]
    for _ in range(20000):
        i, j = int(rng.integers(0, f["W"])), int(rng.integers(0, f["H"]))
        p = complex(xmin + (i + 0.5) * dx, ymin + (j + 0.5) * dy)
        if f["mode"] == 0:
            ref = oracle.map_escape_point(f["map"], p, f["c"], f["max_iter"], f["precision"])
        else:
            ref = oracle.map_escape_point(f["map"], f["map"]["z0"], p, f["max_iter"], f["precision"])
        assert counts[j, i] == ref, (fi, i, j)
    h = out["hist"].cpu().numpy().astype(np.float64)
    assert abs(h.sum() - 1.0) < 1e-5
