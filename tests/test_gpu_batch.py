"""GPU parity of batch plans (one CUDA-graph launch of persistent escape
kernels over many frames, Sec. 3 parameter paths) and of the autotuner's
choices, against the CPU oracle.  All calls go through the C ABI."""
import numpy as np
import pytest

import oracle
import paper_1611_03079_b300 as jl
from paper_1611_03079_b300 import workloads as wl

pytestmark = pytest.mark.gpu

PAL = wl.random_palette(7)


def _np_counts(t):
    import torch
    if t.dtype == torch.uint8:
        return t.cpu().numpy().astype(np.uint16)
    return t.cpu().numpy().view(np.uint16)


def _oracle(f, prec):
    return oracle.render(f.get("c"), f["rect"], f["W"], f["H"], f["max_iter"], f["mode"], prec)


def _check_batch(b, frames, precs=None, hist=True):
    import torch
    torch.cuda.synchronize()
    precs = precs or b.precisions()
    for i, f in enumerate(frames):
        k = _oracle(f, precs[i])
        if b.counts(i) is not None:
            assert (_np_counts(b.counts(i)) == k).all(), (i, f)
        if b.rgba(i) is not None:
            assert (b.rgba(i).cpu().numpy() == oracle.colour(k, f["max_iter"], PAL)).all(), (i, f)
        if hist and b.hist(i) is not None:
            assert (b.hist(i).cpu().numpy() == oracle.hist(k, f["max_iter"])).all(), (i, f)


@pytest.mark.parametrize("chunk_len", [0, 64, 1024])
def test_mixed_batch(cuda, chunk_len):
    """Random frames (ragged sizes, both modes, both precisions, limits 1..300,
    uint8/uint16/no counts, with and without histograms) in one plan."""
    frames = []
    for i, f in enumerate(wl.random_views(40, seed=300 + chunk_len)):
        f = dict(f)
        f["count_type"] = [None, "u16", "u8"][i % 3] if f["max_iter"] <= 255 else [None, "u16"][i % 2]
        f["rgba"] = (i % 4) != 1
        f["hist"] = (i % 2) == 0
        if f["count_type"] is None and not f["rgba"]:
            f["hist"] = True
        frames.append(f)
    b = jl.Batch(frames, palette=PAL, chunk_len=chunk_len)
    b.launch()
    _check_batch(b, frames)
    # replay of the same graph gives the same result
    b.launch()
    _check_batch(b, frames)
    assert b.status() == 0
    b.close()


def test_batch_matches_jl_render(cuda):
    import torch
    frames = [dict(c=complex(-0.7269, 0.1889), rect=(-1.6, 1.6, -1.6, 1.6), W=777, H=513, max_iter=1000,
                   mode=0, precision=p, count_type="u16", hist=True) for p in (0, 1)]
    frames.append(dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=640, H=480, max_iter=255, mode=1,
                       precision=2, count_type="u8", hist=True))
    b = jl.Batch(frames, palette=PAL)
    b.launch()
    torch.cuda.synchronize()
    for i, f in enumerate(frames):
        r = jl.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=f["precision"],
                      mode=f["mode"], count_type=f["count_type"], rgba=True, hist=True, palette=PAL)
        torch.cuda.synchronize()
        assert (_np_counts(r["counts"]) == _np_counts(b.counts(i))).all()
        assert (r["rgba"].cpu().numpy() == b.rgba(i).cpu().numpy()).all()
        assert (r["hist"].cpu().numpy() == b.hist(i).cpu().numpy()).all()


def test_histogram_batch_small_frames(cuda):
    """Surrogate targets: many 128x128 frames over [-2,2]^2, limit 100, only
    histograms (warp-aggregated global bins)."""
    cs = wl.survey_c(300, seed=9)
    frames = [dict(c=complex(float(a), float(b_)), rect=(-2.0, 2.0, -2.0, 2.0), W=128, H=128, max_iter=100,
                   mode=0, precision=0, count_type=None, rgba=False, hist=True) for a, b_ in cs]
    b = jl.Batch(frames, palette=PAL)
    b.launch()
    _check_batch(b, frames)


def test_path_animation_sampled(cuda):
    """The 720-frame path animation (three resolutions up to 3840x2160) in one
    plan; 12 frames checked in full against the oracle."""
    frames = wl.path_animation()
    b = jl.Batch(frames, palette=PAL)
    b.launch()
    import torch
    torch.cuda.synchronize()
    assert b.status() == 0
    rng = np.random.default_rng(1)
    for i in sorted(rng.choice(len(frames), 12, replace=False)):
        f = frames[i]
        k = _oracle(f, 0)
        assert (b.rgba(i).cpu().numpy() == oracle.colour(k, f["max_iter"], PAL)).all(), i
    b.close()


def test_cycle_budget_timeout(cuda):
    """A launch whose cycle budget runs out stops taking work and reports
    JL_ETIMEOUT through the status word (no fault, context stays usable)."""
    frames = [dict(c=complex(-0.7269, 0.1889), rect=(-1.6, 1.6, -1.6, 1.6), W=2048, H=2048, max_iter=1000,
                   mode=0, precision=1, count_type="u16")]
    b = jl.Batch(frames, palette=PAL, cycle_budget=1)
    b.launch()
    assert b.status() == jl._lib.JL_ETIMEOUT
    b.close()
    # the context is still usable
    test_batch_matches_jl_render(cuda)


def test_autotune_choice_is_exact(cuda, tmp_path):
    jl.tune_clear()
    r = jl.autotune("fp32", 100, reps=1)
    assert r["candidates"] >= 6
    g = jl.tune_get("fp32", 100)
    assert g["tuned"] and (g["ppt"], g["unroll"], g["threads"]) == (r["ppt"], r["unroll"], r["threads"])
    f = dict(c=complex(-0.4, 0.6), rect=(-1.6, 1.6, -1.6, 1.6), W=900, H=700, max_iter=100, mode=0, precision=0)
    out = jl.render(f["c"], f["rect"], f["W"], f["H"], 100, precision=0, count_type="u16", palette=PAL)
    import torch
    torch.cuda.synchronize()
    assert (_np_counts(out["counts"]) == _oracle(f, 0)).all()
    p = tmp_path / "tune.txt"
    jl.tune_save(p)
    jl.tune_clear()
    assert not jl.tune_get("fp32", 100)["tuned"]
    jl.tune_load(p)
    assert jl.tune_get("fp32", 100)["tuned"]
    jl.tune_clear()


@pytest.mark.parametrize("prec", [0, 1])
def test_static_variant_batch(cuda, prec):
    """The static kernel (one pixel per thread) in a batch plan, chosen
    explicitly, on ragged frames of both modes."""
    frames = []
    for i, f in enumerate(wl.random_views(24, seed=700 + prec)):
        f = dict(f)
        f["precision"] = prec
        f["count_type"] = "u16"
        f["hist"] = i % 2 == 0
        frames.append(f)
    key = "fp64" if prec else "fp32"
    b = jl.Batch(frames, palette=PAL, variants={key: (0, 0, 256)})
    b.launch()
    _check_batch(b, frames)
    b.close()


def test_cardioid_path_with_minimap(cuda):
    """The paper's clockwise a = 3.9 cardioid path (Sec. 3, Fig. 2), each
    Julia frame paired with the Mandelbrot minimap, as one batch plan."""
    from paper_1611_03079_b300 import paths
    frames = paths.with_minimap(paths.julia_frames(paths.cardioid_path(24), W=160, H=120, count_type="u16"))
    b = jl.Batch(frames, palette=PAL)
    b.launch()
    _check_batch(b, frames)
    b.close()


def test_mandelbrot_deep_zoom_fig3(cuda):
    """Deep zoom on the Mandelbrot set at the Fig. 3 values (AUTO precision,
    limit 2000): counts bit-exact in the precision the library chose."""
    from paper_1611_03079_b300 import paths
    frames = []
    for c in (complex(0.177078, 0.577384), complex(0.185723, 0.588104)):
        frames += paths.mandelbrot_zoom(c, 6, W=320, H=180)
    b = jl.Batch(frames, palette=PAL)
    b.launch()
    precs = b.precisions()
    assert 0 < sum(precs) < len(precs)
    _check_batch(b, frames, precs=precs)
    b.close()


@pytest.mark.parametrize("T", [8, 16])
def test_compact_variant_batch(cuda, T):
    """The compacting tile kernel in a batch plan: parked pixels of different
    frames (limits, modes, count types, histograms) share resumed batches."""
    frames = []
    for i, f in enumerate(wl.random_views(24, seed=800 + T)):
        f = dict(f)
        f["precision"] = 0
        f["count_type"] = "u8" if (i % 3 == 0 and f["max_iter"] <= 255) else "u16"
        f["hist"] = i % 2 == 0
        frames.append(f)
    frames.append(dict(c=complex(-0.7269, 0.1889), rect=(-1.6, 1.6, -1.6, 1.6), W=300, H=257, max_iter=1000,
                       mode=0, precision=0, count_type="u16", hist=True))
    frames.append(dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=257, H=300, max_iter=700, mode=1, precision=0,
                       count_type="u16", hist=False))
    b = jl.Batch(frames, palette=PAL, variants={"fp32": (0, T, 256)})
    b.launch()
    _check_batch(b, frames)
    b.close()


def test_tuned_plan(cuda):
    """A plan that times candidate kernels on its own frames at creation
    (both precisions, histograms on some frames) renders them bit-exactly,
    and launching it again gives the same outputs."""
    import torch
    frames = []
    for i, f in enumerate(wl.random_views(20, seed=950)):
        f = dict(f)
        f["count_type"] = "u16"
        f["hist"] = i % 3 == 0
        frames.append(f)
    frames.append(dict(c=complex(-0.7269, 0.1889), rect=(-1.6, 1.6, -1.6, 1.6), W=256, H=200, max_iter=1000, mode=0,
                       precision=0, count_type="u16", hist=True))
    b = jl.Batch(frames, palette=PAL, tune=True)
    for prec in (0, 1):
        ppt, unroll, threads = b.variant(prec)
        assert ppt >= 0 and unroll >= 0 and threads in (128, 256)
    b.launch()
    _check_batch(b, frames)
    first = b.counts_buf.clone()
    b.launch()
    torch.cuda.synchronize()
    assert torch.equal(first, b.counts_buf)
    _check_batch(b, frames)
    b.close()
