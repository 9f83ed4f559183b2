"""jl_render_frames_to_host: frames rendered into pinned host memory with the
copies overlapped.  Every depth (device slots: 1 .. 16, fewer than, as many
as and more than the frame count, and the default) gives
counts, colours and histograms identical to the oracle and to the device
render of the same frame; repeated calls reuse the buffers; frames without
counts or with histograms only; bad frames are rejected before any work."""
import numpy as np
import pytest

import oracle
import paper_1611_03079_b300 as jl
from paper_1611_03079_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def mixed_frames():
    frames = []
    for i, f in enumerate(wl.random_views(9, seed=77)):
        f = dict(f)
        f["count_type"] = "u8" if f["max_iter"] <= 255 and i % 3 == 0 else "u16"
        f["rgba"] = i % 4 != 1
        f["hist"] = i % 2 == 0
        frames.append(f)
    frames.append(dict(c=complex(-0.7269, 0.1889), rect=(-1.6, 1.6, -1.6, 1.6), W=640, H=480, max_iter=500,
                       mode="julia", precision="fp64", count_type="u16", rgba=True, hist=True))
    frames.append(dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=777, H=333, max_iter=300, mode="mandelbrot",
                       precision="fp32", count_type=None, rgba=True, hist=False))
    return frames


def _oracle_counts(f):
    mode = 0 if f.get("mode", "julia") in ("julia", 0) else 1
    prec = {"fp32": 0, "fp64": 1, 0: 0, 1: 1}[f.get("precision", "fp32")]
    return oracle.render(f["c"] if f["c"] is not None else 0j, f["rect"], f["W"], f["H"], f["max_iter"], mode, prec)


@pytest.mark.parametrize("depth", [1, 2, 3, 8, 11, 16, 0])
def test_host_frames_match_oracle(cuda, depth):
    frames = mixed_frames()
    pal = wl.random_palette(5)
    hf = jl.HostFrames(frames, palette=pal, depth=depth)
    for _ in range(2):
        hf.render()
    for i, f in enumerate(frames):
        ref = _oracle_counts(f)
        if f.get("count_type"):
            assert (hf.counts(i) == ref).all(), i
        else:
            assert hf.counts(i) is None
        if f.get("rgba", True):
            assert (hf.rgba(i) == oracle.colour(ref, f["max_iter"], pal)).all(), i
        if f.get("hist"):
            assert (hf.hist(i) == oracle.hist(ref, f["max_iter"])).all(), i


def test_matches_device_render(cuda):
    import torch
    frames = wl.throughput_sweep(512)
    for f in frames:
        f["count_type"], f["rgba"] = "u16", True
    hf = jl.HostFrames(frames, depth=3)
    hf.render()
    for i, f in enumerate(frames):
        d = jl.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=f["precision"], mode=f["mode"],
                      count_type="u16", rgba=True)
        torch.cuda.synchronize()
        assert (d["counts"].view(torch.int16).cpu().numpy().view(np.uint16) == hf.counts(i)).all()
        assert (d["rgba"].cpu().numpy() == hf.rgba(i)).all()


def test_rejects_bad_frames(cuda):
    bad = [dict(c=0.1, rect=(1.0, -1.0, 0.0, 1.0), W=8, H=8, max_iter=10, count_type="u16")]
    with pytest.raises(jl.JLError):
        jl.HostFrames(bad).render()
    with pytest.raises(jl.JLError):
        jl.HostFrames([dict(c=0.1, rect=(-1, 1, -1, 1), W=8, H=8, max_iter=10, count_type="u16")], depth=65).render()
    with pytest.raises(jl.JLError):
        jl.HostFrames([dict(c=0.1, rect=(-1, 1, -1, 1), W=8, H=8, max_iter=10, count_type="u16")], depth=-1).render()


def test_one_shot_call_matches_plan(cuda):
    """jl_render_frames_to_host (plan created, run and destroyed in one call)
    writes the same bytes as a reused plan."""
    frames = mixed_frames()
    hf = jl.HostFrames(frames, depth=4)
    hf.render()
    c2 = np.zeros_like(hf.counts_buf)
    r2 = np.zeros_like(hf.rgba_buf)
    h2 = np.zeros_like(hf.hist_buf)
    jl._lib.check(jl._lib.lib().jl_render_frames_to_host(hf._arr, len(frames), c2.ctypes.data, r2.ctypes.data,
                                                         h2.ctypes.data, None, 2, None))
    assert (c2 == hf.counts_buf).all() and (r2 == hf.rgba_buf).all() and (h2 == hf.hist_buf).all()
    hf.close()


_BIG = {}


def _big_ref(prec, mode, ct):
    key = (prec, mode, ct)
    if key not in _BIG:
        f = dict(c=complex(-0.4, 0.6) if mode == "julia" else None, rect=(-1.9, 1.1, -1.2, 1.2), W=2049, H=1371,
                 max_iter=200 if ct == "u8" else 300, mode=mode, precision=prec, count_type=ct, rgba=True,
                 hist=False)
        _BIG[key] = (f, _oracle_counts(f))
    return _BIG[key]


@pytest.mark.parametrize("depth", [1, 0])
@pytest.mark.parametrize("prec,mode,ct", [("fp32", "julia", "u16"), ("fp64", "mandelbrot", "u8"),
                                          ("fp32", "mandelbrot", "u16")])
def test_banded_last_frame(cuda, depth, prec, mode, ct):
    """A last frame with 8 MB or more of counts + RGBA renders as row bands of
    whole 32-row tiles (2049 x 1371: 3 bands with uint16 counts, 2 with
    uint8, the last one ragged) copied out band by band; with depth 1 every
    band also waits for the previous frame's copy out of the shared slot.
    Counts and colours equal the oracle's for the whole frame, so the bands
    use the frame's own pixel coordinates."""
    big, ref = _big_ref(prec, mode, ct)
    small = dict(c=complex(0.285, 0.01), rect=(-1.5, 1.5, -1.5, 1.5), W=300, H=200, max_iter=150, mode="julia",
                 precision="fp64", count_type="u16", rgba=True, hist=True)
    pal = wl.random_palette(11)
    hf = jl.HostFrames([small, big], palette=pal, depth=depth)
    assert hf.launches() == 1 + (2 if ct == "u8" else 3)
    for _ in range(2):
        hf.render()
    assert (hf.counts(1) == ref).all()
    assert (hf.rgba(1) == oracle.colour(ref, big["max_iter"], pal)).all()
    sref = _oracle_counts(small)
    assert (hf.counts(0) == sref).all() and (hf.hist(0) == oracle.hist(sref, small["max_iter"])).all()
    hf.close()


def test_last_frame_with_histogram_is_not_banded(cuda):
    big, ref = _big_ref("fp32", "julia", "u16")
    f = dict(big, hist=True)
    hf = jl.HostFrames([f], depth=0)
    assert hf.launches() == 1
    hf.render()
    assert (hf.counts(0) == ref).all() and (hf.hist(0) == oracle.hist(ref, f["max_iter"])).all()
    hf.close()
