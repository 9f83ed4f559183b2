"""The certified binary32 pass of binary64 frames (paper Sec. 3: binary64 for
deep zooms).  A binary64 pixel's count is kept from the binary32 orbit only
when a rigorous bound on the distance between the binary32 and binary64 orbits
settles every binary64 test; the other pixels go to the binary64 kernel.  The
counts must be the binary64 oracle's, bit for bit, with the pass on or off, on
views where the bound settles nearly everything, views where it settles little
(deep zooms on the Julia set), |C| near 2, the Mandelbrot band |C| ~ 2, limits
shorter than a block, ragged sizes and coordinates that overflow binary32.

All calls go through the C ABI (libjl.so via the ctypes binding)."""
import numpy as np
import pytest

import oracle
import paper_1611_03079_b300 as jl
from paper_1611_03079_b300 import workloads as wl

pytestmark = pytest.mark.gpu

PAL = wl.random_palette(11)
FP64 = wl.FP64


def _frames():
    fr = []
    for f in wl.throughput_sweep(192):
        if f["precision"] == FP64:
            fr.append(dict(f, count_type="u16"))
    sq = (-2.2, 2.2, -2.2, 2.2)
    # |C|^2 = 4, > 4, ~4, 3.998 (per-step tests), 0, 0.5625, and 3.980 / 3.9896 (just inside the
    # |C32| <= 2 - 2^-12 range where a block forms only its last test)
    for c in (complex(-2.0, 0.0), complex(2.5, 0.1), complex(-1.9999, 0.0), complex(1.414, 1.414),
              complex(0.0, 0.0), complex(-0.75, 0.0), complex(-1.995, 0.0), complex(0.0, 1.9974)):
        fr.append(dict(c=c, rect=sq, W=64, H=61, max_iter=300, mode=wl.JULIA, precision=FP64, count_type="u16"))
    fr.append(dict(c=None, rect=(-2.05, -1.95, -0.05, 0.05), W=97, H=61, max_iter=500, mode=wl.MANDELBROT,
                   precision=FP64, count_type="u16"))
    # Mandelbrot pixels on both edges of the band |C|^2 in (3.99, 4.01)
    fr.append(dict(c=None, rect=(-0.01, 0.01, 1.994, 2.004), W=37, H=101, max_iter=800, mode=wl.MANDELBROT,
                   precision=FP64, count_type="u16"))
    c = complex(-0.7269, 0.1889)
    for k, z in enumerate(wl.julia_boundary_points(c, 3, seed=5)):
        w = 10.0 ** (-3 - 3 * k)
        fr.append(dict(c=c, rect=(z.real - w / 2, z.real + w / 2, z.imag - w / 4, z.imag + w / 4), W=96, H=48,
                       max_iter=2000, mode=wl.JULIA, precision=FP64, count_type="u16"))
    for mi in (1, 2, 3, 4, 5, 7):
        fr.append(dict(c=complex(-0.8, 0.156), rect=(-1.5, 1.5, -1.5, 1.5), W=33, H=17, max_iter=mi,
                       mode=wl.JULIA, precision=FP64, count_type="u16"))
        fr.append(dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=17, H=33, max_iter=mi, mode=wl.MANDELBROT,
                       precision=FP64, count_type="u16"))
    fr.append(dict(c=complex(0.285, 0.01), rect=(-1e25, 1e25, -1e25, 1e25), W=16, H=16, max_iter=50,
                   mode=wl.JULIA, precision=FP64, count_type="u16"))
    fr.append(dict(c=complex(0.285, 0.01), rect=(-1e300, 1e300, -1e300, 1e300), W=8, H=8, max_iter=50,
                   mode=wl.JULIA, precision=FP64, count_type="u16"))
    fr.append(dict(c=None, rect=(-1e30, 1e30, -1e30, 1e30), W=9, H=7, max_iter=50, mode=wl.MANDELBROT,
                   precision=FP64, count_type="u16"))
    fr.append(dict(c=complex(-0.1, 0.65), rect=(-0.1, 0.1, 0.5, 0.7), W=1, H=1, max_iter=1000, mode=wl.JULIA,
                   precision=FP64, count_type="u16"))
    return fr


def _oracle(f):
    return oracle.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], f["mode"], 1)


def _np_counts(t):
    import torch
    if t.dtype == torch.uint8:
        return t.cpu().numpy().astype(np.uint16)
    return t.cpu().numpy().view(np.uint16)


@pytest.fixture(scope="module")
def frames_and_refs():
    fr = _frames()
    return fr, [_oracle(f) for f in fr]


@pytest.mark.parametrize("certify,certify2", [(True, True), (True, False), (False, True)])
def test_batch_counts_equal_binary64_oracle(cuda, frames_and_refs, certify, certify2):
    import torch
    fr, refs = frames_and_refs
    b = jl.Batch(fr, palette=PAL, certify=certify, certify2=certify2)
    b.launch()
    torch.cuda.synchronize()
    assert b.status() == 0
    for i, (f, k) in enumerate(zip(fr, refs)):
        g = _np_counts(b.counts(i))
        mism = int((g != k).sum())
        assert mism == 0, "frame %d %s: %d count mismatches (certify=%s)" % (i, f, mism, certify)
        assert (b.rgba(i).cpu().numpy() == oracle.colour(k, f["max_iter"], PAL)).all()
    l32, l64, it_df, it64, st32, st_df = b.cert_stats()
    total = sum(f["W"] * f["H"] for f in fr)
    total_it = sum(int(k.astype(np.int64).sum()) for k in refs)
    if certify:
        assert 0 < l32 < total and 0 <= l64 <= l32
        # every pixel decides at least one test in the binary32 pass, every
        # listed pixel at least one in the double-float pass
        assert st32 >= total and (st_df >= l32 if certify2 else st_df == 0)
        # the iterations settled by the double-float pass and run in binary64
        # are parts of the frames' iterations
        assert 0 <= it_df and 0 <= it64 and it_df + it64 <= total_it
        if not certify2:
            assert l64 == l32 and it_df == 0
    else:
        assert (l32, l64, it_df, it64, st32, st_df) == (0, 0, 0, 0, 0, 0)


def test_certified_pass_settles_most_sweep_pixels(cuda):
    """On the sweep's binary64 views the bound settles all but a few per cent of
    the pixels (the rest lie near the sets' boundaries)."""
    import torch
    fr = [f for f in wl.throughput_sweep(512) if f["precision"] == FP64]
    b = jl.Batch(fr, palette=PAL)
    b.launch()
    torch.cuda.synchronize()
    l32, l64, it_df, it64, st32, st_df = b.cert_stats()
    total = sum(f["W"] * f["H"] for f in fr)
    assert 0 < l32 < 0.05 * total, (l32, total)
    # the binary32 pass decides each settled pixel's tests up to its escape
    assert st32 >= sum(int(np.minimum(_oracle(f).astype(np.int64) + 1, f["max_iter"]).sum()) for f in fr) - \
        it_df - it64 - 2 * l32
    # the double-float pass settles most of what the binary32 pass lists
    assert l64 < 0.5 * l32 and it_df > 0, (l32, l64, it_df)
    assert it_df + it64 < sum(int(_oracle(f).astype(np.int64).sum()) for f in fr)
    for i in (1, 7):
        assert (_np_counts(b.counts(i)) == _oracle(fr[i])).all()
    # phase events: both certified passes and the binary64 kernel timed
    p = jl.Batch(fr, palette=PAL, phases=True)
    p.launch()
    torch.cuda.synchronize()
    ms = p.phase_ms()
    assert ms[0] == -1.0 and ms[1] > 0 and ms[2] > 0 and ms[3] > 0, ms


def _variants64():
    import ctypes
    L = jl._lib.lib()
    n = L.jl_variant_list(1, None, 0)
    buf = (ctypes.c_int32 * (2 * n))()
    L.jl_variant_list(1, buf, n)
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(n)]


@pytest.mark.parametrize("threads", [128, 256])
def test_single_frames_every_binary64_variant(cuda, threads):
    """jl_render of binary64 frames (certified pass + the list on the
    lane-refill variants; the static kernel without it), with histograms
    (shared-memory bins in both kernels)."""
    import torch
    fr = [dict(c=complex(-0.7269, 0.1889), rect=(-1.6, 1.6, -1.6, 1.6), W=257, H=131, max_iter=1000,
               mode=wl.JULIA, precision=FP64),
          dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=130, H=97, max_iter=300, mode=wl.MANDELBROT,
               precision=FP64)]
    refs = [_oracle(f) for f in fr]
    for (ppt, u) in _variants64():
        for f, k in zip(fr, refs):
            out = jl.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=FP64, mode=f["mode"],
                            count_type="u16", rgba=True, hist=True, palette=PAL, variant=(ppt, u, threads, 0))
            torch.cuda.synchronize()
            g = out["counts"].view(torch.int16).cpu().numpy().view(np.uint16)
            assert (g == k).all(), "variant %s: %d mismatches" % ((ppt, u, threads), int((g != k).sum()))
            assert (out["rgba"].cpu().numpy() == oracle.colour(k, f["max_iter"], PAL)).all()
            assert (out["hist"].cpu().numpy() == oracle.hist(k, f["max_iter"])).all()


def test_batch_histograms_binary64(cuda):
    """Global histogram bins from both the certified pass and the list kernel."""
    import torch
    fr = [dict(c=complex(-0.4, 0.6), rect=(-1.6, 1.6, -1.6, 1.6), W=150, H=101, max_iter=1000, mode=wl.JULIA,
               precision=FP64, count_type=None, hist=True),
          dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=101, H=150, max_iter=100, mode=wl.MANDELBROT,
               precision=FP64, count_type="u8", hist=True)]
    b = jl.Batch(fr, palette=PAL)
    b.launch()
    torch.cuda.synchronize()
    for i, f in enumerate(fr):
        k = _oracle(f)
        assert (b.hist(i).cpu().numpy() == oracle.hist(k, f["max_iter"])).all()
        assert (b.rgba(i).cpu().numpy() == oracle.colour(k, f["max_iter"], PAL)).all()
    assert (_np_counts(b.counts(1)) == _oracle(fr[1])).all()


@pytest.mark.parametrize("seed", range(10))
def test_boundary_views_binary64(cuda, seed):
    """Binary64 frames centred on Julia and Mandelbrot boundary points, widths
    down to 1e-13 and limits up to 3000 (the certified passes' hardest tests),
    as one plan with both passes and as single frames: bit-exact counts."""
    import torch
    fr = [dict(f, count_type="u16") for f in wl.boundary_views(60, seed=40 + seed)]
    refs = [_oracle(f) for f in fr]
    b = jl.Batch(fr, palette=PAL)
    b.launch()
    torch.cuda.synchronize()
    assert b.status() == 0
    for i, (f, k) in enumerate(zip(fr, refs)):
        g = _np_counts(b.counts(i))
        assert (g == k).all(), "frame %d %s: %d mismatches" % (i, f, int((g != k).sum()))
    for f, k in list(zip(fr, refs))[:12]:
        out = jl.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], precision=FP64, mode=f["mode"],
                        count_type="u16", rgba=False, palette=PAL)
        torch.cuda.synchronize()
        assert (out["counts"].view(torch.int16).cpu().numpy().view(np.uint16) == k).all(), f
