"""Output-overrun checks: every output the library writes is placed between
guard bands of a known byte pattern, and after the call the bands must be
untouched.  This is the stand-in for a memory checker: ragged tiles, row
bands, parked-and-resumed pixels and the batch frame tables must all stay
inside their own outputs.  The outputs themselves are also pre-filled with
the pattern and then compared with the oracle (Sec. 2 escape counts and
colour levels), so every byte inside is written exactly once with the right
value.

All calls go through the C ABI (libjl.so via ctypes)."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1611_03079_b300 as jl
from paper_1611_03079_b300 import _lib, workloads as wl

pytestmark = pytest.mark.gpu

GUARD = 4096
PATTERN = 0xA5
PAL = wl.random_palette(11)


def _round16(n):
    return (n + 15) & ~15


class Arena:
    """One byte buffer (device or pinned host) holding regions separated by
    GUARD-byte bands, everything pre-filled with PATTERN."""

    def __init__(self, sizes, host=False):
        import torch
        self.offsets, o = [], GUARD
        for s in sizes:
            self.offsets.append(o)
            o += _round16(max(int(s), 0)) + GUARD
        self.sizes = [int(s) for s in sizes]
        self.total = o
        if host:
            self.buf = torch.full((o,), PATTERN, dtype=torch.uint8, pin_memory=True)
        else:
            self.buf = torch.full((o,), PATTERN, dtype=torch.uint8, device="cuda")
        self.host = host

    def ptr(self, i):
        return self.buf.data_ptr() + self.offsets[i]

    def bytes(self):
        import torch
        if not self.host:
            torch.cuda.synchronize()
        return self.buf.cpu().numpy()

    def region(self, i, b=None):
        b = self.bytes() if b is None else b
        return b[self.offsets[i]:self.offsets[i] + self.sizes[i]]

    def check_guards(self, what):
        b = self.bytes()
        mask = np.ones(self.total, bool)
        for o, s in zip(self.offsets, self.sizes):
            mask[o:o + s] = False
        bad = np.nonzero(mask & (b != PATTERN))[0]
        assert bad.size == 0, "%s: %d guard bytes overwritten, first at %s" % (what, bad.size, bad[:8])
        return b


def _oracle(f):
    p = f["precision"]
    if p == wl.AUTO:
        p = oracle.precision_for_view(f["rect"], f["W"], f["H"])
    return oracle.render(f.get("c"), f["rect"], f["W"], f["H"], f["max_iter"], f["mode"], p)


def _check_outputs(f, k, counts_bytes, rgba_bytes, hist_bytes, ct):
    H, W = f["H"], f["W"]
    if ct == "u8":
        assert (counts_bytes.reshape(H, W).astype(np.uint16) == k).all()
    elif ct == "u16":
        assert (counts_bytes.view(np.uint16).reshape(H, W) == k).all()
    if rgba_bytes is not None:
        assert (rgba_bytes.reshape(H, W, 4) == oracle.colour(k, f["max_iter"], PAL)).all()
    if hist_bytes is not None:
        assert (hist_bytes.view(np.float32) == oracle.hist(k, f["max_iter"])).all()


RAGGED = [
    dict(c=0.3 + 0.5j, rect=(-2, 2, -2, 2), W=1, H=1, max_iter=100, mode=0, precision=0),
    dict(c=-0.8 + 0.156j, rect=(-2, 2, -2, 2), W=31, H=33, max_iter=100, mode=0, precision=0),
    dict(c=-0.8 + 0.156j, rect=(-2, 2, -2, 2), W=31, H=33, max_iter=300, mode=1, precision=1),
    dict(c=-2 + 0j, rect=(-2.0, 2.0, -0.25, 0.25), W=1001, H=1, max_iter=300, mode=0, precision=0),
    dict(c=0.285 + 0.01j, rect=(-1.6, 1.6, -1.6, 1.6), W=1, H=777, max_iter=1000, mode=0, precision=1),
    dict(c=-0.7269 + 0.1889j, rect=(-1.6, 1.6, -1.6, 1.6), W=97, H=53, max_iter=5000, mode=0, precision=0),
    dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=129, H=65, max_iter=255, mode=1, precision=0),
]


def _variants(prec):
    L = _lib.lib()
    n = L.jl_variant_list(prec, None, 0)
    buf = (ctypes.c_int32 * (2 * n))()
    L.jl_variant_list(prec, buf, n)
    return [None] + [(buf[2 * i], buf[2 * i + 1], 256, 0) for i in range(n)]


def _render_guarded(f, ct, variant=None, static=False):
    npx = f["W"] * f["H"]
    nb = {"u8": npx, "u16": 2 * npx}[ct]
    a = Arena([nb, 4 * npx, 4 * (f["max_iter"] + 1)])
    L = _lib.lib()
    pal = np.ascontiguousarray(PAL, np.uint8)
    cr, ci = (0.0, 0.0) if f.get("c") is None else (complex(f["c"]).real, complex(f["c"]).imag)
    ctc = {"u8": jl.JL_COUNT_U8, "u16": jl.JL_COUNT_U16}[ct]
    args = (cr, ci, _lib.Rect(*[float(v) for v in f["rect"]]), f["W"], f["H"], f["max_iter"], f["precision"],
            f["mode"], ctc, a.ptr(0), a.ptr(1), pal.ctypes.data, a.ptr(2))
    if static:
        _lib.check(L.jl_render_static(*args, None))
    elif variant is None:
        _lib.check(L.jl_render(*args, None))
    else:
        _lib.check(L.jl_render_variant(*args, *variant, 1, None))
    b = a.check_guards("jl_render %s %s variant=%s static=%s" % (f, ct, variant, static))
    return a, b


@pytest.mark.parametrize("idx", range(len(RAGGED)))
def test_render_guards(cuda, idx):
    """Single frames through jl_render, every kernel variant and the
    allocation-free entry point: nothing outside counts / RGBA / histogram."""
    f = RAGGED[idx]
    k = _oracle(f)
    for ct in ("u8", "u16") if f["max_iter"] <= 255 else ("u16",):
        for v in _variants(f["precision"]):
            a, b = _render_guarded(f, ct, variant=v)
            _check_outputs(f, k, a.region(0, b), a.region(1, b), a.region(2, b), ct)
        a, b = _render_guarded(f, ct, static=True)
        _check_outputs(f, k, a.region(0, b), a.region(1, b), a.region(2, b), ct)


@pytest.mark.parametrize("prec", [0, 1])
def test_render_guards_sweep_frame(cuda, prec):
    """A full 4096 x 4096 frame of the throughput sweep (Julia
    C = -0.7269+0.1889i, limit 1000 for binary32, 100 for binary64), uint16
    counts + RGBA8 + histogram: guards intact, and 64 sampled rows equal to
    the oracle's."""
    f = dict(c=-0.7269 + 0.1889j, rect=(-1.6, 1.6, -1.6, 1.6), W=4096, H=4096,
             max_iter=1000 if prec == 0 else 100, mode=0, precision=prec)
    a, b = _render_guarded(f, "u16")
    rows = np.sort(np.random.default_rng(5 + prec).choice(4096, 64, replace=False))
    k = oracle.render_rows(f["c"], f["rect"], f["W"], f["H"], rows, f["max_iter"], f["mode"], prec)
    got = a.region(0, b).view(np.uint16).reshape(4096, 4096)[rows]
    assert (got == k).all()
    assert (a.region(1, b).reshape(4096, 4096, 4)[rows] == oracle.colour(k, f["max_iter"], PAL)).all()


def test_map_guards(cuda):
    """Generic maps (Z^3 + C and a rational map) on ragged frames."""
    L = _lib.lib()
    pal = np.ascontiguousarray(PAL, np.uint8)
    maps = [dict(kind="power", degree=3), dict(kind="rational", num=[1, 0, 1, 0, 1], den=[1, 0, 1])]
    for m in maps:
        for f in RAGGED[:4]:
            npx = f["W"] * f["H"]
            a = Arena([2 * npx, 4 * npx, 4 * (f["max_iter"] + 1)])
            spec = jl.make_map(m)
            cr, ci = (0.0, 0.0) if f.get("c") is None else (complex(f["c"]).real, complex(f["c"]).imag)
            _lib.check(L.jl_render_map(ctypes.byref(spec), cr, ci, _lib.Rect(*[float(v) for v in f["rect"]]),
                                       f["W"], f["H"], f["max_iter"], f["precision"], f["mode"], jl.JL_COUNT_U16,
                                       a.ptr(0), a.ptr(1), pal.ctypes.data, a.ptr(2), None))
            a.check_guards("jl_render_map %s %s" % (m, f))


def _guarded_frames(frames, host=False):
    """A counts arena, an RGBA arena and a histogram arena with one region per
    frame (guards between frames), and the jl_frame array with the offsets."""
    cts = [f.get("count_type", "u16") for f in frames]
    npx = [f["W"] * f["H"] for f in frames]
    ca = Arena([(n if ct == "u8" else 2 * n) if ct else 0 for n, ct in zip(npx, cts)], host=host)
    ra = Arena([4 * n for n in npx], host=host)
    ha = Arena([4 * (f["max_iter"] + 1) if f.get("hist") else 0 for f in frames], host=host)
    arr = (_lib.Frame * len(frames))()
    for i, f in enumerate(frames):
        cr, ci = (0.0, 0.0) if f.get("c") is None else (complex(f["c"]).real, complex(f["c"]).imag)
        ctc = {None: jl.JL_COUNT_NONE, "u8": jl.JL_COUNT_U8, "u16": jl.JL_COUNT_U16}[cts[i]]
        arr[i] = _lib.Frame(cr, ci, _lib.Rect(*[float(v) for v in f["rect"]]), f["W"], f["H"], f["max_iter"],
                            f["mode"], f["precision"], ctc,
                            ca.offsets[i] if cts[i] else -1, ra.offsets[i],
                            ha.offsets[i] if f.get("hist") else -1)
    return ca, ra, ha, arr


def _batch_frames():
    fr = []
    for i, f in enumerate(RAGGED + [dict(c=0.285 + 0.01j, rect=(-1.6, 1.6, -1.6, 1.6), W=1000, H=999,
                                         max_iter=100, mode=0, precision=0)]):
        g = dict(f)
        g["count_type"] = "u8" if (g["max_iter"] <= 255 and i % 2 == 0) else "u16"
        g["hist"] = i % 3 != 1
        fr.append(g)
    return fr


@pytest.mark.parametrize("kernel", ["default", "static", "compact", "tune"])
def test_batch_guards(cuda, kernel):
    """A batch plan over ragged frames of both modes, precisions and count
    types, every output region fenced: the plan's kernels (lane refill, the
    static tile kernel, the compacting kernel with parked pixels, or the
    plan's own tuned choice) write only their frames' outputs."""
    frames = _batch_frames()
    ca, ra, ha, arr = _guarded_frames(frames)
    L = _lib.lib()
    opts = _lib.BatchOpts()
    if kernel == "static":
        opts.fp32_ppt, opts.fp32_unroll, opts.fp32_threads, opts.variant_flags = 0, 0, 256, 1
    elif kernel == "compact":
        opts.fp32_ppt, opts.fp32_unroll, opts.fp32_threads, opts.variant_flags = 0, 16, 256, 1
    elif kernel == "tune":
        opts.tune = 1
    pal = np.ascontiguousarray(PAL, np.uint8)
    h = ctypes.c_void_p()
    _lib.check(L.jl_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(frames), ca.buf.data_ptr(),
                                 ra.buf.data_ptr(), ha.buf.data_ptr(), pal.ctypes.data, ctypes.byref(opts),
                                 ctypes.byref(h)))
    try:
        for _ in range(2):
            _lib.check(L.jl_batch_launch(h, None))
        cb, rb, hb = (x.check_guards("batch %s" % kernel) for x in (ca, ra, ha))
        for i, f in enumerate(frames):
            k = _oracle(f)
            _check_outputs(f, k, ca.region(i, cb), ra.region(i, rb), ha.region(i, hb) if f["hist"] else None,
                           f["count_type"])
    finally:
        L.jl_batch_destroy(h)


def test_host_plan_guards(cuda):
    """A host plan (copies to pinned host memory overlapped with rendering;
    the last frame large enough to be rendered and copied as row bands):
    nothing lands outside each frame's host outputs."""
    frames = _batch_frames()
    frames.append(dict(c=-0.4 + 0.6j, rect=(-1.6, 1.6, -1.6, 1.6), W=2048, H=1601, max_iter=100, mode=0,
                       precision=0, count_type="u16", hist=False))
    ca, ra, ha, arr = _guarded_frames(frames, host=True)
    L = _lib.lib()
    pal = np.ascontiguousarray(PAL, np.uint8)
    h = ctypes.c_void_p()
    _lib.check(L.jl_host_plan_create(arr, len(frames), ca.buf.data_ptr(), ra.buf.data_ptr(), ha.buf.data_ptr(),
                                     pal.ctypes.data, 3, ctypes.byref(h)))
    try:
        assert L.jl_host_plan_launches(h) > len(frames)      # the last frame went out in bands
        for _ in range(2):
            _lib.check(L.jl_host_plan_run(h, None))
        cb, rb, hb = (x.check_guards("host plan") for x in (ca, ra, ha))
        for i, f in enumerate(frames):
            k = _oracle(f)
            _check_outputs(f, k, ca.region(i, cb), ra.region(i, rb), ha.region(i, hb) if f["hist"] else None,
                           f["count_type"])
    finally:
        L.jl_host_plan_destroy(h)


@pytest.mark.parametrize("n", [1, 127, 50001])
def test_surrogate_output_guards(cuda, n):
    """Forward (fused and per-layer), top-k and screening write only their
    n-row outputs."""
    from tests.test_gpu_mlp import Model, setup_model
    p, B = setup_model(6)
    md = Model(p, B)
    import torch
    c = torch.from_numpy(wl.survey_c(n, seed=31)).cuda()
    L = md.L
    try:
        for fn in (L.jl_model_forward, L.jl_model_forward_layered):
            a = Arena([n * 101 * 4, n * 4])
            _lib.check(fn(md.h, c.data_ptr(), n, a.ptr(0), a.ptr(1), None))
            a.check_guards("forward n=%d" % n)
        k = min(n, 1000)
        a = Arena([k * 4, k * 4, n * 4])
        _lib.check(L.jl_survey(md.h, c.data_ptr(), n, k, a.ptr(0), a.ptr(1), a.ptr(2), None))
        _lib.check(L.jl_survey(md.h, c.data_ptr(), n, k, a.ptr(0), a.ptr(1), a.ptr(2), None))
        b = a.check_guards("survey n=%d" % n)
        s = a.region(2, b).view(np.float32)
        idx = a.region(0, b).view(np.int32)
        from oracle import mlp
        assert (idx == mlp.top_k(s, k)).all()
        t = Arena([k * 4, k * 4])
        sd = torch.from_numpy(s.copy()).cuda()
        _lib.check(L.jl_topk(sd.data_ptr(), n, k, t.ptr(0), t.ptr(1), None))
        t.check_guards("topk n=%d" % n)
    finally:
        md.close()
