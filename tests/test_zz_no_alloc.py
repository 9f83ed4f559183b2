"""jl_render_static: the render entry point that allocates nothing, for
callers that cannot allocate device memory while rendering (a real-time loop
that must not stall on an allocation, or a process whose device memory is
reserved up front by another allocator).  Its output must equal jl_render's
bit for bit (escape counts are integers; RGBA8 bytes and histogram values are
compared exactly, as in the other render tests), on two calls in a row, since
the second call finds the first call's leftovers in the shared static array.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FRAMES = [
    # (cr, ci, rect, W, H, max_iter, precision, mode)
    (-0.7269, 0.1889, (-1.6, 1.6, -1.6, 1.6), 1000, 700, 1000, 0, 0),
    (0.0, 0.0, (-2.5, 1.0, -1.75, 1.75), 513, 777, 300, 1, 1),
]


def _call(fn, frame, torch, dev, pal):
    from paper_1611_03079_b300 import _lib
    cr, ci, rect, W, H, mi, prec, mode = frame
    counts = torch.zeros((H, W), dtype=torch.int16, device=dev)
    rgba = torch.zeros((H, W, 4), dtype=torch.uint8, device=dev)
    hist = torch.zeros((mi + 1,), dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream().cuda_stream
    rc = fn(cr, ci, _lib.Rect(*rect), W, H, mi, prec, mode, _lib.JL_COUNT_U16, counts.data_ptr(),
            rgba.data_ptr(), pal.ctypes.data, hist.data_ptr(), st)
    _lib.check(rc)
    torch.cuda.synchronize()
    return counts.cpu().numpy(), rgba.cpu().numpy(), hist.cpu().numpy()


def test_static_matches_jl_render_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_03079_b300 import _lib, workloads as wl
    L = _lib.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    pal = np.ascontiguousarray(wl.random_palette(7))
    for frame in FRAMES + FRAMES[::-1]:
        ref = _call(L.jl_render, frame, torch, dev, pal)
        first = _call(L.jl_render_static, frame, torch, dev, pal)
        second = _call(L.jl_render_static, frame, torch, dev, pal)
        for got in (first, second):
            for a, b in zip(ref, got):
                assert a.shape == b.shape
                assert (a == b).all()


def test_static_rejects_oversized_frames():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_03079_b300 import _lib
    L = _lib.lib()
    # binary64 tables need (W + H) * 8 bytes: 40000 + 1 columns is beyond the limit.
    # The output buffer is full size, so nothing could go out of bounds even
    # if the size check were missing.
    counts = torch.zeros((1, 40000), dtype=torch.int16, device="cuda")
    rc = L.jl_render_static(0.0, 0.0, _lib.Rect(-2, 2, -2, 2), 40000, 1, 100, 1, 0, _lib.JL_COUNT_U16,
                            ctypes.c_void_p(counts.data_ptr()), None, None, None, None)
    torch.cuda.synchronize()
    assert rc == _lib.JL_EINVAL
    msg = L.jl_last_error().decode()
    assert "static scratch" in msg and "32736" in msg


def _pool():
    """The device's default memory pool (the one stream-ordered allocations
    such as jl_render's scratch come from), through the driver API."""
    from cuda.bindings import driver as drv
    drv.cuInit(0)
    err, dev = drv.cuDeviceGet(0)
    assert err == drv.CUresult.CUDA_SUCCESS
    err, pool = drv.cuDeviceGetDefaultMemPool(dev)
    assert err == drv.CUresult.CUDA_SUCCESS
    attr = drv.CUmemPool_attribute.CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def reset():
        (e,) = drv.cuMemPoolSetAttribute(pool, attr, drv.cuuint64_t(0))
        assert e == drv.CUresult.CUDA_SUCCESS

    def high():
        e, v = drv.cuMemPoolGetAttribute(pool, attr)
        assert e == drv.CUresult.CUDA_SUCCESS
        return int(v)
    return reset, high


def test_static_allocates_nothing():
    """The pool's high-water mark of memory in use stays where it was across
    jl_render_static calls, while jl_render (which takes its scratch from the
    pool) raises it: the positive control that shows the measurement works."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_03079_b300 import _lib, workloads as wl
    L = _lib.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    pal = np.ascontiguousarray(wl.random_palette(7))
    reset, high = _pool()
    for frame in FRAMES:
        _call(L.jl_render_static, frame, torch, dev, pal)      # set-up done before measuring
        torch.cuda.synchronize()
        reset()
        h0 = high()
        _call(L.jl_render_static, frame, torch, dev, pal)
        _call(L.jl_render_static, frame, torch, dev, pal)
        torch.cuda.synchronize()
        assert high() == h0
        _call(L.jl_render, frame, torch, dev, pal)
        torch.cuda.synchronize()
        assert high() > h0


@pytest.mark.parametrize("prec,limit", [(1, 32736), (0, 65472)])
def test_static_size_limit_exact(prec, limit):
    """width + height at the stated limit is rendered (and equals jl_render);
    one more is refused with JL_EINVAL."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_03079_b300 import _lib
    L = _lib.lib()
    for W, expect in ((limit - 1, _lib.JL_OK), (limit, _lib.JL_EINVAL)):
        outs = []
        for fn in (L.jl_render_static, L.jl_render) if expect == _lib.JL_OK else (L.jl_render_static,):
            counts = torch.zeros((1, W), dtype=torch.int16, device="cuda")
            rc = fn(-0.8, 0.156, _lib.Rect(-2, 2, -0.5, 0.5), W, 1, 100, prec, 0, _lib.JL_COUNT_U16,
                    ctypes.c_void_p(counts.data_ptr()), None, None, None, None)
            torch.cuda.synchronize()
            assert rc == expect, (W, rc, L.jl_last_error())
            outs.append(counts.cpu().numpy())
        if expect == _lib.JL_OK:
            assert (outs[0] == outs[1]).all()
