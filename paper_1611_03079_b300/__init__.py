"""B300-native escape-time fractal renderer and parameter-space surveyor.

Python binding of libjl.so (include/jl.h): argument marshalling only; every
step of the rendering path runs in the library's CUDA kernels.  PyTorch is
used for device memory and streams.  Paper: "Fractal Art Generation using
GPUs" (arXiv:1611.03079), Sec. 2 (escape-time algorithm, region covering,
colour levels) and Sec. 3 (Mandelbrot mode, deep zoom, parameter paths).
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import (JL_AUTO, JL_COUNT_NONE, JL_COUNT_U8, JL_COUNT_U16, JL_FP32, JL_FP64, JL_JULIA,
                   JL_MANDELBROT, JLError, Rect, check)

__all__ = ["render", "render_to_host", "select_precision", "default_palette", "JLError",
           "JL_FP32", "JL_FP64", "JL_AUTO", "JL_JULIA", "JL_MANDELBROT", "JL_COUNT_NONE",
           "JL_COUNT_U8", "JL_COUNT_U16", "version"]

_PREC = {"fp32": JL_FP32, "fp64": JL_FP64, "auto": JL_AUTO, JL_FP32: JL_FP32, JL_FP64: JL_FP64,
         JL_AUTO: JL_AUTO}
_MODE = {"julia": JL_JULIA, "mandelbrot": JL_MANDELBROT, JL_JULIA: JL_JULIA,
         JL_MANDELBROT: JL_MANDELBROT}
_CT = {None: JL_COUNT_NONE, "none": JL_COUNT_NONE, "u8": JL_COUNT_U8, "u16": JL_COUNT_U16,
       JL_COUNT_NONE: JL_COUNT_NONE, JL_COUNT_U8: JL_COUNT_U8, JL_COUNT_U16: JL_COUNT_U16}


def version():
    return _lib.lib().jl_version().decode()


def _rect(rect):
    xmin, xmax, ymin, ymax = (float(v) for v in rect)
    return Rect(xmin, xmax, ymin, ymax)


def select_precision(rect, width, height):
    """JL_FP32 or JL_FP64 by the library's deep-zoom precision rule."""
    r = _lib.lib().jl_select_precision(_rect(rect), int(width), int(height))
    if r < 0:
        raise JLError(_lib.JL_EINVAL, "invalid rect or size")
    return r


def default_palette():
    """The built-in 256 x 4 uint8 palette (entry 255 = opaque black)."""
    out = np.zeros((256, 4), dtype=np.uint8)
    check(_lib.lib().jl_default_palette(out.ctypes.data))
    return out


def _palette_ptr(palette):
    if palette is None:
        return None, None
    p = np.ascontiguousarray(np.asarray(palette, dtype=np.uint8).reshape(256, 4))
    return p, p.ctypes.data


def _c(c):
    if c is None:
        return 0.0, 0.0
    c = complex(c)
    return c.real, c.imag


def render(c, rect, width, height, max_iter=100, precision="fp32", mode="julia", count_type="u16",
           rgba=True, hist=False, palette=None, out=None, stream=None, variant=None):
    """Render one frame on the current CUDA device.

    Returns a dict with 'counts' (torch uint8/uint16, shape (H, W)), 'rgba'
    (torch uint8, (H, W, 4)) and 'hist' (torch float32, max_iter + 1) for the
    outputs requested.  `out` may supply preallocated tensors under the same
    keys.  `variant` = (ppt, unroll, threads, ctas_per_sm) selects a kernel
    variant explicitly.  Asynchronous on `stream` (default: torch's current
    stream).
    """
    import torch

    prec, md, ct = _PREC[precision], _MODE[mode], _CT[count_type]
    W, H = int(width), int(height)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = dict(out or {})
    if ct != JL_COUNT_NONE and "counts" not in out:
        out["counts"] = torch.empty((H, W), dtype=torch.uint8 if ct == JL_COUNT_U8 else torch.uint16,
                                    device=dev)
    if rgba and "rgba" not in out:
        out["rgba"] = torch.empty((H, W, 4), dtype=torch.uint8, device=dev)
    if hist and "hist" not in out:
        out["hist"] = torch.empty((int(max_iter) + 1,), dtype=torch.float32, device=dev)
    cnt_ptr = out["counts"].data_ptr() if ct != JL_COUNT_NONE else None
    rgba_ptr = out["rgba"].data_ptr() if rgba else None
    hist_ptr = out["hist"].data_ptr() if hist else None
    pal, pal_ptr = _palette_ptr(palette)
    st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    cr, ci = _c(c)
    L = _lib.lib()
    if variant is None:
        rc = L.jl_render(cr, ci, _rect(rect), W, H, int(max_iter), prec, md, ct, cnt_ptr, rgba_ptr, pal_ptr,
                         hist_ptr, st)
    else:
        ppt, unroll, threads, per_sm = (int(v) for v in variant)
        rc = L.jl_render_variant(cr, ci, _rect(rect), W, H, int(max_iter), prec, md, ct, cnt_ptr, rgba_ptr,
                                 pal_ptr, hist_ptr, ppt, unroll, threads, per_sm, st)
    check(rc)
    del pal
    return out


def render_to_host(c, rect, width, height, max_iter=100, precision="fp32", mode="julia",
                   count_type="u16", rgba=True, hist=False, palette=None, out=None, stream=None):
    """Render one frame into host (numpy) buffers through jl_render_to_host;
    synchronous.  `out` may supply preallocated (e.g. pinned) numpy arrays."""
    prec, md, ct = _PREC[precision], _MODE[mode], _CT[count_type]
    W, H = int(width), int(height)
    out = dict(out or {})
    if ct != JL_COUNT_NONE and "counts" not in out:
        out["counts"] = np.empty((H, W), dtype=np.uint8 if ct == JL_COUNT_U8 else np.uint16)
    if rgba and "rgba" not in out:
        out["rgba"] = np.empty((H, W, 4), dtype=np.uint8)
    if hist and "hist" not in out:
        out["hist"] = np.empty((int(max_iter) + 1,), dtype=np.float32)

    def ptr(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        return a.ctypes.data

    pal, pal_ptr = _palette_ptr(palette)
    st = 0
    if stream is not None:
        st = stream.cuda_stream
    cr, ci = _c(c)
    rc = _lib.lib().jl_render_to_host(cr, ci, _rect(rect), W, H, int(max_iter), prec, md, ct,
                                      ptr(out.get("counts")), ptr(out.get("rgba") if rgba else None),
                                      pal_ptr, ptr(out.get("hist") if hist else None), st)
    check(rc)
    del pal
    return out
