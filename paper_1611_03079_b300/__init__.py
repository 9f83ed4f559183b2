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
    keys.  `variant` = (ppt, unroll, threads, ctas_per_sm) selects a
    kernel variant explicitly.  Asynchronous on `stream` (default: torch's current
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
        v = [int(x) for x in variant] + [0] * (4 - len(variant))
        ppt, unroll, threads, per_sm = v[:4]
        rc = L.jl_render_variant(cr, ci, _rect(rect), W, H, int(max_iter), prec, md, ct, cnt_ptr, rgba_ptr,
                                 pal_ptr, hist_ptr, ppt, unroll, threads, per_sm, st)
    check(rc)
    del pal
    return out


def make_map(m):
    """jl_map from a description: {"kind": "power", "degree": d} or
    {"kind": "rational", "num": [a_0, ..., a_n], "den": [b_0, ..., b_m]}
    (complex coefficients, constant term first), with optional "bailout"
    (escape radius squared, default 4.0) and "z0" (Z_0 in parameter-plane
    mode, default 0)."""
    s = _lib.Map()
    s.bailout = float(m.get("bailout", 4.0))
    z0 = complex(m.get("z0", 0.0))
    s.z0r, s.z0i = z0.real, z0.imag
    if m["kind"] == "power":
        s.kind, s.degree = 0, int(m["degree"])
    elif m["kind"] == "rational":
        num, den = [complex(v) for v in m["num"]], [complex(v) for v in m["den"]]
        if not (1 <= len(num) <= 9 and 1 <= len(den) <= 9):
            raise ValueError("a rational map takes 1..9 coefficients for each of P and Q")
        s.kind, s.num_degree, s.den_degree = 1, len(num) - 1, len(den) - 1
        for k, v in enumerate(num):
            s.num[2 * k], s.num[2 * k + 1] = v.real, v.imag
        for k, v in enumerate(den):
            s.den[2 * k], s.den[2 * k + 1] = v.real, v.imag
    else:
        raise ValueError("map kind must be 'power' or 'rational'")
    return s


def render_map(m, c, rect, width, height, max_iter=100, precision="fp32", mode="julia", count_type="u16",
               rgba=True, hist=False, palette=None, out=None, stream=None):
    """Render one frame of a generic map Z <- F(Z) + C (jl_render_map); `m`
    as for make_map, other arguments and the result as for render()."""
    import torch

    spec = make_map(m)
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
    pal, pal_ptr = _palette_ptr(palette)
    st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    cr, ci = _c(c)
    check(_lib.lib().jl_render_map(ctypes.byref(spec), cr, ci, _rect(rect), W, H, int(max_iter), prec, md, ct,
                                   out["counts"].data_ptr() if ct != JL_COUNT_NONE else None,
                                   out["rgba"].data_ptr() if rgba else None, pal_ptr,
                                   out["hist"].data_ptr() if hist else None, st))
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


# ---------------------------------------------------------------------------
# Batches (jl_batch_*) and the autotuner (jl_autotune, jl_tune_*)
# ---------------------------------------------------------------------------
def _frame_struct(f, counts_off, rgba_off, hist_off):
    c = f.get("c")
    cr, ci = _c(c)
    return _lib.Frame(cr, ci, _rect(f["rect"]), int(f["W"]), int(f["H"]), int(f["max_iter"]),
                      _MODE[f.get("mode", "julia")], _PREC[f.get("precision", "fp32")],
                      _CT[f.get("count_type")], counts_off, rgba_off, hist_off)


def _layout(frames):
    """Byte offsets of every frame's outputs in flat counts / RGBA8 /
    histogram buffers (-1 = none) and the three buffer sizes."""
    c_off, r_off, h_off = [], [], []
    cb = rb = hb = 0
    for f in frames:
        ct = _CT[f.get("count_type")]
        npx = int(f["W"]) * int(f["H"])
        if ct != JL_COUNT_NONE:
            cb = (cb + 1) & ~1
            c_off.append(cb)
            cb += npx * (1 if ct == JL_COUNT_U8 else 2)
        else:
            c_off.append(-1)
        if f.get("rgba", True):
            r_off.append(rb)
            rb += npx * 4
        else:
            r_off.append(-1)
        if f.get("hist", False):
            h_off.append(hb)
            hb += (int(f["max_iter"]) + 1) * 4
        else:
            h_off.append(-1)
    return c_off, r_off, h_off, cb, rb, hb


class HostFrames:
    """Frames rendered into (pinned) host memory through a host plan
    (jl_host_plan_*): copies to the host overlap with rendering, `depth`
    device output slots (0 = one per frame up to 16).  `frames` as for Batch.  The host buffers are allocated
    once (page-locked through torch) and the plan (coordinate tables, device
    slots, streams) once; every render() call renders all frames again.
    counts(i), rgba(i) and hist(i) return numpy views of frame i."""

    def __init__(self, frames, palette=None, depth=0):
        import torch
        self._L = _lib.lib()
        self.frames = list(frames)
        self.depth = int(depth)
        self._c_off, self._r_off, self._h_off, cb, rb, hb = _layout(self.frames)
        self.counts_buf = torch.empty(max(cb, 2), dtype=torch.uint8, pin_memory=True).numpy()
        self.rgba_buf = torch.empty(max(rb, 4), dtype=torch.uint8, pin_memory=True).numpy()
        self.hist_buf = torch.empty(max(hb // 4, 1), dtype=torch.float32, pin_memory=True).numpy()
        self._arr = (_lib.Frame * len(self.frames))(
            *[_frame_struct(f, self._c_off[i], self._r_off[i], self._h_off[i]) for i, f in enumerate(self.frames)])
        self._pal, self._pal_ptr = _palette_ptr(palette)
        self.d2h_bytes = sum(cb_ for cb_ in (cb, rb, hb))
        h = ctypes.c_void_p()
        check(self._L.jl_host_plan_create(self._arr, len(self.frames), self.counts_buf.ctypes.data,
                                          self.rgba_buf.ctypes.data, self.hist_buf.ctypes.data, self._pal_ptr,
                                          self.depth, ctypes.byref(h)))
        self._h = h

    def render(self, stream=None):
        import torch
        st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        check(self._L.jl_host_plan_run(self._h, st))

    def launches(self):
        """Escape-kernel launches per render(): frames plus the last frame's row bands."""
        return int(self._L.jl_host_plan_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._L.jl_host_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def counts(self, i):
        f, o = self.frames[i], self._c_off[i]
        if o < 0:
            return None
        npx = int(f["W"]) * int(f["H"])
        if _CT[f.get("count_type")] == JL_COUNT_U8:
            return self.counts_buf[o:o + npx].reshape(int(f["H"]), int(f["W"]))
        return self.counts_buf[o:o + 2 * npx].view(np.uint16).reshape(int(f["H"]), int(f["W"]))

    def rgba(self, i):
        f, o = self.frames[i], self._r_off[i]
        if o < 0:
            return None
        npx = int(f["W"]) * int(f["H"])
        return self.rgba_buf[o:o + 4 * npx].reshape(int(f["H"]), int(f["W"]), 4)

    def hist(self, i):
        o = self._h_off[i]
        if o < 0:
            return None
        return self.hist_buf[o // 4:o // 4 + int(self.frames[i]["max_iter"]) + 1]


class Batch:
    """A batch plan: frames rendered together by one CUDA-graph launch.

    `frames` are dicts with keys c, rect, W, H, max_iter, mode, precision,
    count_type (None for no counts), and optional rgba (default True) and hist
    (default False).  Outputs are allocated here as flat device buffers;
    `counts(i)`, `rgba(i)` and `hist(i)` return per-frame views.  `tune=True`
    lets the plan time candidate kernels on its own frames at creation.
    `certify=False` turns off the certified passes of binary64 frames,
    `certify2=False` only the double-float one;
    `phases=True` records timing events around the kernels (`phase_ms`).
    """

    def __init__(self, frames, palette=None, chunk_len=0, variants=None, cycle_budget=0, tune=False,
                 certify=True, certify2=True, phases=False):
        import torch
        self._L = _lib.lib()
        self.frames = list(frames)
        n = len(self.frames)
        self._c_off, self._r_off, self._h_off = [], [], []
        cb = rb = hb = 0
        for f in self.frames:
            ct = _CT[f.get("count_type")]
            npx = int(f["W"]) * int(f["H"])
            if ct != JL_COUNT_NONE:
                cb = (cb + 1) & ~1
                self._c_off.append(cb)
                cb += npx * (1 if ct == JL_COUNT_U8 else 2)
            else:
                self._c_off.append(-1)
            if f.get("rgba", True):
                self._r_off.append(rb)
                rb += npx * 4
            else:
                self._r_off.append(-1)
            if f.get("hist", False):
                self._h_off.append(hb)
                hb += (int(f["max_iter"]) + 1) * 4
            else:
                self._h_off.append(-1)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.counts_buf = torch.empty(max(cb, 2), dtype=torch.uint8, device=dev)
        self.rgba_buf = torch.empty(max(rb, 4), dtype=torch.uint8, device=dev)
        self.hist_buf = torch.empty(max(hb // 4, 1), dtype=torch.float32, device=dev)
        arr = (_lib.Frame * n)(*[_frame_struct(f, self._c_off[i], self._r_off[i], self._h_off[i])
                                 for i, f in enumerate(self.frames)])
        opts = _lib.BatchOpts()
        opts.chunk_len = int(chunk_len)
        if variants:
            if "fp32" in variants:
                opts.fp32_ppt, opts.fp32_unroll, opts.fp32_threads = (int(v) for v in variants["fp32"])
                opts.variant_flags |= 1
            if "fp64" in variants:
                v64 = [int(v) for v in variants["fp64"]]
                opts.fp64_ppt, opts.fp64_unroll, opts.fp64_threads = v64[:3]
                opts.variant_flags |= 2
        if not certify:
            opts.variant_flags |= 4
        if phases:
            opts.variant_flags |= 8
        if not certify2:
            opts.variant_flags |= 16
        opts.cycle_budget = int(cycle_budget)
        opts.tune = 1 if tune else 0
        pal, pal_ptr = _palette_ptr(palette)
        h = ctypes.c_void_p()
        check(self._L.jl_batch_create(ctypes.cast(arr, ctypes.c_void_p), n, self.counts_buf.data_ptr(),
                                      self.rgba_buf.data_ptr(), self.hist_buf.data_ptr(), pal_ptr,
                                      ctypes.byref(opts), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        import torch
        st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        check(self._L.jl_batch_launch(self._h, st))

    def status(self, stream=None):
        import torch
        st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        v = ctypes.c_int32(0)
        check(self._L.jl_batch_status(self._h, st, ctypes.byref(v)))
        return v.value

    def variant(self, precision):
        """(ppt, unroll, threads) of the kernel the plan uses for
        precision 0 (binary32) or 1 (binary64)."""
        v = [ctypes.c_int32(0) for _ in range(3)]
        check(self._L.jl_batch_variant(self._h, int(precision), *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def precisions(self):
        n = len(self.frames)
        buf = (ctypes.c_int32 * n)()
        self._L.jl_batch_precisions(self._h, buf, n)
        return list(buf)

    def pixels(self):
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        check(self._L.jl_batch_pixels(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def cert_stats(self, stream=None):
        """For the last launch's binary64 frames: (pixels left by the binary32
        pass, pixels left to the binary64 kernel, iterations the double-float
        pass settled, iterations the binary64 kernel ran, tests the binary32
        pass decided, tests the double-float pass decided)."""
        import torch
        st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        v = (ctypes.c_int64 * 6)()
        check(self._L.jl_batch_cert_stats(self._h, st, v))
        return tuple(int(x) for x in v)

    def phase_ms(self):
        """Device ms of the last completed launch: [binary32 kernel, binary32
        certified pass, double-float pass, binary64 kernel] (-1 where absent);
        needs phases=True."""
        ms = (ctypes.c_float * 4)()
        check(self._L.jl_batch_phase_ms(self._h, ms))
        return [float(v) for v in ms]

    def counts(self, i):
        import torch
        f = self.frames[i]
        o = self._c_off[i]
        if o < 0:
            return None
        npx = int(f["W"]) * int(f["H"])
        if _CT[f.get("count_type")] == JL_COUNT_U8:
            return self.counts_buf[o:o + npx].view(int(f["H"]), int(f["W"]))
        return self.counts_buf[o:o + 2 * npx].view(torch.int16).view(int(f["H"]), int(f["W"]))

    def rgba(self, i):
        f = self.frames[i]
        o = self._r_off[i]
        if o < 0:
            return None
        npx = int(f["W"]) * int(f["H"])
        return self.rgba_buf[o:o + 4 * npx].view(int(f["H"]), int(f["W"]), 4)

    def hist(self, i):
        o = self._h_off[i]
        if o < 0:
            return None
        return self.hist_buf[o // 4:o // 4 + int(self.frames[i]["max_iter"]) + 1]

    def close(self):
        if getattr(self, "_h", None):
            self._L.jl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(precision="fp32", max_iter=100, calib=None, reps=3):
    """Run the launch-shape autotuner; returns the chosen variant as a dict."""
    L = _lib.lib()
    res = _lib.TuneResult()
    if calib:
        arr = (_lib.Frame * len(calib))(*[_frame_struct(f, -1, -1, -1) for f in calib])
        ptr, n = ctypes.cast(arr, ctypes.c_void_p), len(calib)
    else:
        ptr, n = None, 0
    check(L.jl_autotune(_PREC[precision], int(max_iter), ptr, n, int(reps), ctypes.byref(res)))
    return {"ppt": res.ppt, "unroll": res.unroll, "threads": res.threads, "ctas_per_sm": res.ctas_per_sm,
            "ms": res.ms, "candidates": res.candidates}


def tune_get(precision="fp32", max_iter=100):
    res = _lib.TuneResult()
    check(_lib.lib().jl_tune_get(_PREC[precision], int(max_iter), ctypes.byref(res)))
    return {"ppt": res.ppt, "unroll": res.unroll, "threads": res.threads, "ctas_per_sm": res.ctas_per_sm,
            "tuned": bool(res.candidates), "ms": res.ms, "candidates": res.candidates}


def tune_clear():
    check(_lib.lib().jl_tune_clear())


def tune_save(path):
    check(_lib.lib().jl_tune_save(str(path).encode()))


def tune_load(path):
    check(_lib.lib().jl_tune_load(str(path).encode()))
