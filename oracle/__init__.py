"""CPU oracle for the escape-time path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference`` arm) may import this package.
The product library never imports, links or calls it; it shares no code with
the CUDA sources (``paper_1611_03079_b300/csrc``) and the CUDA path shares none
with it.  Seeded inputs come from ``paper_1611_03079_b300.workloads``, which
holds no arithmetic of the method.

Contents
  render / colour / hist / escape_point : the C oracle (jl_oracle.c), escape
      time for Z <- Z^2 + C (paper Sec. 2; Mandelbrot mode Sec. 3), colour
      levels and the normalised escape-count histogram;
  precision_for_view : the binary32 / binary64 selection rule for deep zooms
      (Sec. 3 deep zoom; threshold 1000 binary32 ulps of the largest coordinate);
  render_map / map_escape_point / map_step : generic maps Z <- Z^d + C and
      Z <- P(Z)/Q(Z) + C (jl_oracle_maps.c; Sec. 2 "other functions", Fig. 4);
  mlp (submodule) : the surrogate network in float64 numpy.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        vp = ctypes.c_void_p
        lib.jlo_render.argtypes = [d, d, d, d, d, d, i32, i32, i32, i32, i32, vp, i32]
        lib.jlo_render.restype = ctypes.c_int
        lib.jlo_render_rows.argtypes = [d, d, d, d, d, d, i32, i32, i32, i32, i32, i32, i32, vp]
        lib.jlo_render_rows.restype = ctypes.c_int
        lib.jlo_render_strided.argtypes = [d, d, d, d, d, d, i32, i32, i32, i32, i32, i32, i32, i32, vp, i32]
        lib.jlo_render_strided.restype = ctypes.c_int
        lib.jlo_escape_point.argtypes = [d, d, d, d, i32, i32]
        lib.jlo_escape_point.restype = i32
        lib.jlo_colour.argtypes = [vp, i64, i32, vp, vp]
        lib.jlo_colour.restype = ctypes.c_int
        lib.jlo_hist.argtypes = [vp, i64, i32, vp]
        lib.jlo_hist.restype = ctypes.c_int
        lib.jlo_render_map.argtypes = [vp, d, d, d, d, d, d, i32, i32, i32, i32, i32, vp, i32]
        lib.jlo_render_map.restype = ctypes.c_int
        lib.jlo_map_escape_point.argtypes = [vp, d, d, d, d, i32, i32]
        lib.jlo_map_escape_point.restype = i32
        lib.jlo_map_step.argtypes = [vp, d, d, d, d, i32, vp]
        lib.jlo_map_step.restype = ctypes.c_int
        _lib = lib
    return _lib


JULIA, MANDELBROT = 0, 1
FP32, FP64 = 0, 1


def render(c, rect, W, H, max_iter=100, mode=JULIA, precision=FP32, threads=None):
    """Escape counts (uint16, shape (H, W), row 0 at y = ymin) of a W x H grid over
    rect = (xmin, xmax, ymin, ymax).  Paper Sec. 2 (region covering, escape time,
    limit 100) and Sec. 3 (Mandelbrot mode: Z_0 = 0, C = pixel)."""
    lib = _load()
    out = np.zeros((H, W), dtype=np.uint16)
    cr, ci = (complex(c).real, complex(c).imag) if c is not None else (0.0, 0.0)
    xmin, xmax, ymin, ymax = (float(v) for v in rect)
    if threads is None:
        threads = min(os.cpu_count() or 1, 64)
    rc = lib.jlo_render(cr, ci, xmin, xmax, ymin, ymax, int(W), int(H), int(max_iter), int(mode),
                        int(precision), out.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError("jlo_render: invalid arguments")
    return out


def render_rows(c, rect, W, H, rows, max_iter=100, mode=JULIA, precision=FP32):
    """Escape counts of the listed rows of the W x H frame (uint16, shape
    (len(rows), W)); same arithmetic as render()."""
    lib = _load()
    cr, ci = (complex(c).real, complex(c).imag) if c is not None else (0.0, 0.0)
    xmin, xmax, ymin, ymax = (float(v) for v in rect)
    out = np.zeros((len(rows), W), dtype=np.uint16)
    for k, j in enumerate(rows):
        row = np.zeros((1, W), dtype=np.uint16)
        rc = lib.jlo_render_rows(cr, ci, xmin, xmax, ymin, ymax, int(W), int(H), int(max_iter), int(mode),
                                 int(precision), int(j), int(j) + 1, row.ctypes.data)
        if rc != 0:
            raise ValueError("jlo_render_rows: invalid arguments")
        out[k] = row[0]
    return out


def render_strided(c, rect, W, H, row_start, row_stride, n_rows, max_iter=100, mode=JULIA,
                   precision=FP32, threads=None):
    """Rows row_start + k*row_stride (k < n_rows) of the W x H frame, threaded;
    uint16 (n_rows, W).  Same arithmetic as render()."""
    lib = _load()
    cr, ci = (complex(c).real, complex(c).imag) if c is not None else (0.0, 0.0)
    xmin, xmax, ymin, ymax = (float(v) for v in rect)
    if threads is None:
        threads = min(os.cpu_count() or 1, 64)
    out = np.zeros((n_rows, W), dtype=np.uint16)
    rc = lib.jlo_render_strided(cr, ci, xmin, xmax, ymin, ymax, int(W), int(H), int(max_iter), int(mode),
                                int(precision), int(row_start), int(row_stride), int(n_rows), out.ctypes.data,
                                int(threads))
    if rc != 0:
        raise ValueError("jlo_render_strided: invalid arguments")
    return out


def escape_point(z0, c, max_iter=100, precision=FP32):
    """Escape count of one starting point z0 under Z <- Z^2 + c (Sec. 2), both
    rounded once to the working precision."""
    lib = _load()
    z0, c = complex(z0), complex(c)
    return int(lib.jlo_escape_point(z0.real, z0.imag, c.real, c.imag, int(max_iter), int(precision)))


def colour(counts, max_iter, palette):
    """RGBA8 image (shape counts.shape + (4,)) from counts and a 256 x 4 uint8
    palette: entry 255 where count == max_iter, else (count * 255) // max_iter
    (Sec. 2 colour levels)."""
    lib = _load()
    counts = np.ascontiguousarray(counts, dtype=np.uint16)
    palette = np.ascontiguousarray(palette, dtype=np.uint8).reshape(256, 4)
    out = np.zeros(counts.shape + (4,), dtype=np.uint8)
    rc = lib.jlo_colour(counts.ctypes.data, counts.size, int(max_iter), palette.ctypes.data,
                        out.ctypes.data)
    if rc != 0:
        raise ValueError("jlo_colour: invalid arguments")
    return out


def hist(counts, max_iter):
    """Normalised escape-count histogram, max_iter + 1 float32 bins; bin b holds
    #{count == b} / #pixels, the quotient rounded once from binary64."""
    lib = _load()
    counts = np.ascontiguousarray(counts, dtype=np.uint16)
    out = np.zeros(int(max_iter) + 1, dtype=np.float32)
    rc = lib.jlo_hist(counts.ctypes.data, counts.size, int(max_iter), out.ctypes.data)
    if rc != 0:
        raise ValueError("jlo_hist: invalid arguments")
    return out


def ulp32(v):
    """Spacing of binary32 numbers at |v| (the ulp of the float nearest |v|)."""
    f = np.float32(abs(v))
    return float(np.spacing(f))


def precision_for_view(rect, W, H, factor=1000.0):
    """Precision rule for deep zooms (Sec. 3): binary64 when the smaller pixel
    spacing is below `factor` binary32 ulps of the largest coordinate magnitude
    of the view, else binary32.  Returns FP32 or FP64."""
    xmin, xmax, ymin, ymax = (float(v) for v in rect)
    dx = (xmax - xmin) / W
    dy = (ymax - ymin) / H
    m = max(abs(xmin), abs(xmax), abs(ymin), abs(ymax))
    return FP64 if min(dx, dy) < factor * ulp32(m) else FP32


def hist_l1(p, q):
    """L1 distance sum_b |p_b - q_b| between histograms (last axis), float64."""
    return np.abs(np.asarray(p, np.float64) - np.asarray(q, np.float64)).sum(axis=-1)


class _Map(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("degree", ctypes.c_int32), ("num_degree", ctypes.c_int32),
                ("den_degree", ctypes.c_int32), ("num", ctypes.c_double * 18), ("den", ctypes.c_double * 18),
                ("bailout", ctypes.c_double), ("z0r", ctypes.c_double), ("z0i", ctypes.c_double)]


def _map_struct(m):
    """m: {"kind": "power", "degree": d} or {"kind": "rational", "num": [a_0..a_n],
    "den": [b_0..b_m]} (complex coefficients, constant term first), with optional
    "bailout" (default 4.0) and "z0" (parameter-plane start, default 0)."""
    s = _Map()
    s.bailout = float(m.get("bailout", 4.0))
    z0 = complex(m.get("z0", 0.0))
    s.z0r, s.z0i = z0.real, z0.imag
    if m["kind"] == "power":
        s.kind, s.degree = 0, int(m["degree"])
    elif m["kind"] == "rational":
        s.kind = 1
        num, den = [complex(v) for v in m["num"]], [complex(v) for v in m["den"]]
        if not (1 <= len(num) <= 9 and 1 <= len(den) <= 9):
            raise ValueError("rational map: 1..9 coefficients each")
        s.num_degree, s.den_degree = len(num) - 1, len(den) - 1
        for k, v in enumerate(num):
            s.num[2 * k], s.num[2 * k + 1] = v.real, v.imag
        for k, v in enumerate(den):
            s.den[2 * k], s.den[2 * k + 1] = v.real, v.imag
    else:
        raise ValueError("unknown map kind")
    return s


def render_map(m, c, rect, W, H, max_iter=100, mode=JULIA, precision=FP32, threads=None):
    """Escape counts (uint16, (H, W)) of a grid under a generic map (see
    _map_struct); region covering and count rule as in render()."""
    lib = _load()
    out = np.zeros((H, W), dtype=np.uint16)
    s = _map_struct(m)
    c = complex(c)
    nt = threads if threads else (os.cpu_count() or 1)
    rc = lib.jlo_render_map(ctypes.byref(s), c.real, c.imag, *map(float, rect), W, H, max_iter, mode, precision,
                            out.ctypes.data, nt)
    if rc != 0:
        raise ValueError("jlo_render_map: invalid arguments")
    return out


def map_escape_point(m, z0, c, max_iter, precision=FP32):
    """Escape count from Z_0 = z0 with constant c under a generic map."""
    s = _map_struct(m)
    z0, c = complex(z0), complex(c)
    n = _load().jlo_map_escape_point(ctypes.byref(s), z0.real, z0.imag, c.real, c.imag, max_iter, precision)
    if n < 0:
        raise ValueError("jlo_map_escape_point: invalid arguments")
    return n


def map_step(m, z, c, precision=FP32):
    """One update F(z) + c (no escape test), as a Python complex."""
    s = _map_struct(m)
    z, c = complex(z), complex(c)
    out = np.zeros(2, np.float64)
    if _load().jlo_map_step(ctypes.byref(s), z.real, z.imag, c.real, c.imag, precision, out.ctypes.data) != 0:
        raise ValueError("jlo_map_step: invalid arguments")
    return complex(out[0], out[1])
