"""Parameter paths for animations (paper Sec. 3) as batch-plan front ends.

The paper moves C along prescribed paths so the Julia set changes smoothly:
clockwise along the cardioid f(t) = ((2 cos t - cos 2t)/a, (2 sin t - sin 2t)/a)
with a = 3.9, just outside the main cardioid of the Mandelbrot set (a = 4 is
its boundary), and then along growing cardioids (decreasing a) so that a few
trips cover the relevant parameter values.  These helpers only produce the C
values and frame descriptions; the rendering is one batch plan.
"""
import math

import numpy as np


def cardioid_point(t, a=3.9):
    """f(t) of the paper's cardioid path (binary64 complex)."""
    return complex((2 * math.cos(t) - math.cos(2 * t)) / a, (2 * math.sin(t) - math.sin(2 * t)) / a)


def cardioid_path(n, a=3.9, t0=0.0, clockwise=True):
    """n values of C evenly spaced in t over one trip, starting at t0."""
    sgn = -1.0 if clockwise else 1.0
    return [cardioid_point(t0 + sgn * 2 * math.pi * k / n, a) for k in range(n)]


def expanding_sweep(n_per_trip, trips, a0=3.9, a1=3.0, clockwise=True):
    """Several trips around growing cardioids: a decreases linearly from a0 to
    a1 over the whole sweep, so consecutive values stay close."""
    total = n_per_trip * trips
    out = []
    sgn = -1.0 if clockwise else 1.0
    for k in range(total):
        a = a0 + (a1 - a0) * k / max(total - 1, 1)
        out.append(cardioid_point(sgn * 2 * math.pi * k / n_per_trip, a))
    return out


def julia_frames(cs, W=640, H=480, half_height=1.5, max_iter=100, precision=0, count_type=None, rgba=True):
    """One Julia frame per C: square pixels, centred view of half-height
    `half_height`."""
    hw = half_height * W / H
    return [dict(c=complex(c), rect=(-hw, hw, -half_height, half_height), W=W, H=H, max_iter=max_iter, mode=0,
                 precision=precision, count_type=count_type, rgba=rgba) for c in cs]


def with_minimap(frames, W=256, H=192, rect=(-2.5, 1.0, -1.3125, 1.3125), max_iter=100):
    """Interleave each Julia frame with the Mandelbrot-set minimap the paper
    shows next to it (Sec. 3; the cursor drawn at C is display work, not
    computed here).  The minimap does not depend on C, so it is the same
    frame each time; returns the new frame list."""
    out = []
    for f in frames:
        out.append(f)
        out.append(dict(c=None, rect=rect, W=W, H=H, max_iter=max_iter, mode=1, precision=0,
                        count_type=None, rgba=True))
    return out


def mandelbrot_zoom(centre, n, W=1920, H=1080, w0=3.0, w1=1e-12, max_iter=2000):
    """Deep zoom on the Mandelbrot set around `centre` (Sec. 3, Fig. 3):
    widths w0 -> w1 geometric, precision chosen per frame (JL_AUTO)."""
    frames = []
    for k in range(n):
        w = w0 * (w1 / w0) ** (k / max(n - 1, 1))
        h = w * H / W
        z = complex(centre)
        frames.append(dict(c=None, rect=(z.real - w / 2, z.real + w / 2, z.imag - h / 2, z.imag + h / 2), W=W, H=H,
                           max_iter=max_iter, mode=1, precision=2, count_type="u16", rgba=False))
    return frames


def fit_cardioid_parameter(c, a=3.9, iters=60):
    """The t minimising |f(t) - c| (golden-section refinement of a grid
    search) and that distance."""
    ts = np.linspace(0, 2 * math.pi, 4096, endpoint=False)
    d = np.abs((2 * np.cos(ts) - np.cos(2 * ts)) / a + 1j * (2 * np.sin(ts) - np.sin(2 * ts)) / a - c)
    k = int(np.argmin(d))
    lo, hi = ts[k] - 2 * math.pi / 4096, ts[k] + 2 * math.pi / 4096
    g = (math.sqrt(5) - 1) / 2
    for _ in range(iters):
        m1, m2 = hi - g * (hi - lo), lo + g * (hi - lo)
        if abs(cardioid_point(m1, a) - c) < abs(cardioid_point(m2, a) - c):
            hi = m2
        else:
            lo = m1
    t = 0.5 * (lo + hi)
    return t % (2 * math.pi), abs(cardioid_point(t, a) - c)
