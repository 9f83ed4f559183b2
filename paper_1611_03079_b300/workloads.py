"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

Both the CUDA path and the CPU oracle take their inputs from here, so every
parity test and the benchmark see identical frames, palettes and parameter
samples.  Nothing in this module computes escape counts, colours, histograms
or network outputs.

Workloads (the paper's images are synthetic renders; there is no dataset):
  single_frame()      Julia C = -0.8+0.156i, 512x512 over [-2,2]^2, binary32,
                      limit 100 (Sec. 2 uses limit 100), uint8 counts.
  throughput_sweep()  4096x4096 Julia frames over [-1.6,1.6]^2 for three C,
                      limits 100 and 1000, binary32 and binary64, uint16 counts
                      + RGBA8; plus Mandelbrot 4096x4096 over
                      [-2.5,1]x[-1.75,1.75] (Sec. 3 parameter plane) at the
                      same limits and precisions.
  path_animation()    720 frames with C(t) = 0.7885 exp(i t), t_k = 2 pi k/720,
                      sizes drawn by seed from {640x480, 1920x1080, 3840x2160},
                      square pixels with vertical half-span 1.0125, limit 100
                      (Sec. 3: paths of C animated in real time).
  deep_zoom()         64 frames 1920x1080 centred on seeded points of the
                      Julia set of C = -0.7269+0.1889i, widths 4 -> 1e-12
                      geometric, limit 2000 (Sec. 3 deep zoom).
  survey_*()          C samples for the learned surrogate: uniform over
                      [-2,0.5]x[-1.25,1.25] (the Mandelbrot set's bounding box,
                      Sec. 3 "roadmap"), seeds 0 (train), 1 (candidates),
                      2 (held out).
  cardioid_path()     C(t) = ((2 cos t - cos 2t)/a, (2 sin t - sin 2t)/a), the
                      prescribed path of Sec. 3 (a = 3.9 in the paper).
"""
import math

import numpy as np

FP32, FP64, AUTO = 0, 1, 2
JULIA, MANDELBROT = 0, 1


def random_palette(seed=7):
    """256 x 4 uint8 palette of random RGB bytes with alpha 255 (entry 255 is
    random as well, so tests can tell it apart from every other entry)."""
    rng = np.random.default_rng(seed)
    p = rng.integers(0, 256, size=(256, 4), dtype=np.uint8)
    p[:, 3] = 255
    # keep entry 255 distinct from all others
    while any((p[k, :3] == p[255, :3]).all() for k in range(255)):
        p[255, :3] = rng.integers(0, 256, size=3, dtype=np.uint8)
    return p


def single_frame():
    return dict(c=complex(-0.8, 0.156), rect=(-2.0, 2.0, -2.0, 2.0), W=512, H=512, max_iter=100,
                mode=JULIA, precision=FP32, count_type="u8")


SWEEP_C = (complex(0.285, 0.01), complex(-0.7269, 0.1889), complex(-0.4, 0.6))


def throughput_sweep(size=4096):
    """The 16 renders of the throughput sweep (12 Julia + 4 Mandelbrot)."""
    out = []
    for prec in (FP32, FP64):
        for mi in (100, 1000):
            for c in SWEEP_C:
                out.append(dict(c=c, rect=(-1.6, 1.6, -1.6, 1.6), W=size, H=size, max_iter=mi, mode=JULIA,
                                precision=prec, count_type="u16"))
            out.append(dict(c=None, rect=(-2.5, 1.0, -1.75, 1.75), W=size, H=size, max_iter=mi,
                            mode=MANDELBROT, precision=prec, count_type="u16"))
    return out


PATH_SIZES = ((640, 480), (1920, 1080), (3840, 2160))


def path_animation(n=720, seed=0, radius=0.7885, half_height=1.0125, max_iter=100):
    """Frames of the circular C path (one dict per frame)."""
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, 3, size=n)
    frames = []
    for k in range(n):
        t = 2.0 * math.pi * k / n
        W, H = PATH_SIZES[int(pick[k])]
        hw = half_height * W / H
        frames.append(dict(c=complex(radius * math.cos(t), radius * math.sin(t)),
                           rect=(-hw, hw, -half_height, half_height), W=W, H=H, max_iter=max_iter,
                           mode=JULIA, precision=FP32, count_type=None))
    return frames


def julia_boundary_points(c, n, seed=0, burn_in=1000):
    """Seeded points near the Julia set of c by inverse iteration
    z <- +-sqrt(z - c) with a random sign per step (binary64)."""
    rng = np.random.default_rng(seed)
    z = complex(0.5, 0.5)
    signs = rng.integers(0, 2, size=burn_in + n * 7)
    pts = []
    k = 0
    for s in signs:
        z = np.sqrt(z - c)
        if s:
            z = -z
        k += 1
        if k > burn_in and (k - burn_in) % 7 == 0 and len(pts) < n:
            pts.append(complex(z))
    return pts


def deep_zoom(n=64, seed=0, W=1920, H=1080, c=complex(-0.7269, 0.1889), w0=4.0, w1=1e-12, max_iter=2000):
    """Deep-zoom frames: width w_k = w0 (w1/w0)^(k/(n-1)), height w_k H/W."""
    centres = julia_boundary_points(c, n, seed=seed)
    frames = []
    for k in range(n):
        w = w0 * (w1 / w0) ** (k / (n - 1))
        h = w * H / W
        z = centres[k]
        frames.append(dict(c=c, rect=(z.real - w / 2, z.real + w / 2, z.imag - h / 2, z.imag + h / 2), W=W,
                           H=H, max_iter=max_iter, mode=JULIA, precision=AUTO, count_type="u16"))
    return frames


def survey_c(n, seed):
    """n values of C uniform over [-2, 0.5] x [-1.25, 1.25], float32 (n, 2)."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-2.0, 0.5, size=n)
    im = rng.uniform(-1.25, 1.25, size=n)
    return np.stack([re, im], axis=1).astype(np.float32)


def survey_train(n=65536):
    return survey_c(n, 0)


def survey_candidates(n=1048576):
    return survey_c(n, 1)


def survey_heldout(n=4096):
    return survey_c(n, 2)


SURVEY_FRAME = dict(rect=(-2.0, 2.0, -2.0, 2.0), W=128, H=128, max_iter=100)


def fourier_matrix(seed=3, n_freq=32, sigma=2.0):
    """Gaussian Fourier-feature matrix B (n_freq x 2), entries N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n_freq, 2)) * sigma).astype(np.float32)


def mlp_init(seed=4, n_in=64, hidden=256, n_out=101):
    """He-normal initial weights (out x in, float32) and zero biases."""
    rng = np.random.default_rng(seed)
    dims = [(hidden, n_in), (hidden, hidden), (n_out, hidden)]
    p = {}
    for li, (o, i) in enumerate(dims, start=1):
        p["W%d" % li] = (rng.standard_normal((o, i)) * math.sqrt(2.0 / i)).astype(np.float32)
        p["b%d" % li] = np.zeros((o,), dtype=np.float32)
    return p


def cardioid_path(n, a=3.9, t0=0.0, t1=2.0 * math.pi, clockwise=True):
    """n values of C on the cardioid path of Sec. 3 (binary64 complex)."""
    ts = np.linspace(t0, t1, n, endpoint=False)
    if clockwise:
        ts = -ts
    return (2 * np.cos(ts) - np.cos(2 * ts)) / a + 1j * (2 * np.sin(ts) - np.sin(2 * ts)) / a


def random_views(n, seed, max_side=97):
    """Small random frames (ragged sizes, random C and views) for parity tests."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        W = int(rng.integers(1, max_side + 1))
        H = int(rng.integers(1, max_side + 1))
        cx, cy = rng.uniform(-1.0, 1.0, size=2)
        w = float(10 ** rng.uniform(-3, 0.7))
        h = w * H / W
        c = complex(*rng.uniform(-1.0, 1.0, size=2))
        mode = int(rng.integers(0, 2))
        out.append(dict(c=c, rect=(cx - w / 2, cx + w / 2, cy - h / 2, cy + h / 2), W=W, H=H,
                        max_iter=int(rng.choice([1, 2, 7, 50, 100, 255, 300])), mode=mode,
                        precision=int(rng.integers(0, 2))))
    return out


def boundary_views(n, seed, max_side=48):
    """Small binary64 frames centred on points of Julia and Mandelbrot set
    boundaries (where an escape test is closest to its threshold for the most
    steps), widths 10^-13 .. 4, limits up to 3000, both modes, for parity tests
    of binary64 paths.  Julia centres by inverse iteration (julia_boundary_points)
    for a random C; Mandelbrot centres on the main cardioid's boundary
    e^{it}/2 - e^{2it}/4 or the period-2 disk's -1 + e^{it}/4."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        W = int(rng.integers(1, max_side + 1))
        H = int(rng.integers(1, max_side + 1))
        w = float(10 ** rng.uniform(-13, 0.6))
        h = w * H / W
        mode = int(rng.integers(0, 2))
        if mode == JULIA:
            c = complex(*rng.uniform(-1.2, 1.2, size=2))
            z = julia_boundary_points(c, 1, seed=int(rng.integers(0, 1 << 30)), burn_in=200)[0]
        else:
            c = None
            t = float(rng.uniform(0.0, 2.0 * math.pi))
            e1 = complex(math.cos(t), math.sin(t))
            z = e1 / 2 - e1 * e1 / 4 if rng.integers(0, 2) else -1 + e1 / 4
        out.append(dict(c=c, rect=(z.real - w / 2, z.real + w / 2, z.imag - h / 2, z.imag + h / 2), W=W, H=H,
                        max_iter=int(rng.choice([1, 3, 4, 5, 100, 1000, 3000])), mode=mode, precision=FP64))
    return out


# ---- generic maps (Sec. 2: other functions than Z^2 + C; Fig. 4) ----------
# Map descriptions are plain data: {"kind": "power", "degree": d} or
# {"kind": "rational", "num": [a_0 .. a_n], "den": [b_0 .. b_m]} with complex
# coefficients, constant term first, plus "bailout" (|Z|^2 escape threshold)
# and "z0" (Z_0 of the parameter-plane mode).

FIG4_C = complex(0.862085, 0.64695)


def power_map(d, bailout=4.0):
    """Z <- Z^d + C (Multibrot / Multi-Julia family)."""
    return {"kind": "power", "degree": int(d), "bailout": float(bailout), "z0": 0j}


def rational_map(num, den, bailout=4.0, z0=0j):
    return {"kind": "rational", "num": [complex(v) for v in num], "den": [complex(v) for v in den],
            "bailout": float(bailout), "z0": complex(z0)}


def fig4_map():
    """Fig. 4's map as printed, z^4 + (z^2 + 1)/(z^2 + 1) + C, as one quotient
    P/Q + C: P = z^4 (z^2 + 1) + (z^2 + 1) = 1 + z^2 + z^4 + z^6, Q = 1 + z^2.
    (As printed the fraction cancels, so away from z = +-i this is z^4 + 1 + C.)"""
    return rational_map([1, 0, 1, 0, 1, 0, 1], [1, 0, 1])


def random_rational_map(seed, num_degree=3, den_degree=2, scale=0.6, bailout=16.0):
    """Seeded rational map with complex Gaussian coefficients (scale^k damping
    on the k-th coefficient keeps the orbit scale moderate)."""
    rng = np.random.default_rng(seed)

    def coeffs(n):
        z = rng.standard_normal(n + 1) + 1j * rng.standard_normal(n + 1)
        return [complex(v * scale ** k) for k, v in enumerate(z)]
    num = coeffs(num_degree)
    num[-1] = 1.0 + 0j
    return rational_map(num, coeffs(den_degree), bailout=bailout)


def map_sweep(size=4096):
    """Generic-map benchmark frames: Multibrot parameter planes for d = 3, 4,
    5, 8 over [-1.6, 1.6]^2 and Fig. 4's map (as printed) at C = .862085 +
    .64695i over [-1.6, 1.6]^2, limit 100, binary32; plus the d = 3 plane in
    binary64."""
    frames = []
    for d in (3, 4, 5, 8):
        frames.append(dict(map=power_map(d), c=0j, rect=(-1.6, 1.6, -1.6, 1.6), W=size, H=size, max_iter=100,
                           mode=MANDELBROT, precision=FP32))
    frames.append(dict(map=fig4_map(), c=FIG4_C, rect=(-1.6, 1.6, -1.6, 1.6), W=size, H=size, max_iter=100,
                       mode=JULIA, precision=FP32))
    frames.append(dict(map=power_map(3), c=0j, rect=(-1.6, 1.6, -1.6, 1.6), W=size, H=size, max_iter=100,
                       mode=MANDELBROT, precision=FP64))
    return frames
