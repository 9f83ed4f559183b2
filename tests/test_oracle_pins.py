"""Pins for the CPU oracle: facts the mathematics fixes, checked without the
oracle checking itself.  (Escape time for Z <- Z^2 + C, paper Sec. 2;
Mandelbrot mode, Sec. 3.)

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed operand, >= for >, an off-by-one count, a wrong
pixel centre) fails at least one of them.
"""
import math
from fractions import Fraction

import mpmath
import numpy as np
import pytest

import oracle
from paper_1611_03079_b300 import workloads as wl


def grid(rect, W, H, prec):
    """Pixel-centre coordinates in the working precision (test-side restatement
    of Sec. 2 region covering, used only to pick pixels and to form C)."""
    xmin, xmax, ymin, ymax = rect
    dx = (xmax - xmin) / W
    dy = (ymax - ymin) / H
    xs = xmin + (np.arange(W, dtype=np.float64) + 0.5) * dx
    ys = ymin + (np.arange(H, dtype=np.float64) + 0.5) * dy
    if prec == oracle.FP32:
        xs, ys = xs.astype(np.float32), ys.astype(np.float32)
    return xs, ys


# ---------------------------------------------------------------- c = 0 ----
@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64])
def test_c0_closed_form(prec):
    """C = 0: Z_n = Z_0^(2^n), so |Z_n|^2 = s^(2^n) with s = |Z_0|^2.  The count
    is max_iter for s <= 1, 0 for s > 4, else the first n with
    2^n log s > log 4.  Pixels whose decision is within the rounding drift of
    the boundary are excluded and must be rare."""
    W = H = 512
    rect = (-2.0, 2.0, -2.0, 2.0)
    mi = 100
    k = oracle.render(0j, rect, W, H, mi, oracle.JULIA, prec).astype(np.int64)
    xs, ys = grid(rect, W, H, prec)
    mpmath.mp.dps = 40
    u = 2.0 ** -24 if prec == oracle.FP32 else 2.0 ** -53
    bad = 0
    excluded = 0
    log4 = mpmath.log(4)
    for j in range(H):
        for i in range(W):
            s = mpmath.mpf(float(xs[i])) ** 2 + mpmath.mpf(float(ys[j])) ** 2
            if s > 4:
                exp = 0
            elif s <= 1:
                exp = mi
            else:
                ls = mpmath.log(s)
                n = 0
                while n < mi and (2 ** n) * ls <= log4:
                    n += 1
                exp = n
                # rounding drift of log|Z_n|^2 grows like 2^n * few ulps
                margins = [abs((2 ** m) * ls - log4) / log4 for m in (n - 1, n) if m >= 0]
                if min(margins) < (2 ** n) * 8 * u:
                    excluded += 1
                    continue
            if s <= 1 and 1 - s < 64 * u:
                excluded += 1
                continue
            bad += int(k[j, i] != exp)
    assert bad == 0
    assert excluded < 50


# --------------------------------------------------------------- c = -2 ----
def test_cm2_chebyshev_closed_form():
    """C = -2: with Z_0 = w + 1/w (|w| > 1), Z_n = w^(2^n) + w^(-2^n) exactly
    (Chebyshev conjugacy), evaluated in 60-digit arithmetic.  Binary64 counts
    must agree wherever the exact |Z_n|^2 stays clear of 4 by more than the
    rounding drift (which grows by at most 4x per step)."""
    W = H = 64
    rect = (-2.0, 2.0, -2.0, 2.0)
    mi = 100
    k = oracle.render(-2 + 0j, rect, W, H, mi, oracle.JULIA, oracle.FP64).astype(np.int64)
    xs, ys = grid(rect, W, H, oracle.FP64)
    mpmath.mp.dps = 60
    checked = 0
    for j in range(H):
        for i in range(W):
            z0 = mpmath.mpc(float(xs[i]), float(ys[j]))
            w = (z0 + mpmath.sqrt(z0 * z0 - 4)) / 2
            if abs(w) < 1:
                w = 1 / w
            if abs(abs(w) - 1) < mpmath.mpf("1e-30"):
                continue
            exp = None
            ok = True
            for n in range(0, 14):
                zn = w ** (2 ** n) + w ** (-(2 ** n))
                s = abs(zn) ** 2
                drift = (4.0 ** n) * 1e-14
                if abs(s - 4) / 4 < drift:
                    ok = False
                    break
                if s > 4:
                    exp = n
                    break
            if not ok or exp is None:
                continue
            checked += 1
            assert k[j, i] == exp, (i, j, k[j, i], exp)
    assert checked > 3000


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64])
def test_cm2_real_segment_never_escapes(prec):
    """The segment [-2, 2] is the Julia set of C = -2: a one-row frame puts
    y = 0 exactly and every x in (-2, 2) keeps x in [-2, 2] forever."""
    W = 1001
    mi = 300
    k = oracle.render(-2 + 0j, (-2.0, 2.0, -0.25, 0.25), W, 1, mi, oracle.JULIA, prec)
    assert (k == mi).all()


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64])
def test_escape_test_is_strict(prec):
    """Z_0 = 2, C = -2 is a fixed point with |Z|^2 == 4 exactly: the test
    |Z|^2 > 4 never fails, so the count is the limit (a >= test gives 0)."""
    assert oracle.escape_point(2 + 0j, -2 + 0j, 50, prec) == 50
    # pixel-centre version: W = 1 over [1.5, 2.5] has its centre at x = 2
    k = oracle.render(-2 + 0j, (1.5, 2.5, -0.5, 0.5), 1, 1, 50, oracle.JULIA, prec)
    assert k[0, 0] == 50


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64])
def test_count_convention(prec):
    """|Z_0|^2 > 4 gives 0; Z_0 = 3, C = 0: one test fails at once -> 0;
    Z_0 = 1.5, C = 0: 2.25 passes, 5.0625 fails -> 1 update; Mandelbrot C = 3:
    Z_0 = 0 passes, Z_1 = 3 fails -> 1."""
    assert oracle.escape_point(3 + 0j, 0j, 100, prec) == 0
    assert oracle.escape_point(1.5 + 0j, 0j, 100, prec) == 1
    assert oracle.escape_point(0j, 3 + 0j, 100, prec) == 1
    assert oracle.escape_point(0j, 0j, 7, prec) == 7


# ------------------------------------------------------------ symmetries ----
@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64])
@pytest.mark.parametrize("c,rect,W,H", [
    (complex(-0.8, 0.156), (-2.0, 2.0, -2.0, 2.0), 512, 512),
    (complex(-0.7269, 0.1889), (-1.6, 1.6, -1.6, 1.6), 256, 192),
    (complex(0.285, 0.01), (-1.8, 1.8, -1.0125, 1.0125), 1920, 1080),
])
def test_rotation_symmetry(prec, c, rect, W, H):
    """Z and -Z have the same orbit from step 1 on (squares are sign-blind and
    rounding is symmetric), so Julia counts are 180-degree symmetric for every
    pixel pair whose working-precision coordinates are exact negatives."""
    k = oracle.render(c, rect, W, H, 200, oracle.JULIA, prec)
    xs, ys = grid(rect, W, H, prec)
    okx = xs[::-1] == -xs
    oky = ys[::-1] == -ys
    rot = k[::-1, ::-1]
    mask = oky[:, None] & okx[None, :]
    assert mask.sum() > 0.05 * W * H  # binary64 grids over non-dyadic spans qualify only in part
    assert (k[mask] == rot[mask]).all()


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64])
def test_conjugate_symmetry(prec):
    """J(conj C) is the mirror image of J(C): y -> -y flips the sign of every
    imaginary part exactly, so counts(conj C) equal the row-flipped counts(C)
    wherever row coordinates are exact negatives."""
    rect = (-2.0, 2.0, -2.0, 2.0)
    c = complex(-0.8, 0.156)
    a = oracle.render(c, rect, 256, 256, 100, oracle.JULIA, prec)
    b = oracle.render(c.conjugate(), rect, 256, 256, 100, oracle.JULIA, prec)
    assert (a == b[::-1, :]).all()
    m = oracle.render(None, (-2.5, 1.0, -1.75, 1.75), 300, 256, 100, oracle.MANDELBROT, prec)
    assert (m == m[::-1, :]).all()


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64])
def test_mandelbrot_julia_identity(prec):
    """Mandelbrot mode (Sec. 3): Z_0 = 0 passes the test and Z_1 = C exactly,
    so M(C) = min(limit, 1 + J_C(Z_0 = C, limit - 1))."""
    rect = (-2.2, 0.8, -1.3, 1.3)
    W, H, mi = 61, 47, 150
    m = oracle.render(None, rect, W, H, mi, oracle.MANDELBROT, prec)
    xs, ys = grid(rect, W, H, prec)
    for j in range(0, H, 3):
        for i in range(0, W, 2):
            c = complex(float(xs[i]), float(ys[j]))
            jc = oracle.escape_point(c, c, mi - 1, prec)
            assert m[j, i] == min(mi, 1 + jc)


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64])
def test_mandelbrot_interiors_and_exterior(prec):
    """Points well inside the main cardioid or the period-2 disk never escape;
    points with |C| > 2 escape after exactly one update."""
    rect = (-2.5, 1.0, -1.75, 1.75)
    W, H, mi = 350, 350, 300
    m = oracle.render(None, rect, W, H, mi, oracle.MANDELBROT, prec)
    xs, ys = grid(rect, W, H, prec)
    X, Y = np.meshgrid(xs.astype(np.float64), ys.astype(np.float64))
    q = (X - 0.25) ** 2 + Y ** 2
    cardioid = q * (q + (X - 0.25)) < 0.25 * Y ** 2 - 0.02
    disk = (X + 1) ** 2 + Y ** 2 < 1 / 16 - 0.01
    outside = X ** 2 + Y ** 2 > 4.05
    assert cardioid.sum() > 1000 and disk.sum() > 100 and outside.sum() > 1000
    assert (m[cardioid] == mi).all()
    assert (m[disk] == mi).all()
    assert (m[outside] == 1).all()


# ----------------------------------------------- exact rational arithmetic ----
def _round_to(v, prec):
    return float(np.float32(v)) if prec == oracle.FP32 else float(v)


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP64])
def test_exact_rational_orbits(prec):
    """Brute force in exact rationals: for points that escape within 8 steps
    and whose |Z_n|^2 stays clear of 4 by a margin far larger than rounding,
    the working-precision count equals the exact count.  A transposed operand
    (cr for ci), a sign slip or a dropped term changes these counts."""
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(600):
        z0 = complex(*rng.uniform(-1.6, 1.6, size=2))
        c = complex(*rng.uniform(-1.2, 1.2, size=2))
        zr = Fraction(_round_to(z0.real, prec))
        zi = Fraction(_round_to(z0.imag, prec))
        cr = Fraction(_round_to(c.real, prec))
        ci = Fraction(_round_to(c.imag, prec))
        exp = None
        clear = True
        for n in range(9):
            s = zr * zr + zi * zi
            if abs(float(s) - 4.0) < 1e-3:
                clear = False
                break
            if s > 4:
                exp = n
                break
            zr, zi = zr * zr - zi * zi + cr, 2 * zr * zi + ci
        if exp is None or not clear:
            continue
        checked += 1
        got = oracle.escape_point(complex(_round_to(z0.real, prec), _round_to(z0.imag, prec)),
                                  complex(_round_to(c.real, prec), _round_to(c.imag, prec)), 100, prec)
        assert got == exp, (z0, c, got, exp)
    assert checked > 200


def test_pixel_centres_and_orientation():
    """Region covering: pixel (i, j) is the centre xmin + (i + 1/2) dx, row 0 at
    ymin.  With C = 0 and a view where only one corner lies inside the unit
    disk the max_iter pixel must land at that corner."""
    rect = (0.5, 2.5, 0.5, 2.5)
    k = oracle.render(0j, rect, 2, 2, 10, oracle.JULIA, oracle.FP64)
    # centres: x in {1.0, 2.0}, y in {1.0, 2.0}; |z|^2: (1,1)=2, (2,1)=5, (1,2)=5, (2,2)=8
    # (1,1): 2 -> 4 (passes, 4 is not > 4) -> |z|^2 = 16 fails: count 2
    assert k[0, 0] == 2
    assert k[0, 1] == 0 and k[1, 0] == 0 and k[1, 1] == 0
    k = oracle.render(0j, (-0.5, 3.5, -0.5, 0.5), 4, 1, 10, oracle.JULIA, oracle.FP64)
    # centres 0, 1, 2, 3 on the real axis: 0 -> inside, 1 -> inside, 2 -> 4 -> 16: count 1, 3 -> 0
    assert list(k[0]) == [10, 10, 1, 0]


# ------------------------------------------------------ colour, histogram ----
def test_colour_levels():
    """Colour levels (Sec. 2): entry 255 exactly for never-escaped points,
    otherwise floor(count * 255 / limit) (checked with exact Fractions)."""
    pal = wl.random_palette(5)
    for mi in (1, 2, 7, 100, 255, 1000, 65535):
        counts = np.unique(np.concatenate([np.arange(min(mi, 600) + 1), [mi, max(mi - 1, 0)]]))
        counts = counts[counts <= mi].astype(np.uint16)
        rgba = oracle.colour(counts, mi, pal)
        for n, px in zip(counts, rgba):
            idx = 255 if n == mi else math.floor(Fraction(int(n) * 255, mi))
            assert idx <= 255 and (idx < 255 or n == mi)
            assert (px == pal[idx]).all()


def test_histogram():
    """Histogram bins recover numpy.bincount exactly and sum to one."""
    rng = np.random.default_rng(2)
    for mi, n in ((100, 128 * 128), (1000, 4096), (1, 7)):
        counts = rng.integers(0, mi + 1, size=n).astype(np.uint16)
        h = oracle.hist(counts, mi)
        assert h.shape == (mi + 1,)
        ref = np.bincount(counts, minlength=mi + 1)
        assert (np.rint(h.astype(np.float64) * n).astype(np.int64) == ref).all()
        assert abs(float(h.astype(np.float64).sum()) - 1.0) < 1e-5


def test_precision_rule():
    """Deep-zoom precision rule: binary64 iff min(dx, dy) < 1000 ulp32(max|coord|)."""
    # 512 px over [-2, 2]: dx = 2^-7, ulp32(2) = 2^-22 -> 1000 ulp = 2.4e-4 < 2^-7 -> binary32
    assert oracle.precision_for_view((-2, 2, -2, 2), 512, 512) == oracle.FP32
    # width 1e-6 around 0.3 over 1920 px: dx = 5.2e-10 < 1000 * 2^-25 -> binary64
    assert oracle.precision_for_view((0.3 - 5e-7, 0.3 + 5e-7, -2.8e-7, 2.8e-7), 1920, 1080) == oracle.FP64
    # boundary: m = 1 (ulp32(1) = 2^-23), dx exactly 1000 * 2^-23 is not below -> binary32
    d = 1000 * 2.0 ** -23
    assert oracle.precision_for_view((-1.0, -1.0 + 16 * d, 0.0, 16 * d), 16, 16) == oracle.FP32
    assert oracle.precision_for_view((-1.0, -1.0 + 16 * d * 0.999, 0.0, 16 * d), 16, 16) == oracle.FP64
    frames = wl.deep_zoom()
    n64 = sum(oracle.precision_for_view(f["rect"], f["W"], f["H"]) for f in frames)
    assert 50 <= n64 <= 60


def test_numpy_float32_cross_check():
    """An independent vectorised numpy float32 iteration (IEEE, no fused ops)
    agrees with the C oracle on the single-frame workload."""
    f = wl.single_frame()
    k = oracle.render(f["c"], f["rect"], f["W"], f["H"], f["max_iter"], f["mode"], f["precision"])
    xs, ys = grid(f["rect"], f["W"], f["H"], oracle.FP32)
    X, Y = np.meshgrid(xs, ys)
    X = X.astype(np.float32)
    Y = Y.astype(np.float32)
    cr, ci = np.float32(f["c"].real), np.float32(f["c"].imag)
    cnt = np.full(X.shape, f["max_iter"], dtype=np.int64)
    alive = np.ones(X.shape, dtype=bool)
    four = np.float32(4.0)
    with np.errstate(over="ignore", invalid="ignore"):
        for n in range(f["max_iter"]):
            x2 = X * X
            y2 = Y * Y
            esc = alive & ((x2 + y2) > four)
            cnt[esc] = n
            alive &= ~esc
            t = (X + X) * Y
            Y = t + ci
            X = (x2 - y2) + cr
    assert (cnt == k).all()
    # survey statistics of this frame: mean count ~9.09, 56,252 zeros, 12,986 at the limit
    assert abs(k.mean() - 9.09) < 0.01
    assert int((k == 0).sum()) == 56252 and int((k == 100).sum()) == 12986
