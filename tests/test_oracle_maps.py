"""Pins for the generic-map oracle (Z <- Z^d + C and Z <- P(Z)/Q(Z) + C; paper
Sec. 2 "other functions", Fig. 4): facts fixed by the mathematics or by an
already-pinned routine, not by re-running the oracle's own formulas.

  - reductions: Z^2 + C, z^2/1 + C and 2z^2/2 + C give the quadratic oracle's
    counts bit for bit (every rounding is then the same);
  - C = 0 closed form for Z^d: |Z_n|^2 = |Z_0|^(2 d^n);
  - one step F(Z) + C against a 60-digit evaluation of the polynomial or
    quotient (mpmath) within the rounding error of the working precision;
  - Fig. 4's map as printed equals z^4 + 1 + C away from z = +-i;
  - exact orbits (integers and units) for the escape test and the bailout;
  - parameter-plane mode starts from the map's z0; conjugation symmetry.
"""
import cmath

import mpmath
import numpy as np
import pytest

import oracle
from paper_1611_03079_b300 import workloads as wl

mpmath.mp.dps = 60
PRECS = [oracle.FP32, oracle.FP64]


def _rnd(v, prec):
    """Round a complex number to the working precision, part by part."""
    t = np.float32 if prec == oracle.FP32 else np.float64
    return complex(float(t(v.real)), float(t(v.imag)))


# ---------------------------------------------------------- reductions ----
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", [oracle.JULIA, oracle.MANDELBROT])
def test_power2_equals_quadratic(prec, mode):
    for c, rect, mi in ((complex(-0.8, 0.156), (-2, 2, -2, 2), 100),
                        (complex(0.285, 0.01), (-1.6, 1.6, -1.6, 1.6), 300),
                        (complex(-0.7269, 0.1889), (-0.3, 0.1, 0.2, 0.45), 500)):
        if mode == oracle.MANDELBROT:
            rect = (-2.5, 1.0, -1.75, 1.75) if mi == 100 else (-0.8, -0.7, 0.05, 0.15)
        a = oracle.render_map(wl.power_map(2), c, rect, 97, 61, mi, mode, prec)
        b = oracle.render(c, rect, 97, 61, mi, mode, prec)
        assert (a == b).all()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mode", [oracle.JULIA, oracle.MANDELBROT])
def test_rational_forms_of_the_quadratic(prec, mode):
    """z^2 / 1 and (2 z^2) / 2: Horner and the quotient add only exact steps
    (products by 1 and 2, sums with 0), so the counts are the quadratic's."""
    c = complex(-0.4, 0.6)
    rect = (-1.5, 1.5, -1.2, 1.2) if mode == oracle.JULIA else (-2.2, 0.8, -1.3, 1.3)
    ref = oracle.render(c, rect, 80, 64, 200, mode, prec)
    for m in (wl.rational_map([0, 0, 1], [1]), wl.rational_map([0, 0, 2], [2])):
        assert (oracle.render_map(m, c, rect, 80, 64, 200, mode, prec) == ref).all()


# ------------------------------------------------------ c = 0 closed form --
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d", [2, 3, 4, 5, 7, 8, 11, 16])
def test_power_c0_closed_form(prec, d):
    """C = 0: |Z_n|^2 = s^(d^n) with s = |Z_0|^2, so the count is 0 for
    s > 4, the limit for s < 1, else the first n with d^n log s > log 4.
    Points within 1e-3 (relative) of a decision are skipped; the rounding
    drift is far below that for s >= 1.01."""
    rng = np.random.default_rng(d)
    mi = 60
    checked = 0
    for _ in range(1500):
        r = rng.uniform(0.05, 2.3)
        if 0.985 < r * r < 1.01:
            continue
        z0 = _rnd(cmath.rect(r, rng.uniform(-np.pi, np.pi)), prec)
        s = abs(z0) ** 2
        if abs(s - 4.0) < 4e-3:
            continue
        if s > 4.0:
            expect = 0
        elif s < 1.0:
            expect = mi
        else:
            ls, l4 = np.log(s), np.log(4.0)
            n, near = 0, False
            while True:
                v = d ** n * ls
                if abs(v - l4) < 1e-3 * l4:
                    near = True
                if v > l4:
                    break
                n += 1
            if near:
                continue
            expect = min(n, mi)
        assert oracle.map_escape_point(wl.power_map(d), z0, 0j, mi, prec) == expect, (d, z0)
        checked += 1
    assert checked > 1000


# ----------------------------------------------------------- one step -----
def _mp_poly(coeffs, z):
    acc = mpmath.mpc(0)
    for k, a in enumerate(coeffs):
        acc += mpmath.mpc(a.real, a.imag) * z ** k
    return acc


@pytest.mark.parametrize("prec", PRECS)
def test_power_step_against_high_precision(prec):
    rng = np.random.default_rng(11)
    rel = 1e-13 if prec == oracle.FP64 else 5e-6
    for _ in range(400):
        d = int(rng.integers(2, 17))
        z = _rnd(complex(*rng.uniform(-1.3, 1.3, 2)), prec)
        c = _rnd(complex(*rng.uniform(-1, 1, 2)), prec)
        got = oracle.map_step(wl.power_map(d), z, c, prec)
        zz = mpmath.mpc(z.real, z.imag)
        exact = zz ** d + mpmath.mpc(c.real, c.imag)
        scale = abs(z) ** d + abs(c) + 1e-30
        assert abs(complex(exact) - got) <= rel * d * scale, (d, z, c, got, complex(exact))


@pytest.mark.parametrize("prec", PRECS)
def test_rational_step_against_high_precision(prec):
    rng = np.random.default_rng(12)
    eps = 2.0 ** -52 if prec == oracle.FP64 else 2.0 ** -23
    checked = 0
    for t in range(600):
        nd, nq = int(rng.integers(0, 9)), int(rng.integers(0, 9))
        m = wl.rational_map([_rnd(complex(*rng.standard_normal(2)), prec) for _ in range(nd + 1)],
                            [_rnd(complex(*rng.standard_normal(2)), prec) for _ in range(nq + 1)])
        z = _rnd(complex(*rng.uniform(-1.2, 1.2, 2)), prec)
        c = _rnd(complex(*rng.uniform(-1, 1, 2)), prec)
        zz = mpmath.mpc(z.real, z.imag)
        P, Q = _mp_poly(m["num"], zz), _mp_poly(m["den"], zz)
        if abs(Q) < 0.25:
            continue
        exact = P / Q + mpmath.mpc(c.real, c.imag)
        # forward error of Horner (about 2 n eps sum |a_k| |z|^k per polynomial)
        # and of the quotient, relative to |Q|
        absP = sum(abs(a) * abs(z) ** k for k, a in enumerate(m["num"]))
        absQ = sum(abs(a) * abs(z) ** k for k, a in enumerate(m["den"]))
        bound = 8 * (nd + nq + 4) * eps * (absP / abs(Q) + abs(P) * absQ / abs(Q) ** 2 + abs(c) + 1.0)
        got = oracle.map_step(m, z, c, prec)
        assert abs(complex(exact) - got) <= bound, (nd, nq, z, got, complex(exact), bound)
        checked += 1
    assert checked > 300


@pytest.mark.parametrize("prec", PRECS)
def test_fig4_as_printed_is_z4_plus_1(prec):
    """Fig. 4: z^4 + (z^2 + 1)/(z^2 + 1) + C equals z^4 + 1 + C where z^2 != -1."""
    rng = np.random.default_rng(13)
    m = wl.fig4_map()
    c = _rnd(wl.FIG4_C, prec)
    tol = 1e-12 if prec == oracle.FP64 else 2e-5
    for _ in range(300):
        z = _rnd(complex(*rng.uniform(-1.4, 1.4, 2)), prec)
        if abs(z * z + 1) < 0.2:
            continue
        expect = z ** 4 + 1 + c
        assert abs(oracle.map_step(m, z, c, prec) - expect) <= tol * (abs(z) ** 6 + 3), z


# --------------------------------------------------------- exact orbits ----
@pytest.mark.parametrize("prec", PRECS)
def test_exact_orbits_and_bailout(prec):
    P = lambda d: wl.power_map(d)  # noqa: E731
    # |Z_0|^2 = 4 passes the test (not > 4); Z_1 = 8 escapes
    assert oracle.map_escape_point(P(3), 2, 0, 50, prec) == 1
    # 0 -> -2 -> 2 -> 2 ...: |Z|^2 = 4 forever
    assert oracle.map_escape_point(P(2), 0, -2, 50, prec) == 50
    # unit fixed points and cycles
    assert oracle.map_escape_point(P(3), -1, 0, 50, prec) == 50
    assert oracle.map_escape_point(P(3), 1j, 0, 50, prec) == 50
    assert oracle.map_escape_point(P(4), 1j, 0, 50, prec) == 50
    # 2 + 0i with C = 0 under z^5: 2 -> 32
    assert oracle.map_escape_point(P(5), 2, 0, 50, prec) == 1
    # z^3 / z at z = 2: 8 / 2 = 4 exactly; bailout 4 vs 16 vs 256
    m = wl.rational_map([0, 0, 0, 1], [0, 1])
    assert oracle.map_step(m, 2, 0, prec) == 4
    assert oracle.map_escape_point(m, 2, 0, 50, prec) == 1
    assert oracle.map_escape_point(dict(m, bailout=16.0), 2, 0, 50, prec) == 2
    assert oracle.map_escape_point(dict(m, bailout=256.0), 2, 0, 50, prec) == 3
    # Q = 0: the first update is 0/0 (NaN), which fails the next test
    z = wl.rational_map([1, 1], [0])
    assert oracle.map_escape_point(z, 0.5, 0.25, 50, prec) == 1
    assert oracle.map_escape_point(z, 3, 0, 50, prec) == 0


@pytest.mark.parametrize("prec", PRECS)
def test_parameter_plane_starts_from_z0(prec):
    m = wl.rational_map([0.3, 0, 0, 1], [1, 0.2j], z0=0.5 + 0.25j)
    rect, W, H = (-1.2, 0.9, -1.0, 1.1), 23, 17
    got = oracle.render_map(m, 0j, rect, W, H, 80, oracle.MANDELBROT, prec)
    dx, dy = (rect[1] - rect[0]) / W, (rect[3] - rect[2]) / H
    for j in range(H):
        for i in range(W):
            cpix = complex(rect[0] + (i + 0.5) * dx, rect[2] + (j + 0.5) * dy)
            assert got[j, i] == oracle.map_escape_point(m, m["z0"], cpix, 80, prec)
    # a different z0 changes the picture
    other = oracle.render_map(dict(m, z0=0j), 0j, rect, W, H, 80, oracle.MANDELBROT, prec)
    assert (other != got).any()


@pytest.mark.parametrize("prec", PRECS)
def test_julia_render_matches_points(prec):
    m = wl.random_rational_map(5)
    c, rect, W, H = complex(0.1, -0.3), (-2.0, 1.5, -1.4, 1.9), 19, 13
    got = oracle.render_map(m, c, rect, W, H, 120, oracle.JULIA, prec)
    dx, dy = (rect[1] - rect[0]) / W, (rect[3] - rect[2]) / H
    for j in range(H):
        for i in range(W):
            z = complex(rect[0] + (i + 0.5) * dx, rect[2] + (j + 0.5) * dy)
            assert got[j, i] == oracle.map_escape_point(m, z, c, 120, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_conjugate_symmetry(prec):
    """Real coefficients and real C: the orbit of conj(Z_0) is the conjugate
    orbit, operation by operation, so counts agree exactly."""
    rng = np.random.default_rng(14)
    maps = [wl.power_map(3), wl.power_map(6), wl.rational_map([0.2, -0.5, 0, 1], [1, 0, 0.3]),
            wl.fig4_map()]
    for m in maps:
        for _ in range(200):
            x, y = rng.uniform(-1.6, 1.6, 2)
            cr = float(rng.uniform(-1, 0.5))
            a = oracle.map_escape_point(m, complex(x, y), cr, 200, prec)
            b = oracle.map_escape_point(m, complex(x, -y), cr, 200, prec)
            assert a == b


def test_invalid_maps_rejected():
    with pytest.raises(ValueError):
        oracle.render_map(wl.power_map(1), 0j, (-1, 1, -1, 1), 4, 4, 10)
    with pytest.raises(ValueError):
        oracle.render_map(wl.power_map(17), 0j, (-1, 1, -1, 1), 4, 4, 10)
    with pytest.raises(ValueError):
        oracle.render_map(dict(wl.power_map(2), bailout=0.0), 0j, (-1, 1, -1, 1), 4, 4, 10)
    with pytest.raises(ValueError):
        oracle.render_map(wl.rational_map([1] * 10, [1]), 0j, (-1, 1, -1, 1), 4, 4, 10)
