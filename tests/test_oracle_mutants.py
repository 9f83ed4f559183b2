"""The oracle pins have teeth: each plausible slip, planted in a temporary copy
of the C oracle (on the CPU), makes at least one pin fail."""
import ctypes
import os
import subprocess

import pytest

import oracle
from oracle import build as obuild
from tests import test_oracle_pins as pins

MUTANTS = {
    "strict_test_ge": ("if (r > 4.0f)", "if (r >= 4.0f)"),
    "swap_c_parts": ("y = t + ci;\n        float u", "y = t + cr;\n        float u"),
    "drop_cr": ("x = u + cr;\n    }\n    return max_iter;\n}\n\n/* Same", "x = u;\n    }\n    return max_iter;\n}\n\n/* Same"),
    "minus_sign": ("float u = x2 - y2;", "float u = x2 + y2;"),
    "count_off_by_one": ("            return n;\n        float t", "            return n + 1;\n        float t"),
    "pixel_corner": ("double yd = jb->ymin + ((double)j + 0.5) * dy;", "double yd = jb->ymin + ((double)j) * dy;"),
    "no_doubling": ("float t = x + x;", "float t = x;"),
}

CHECKS = [
    lambda: pins.test_escape_test_is_strict(oracle.FP32),
    lambda: pins.test_count_convention(oracle.FP32),
    lambda: pins.test_exact_rational_orbits(oracle.FP32),
    lambda: pins.test_pixel_centres_and_orientation(),
    lambda: pins.test_numpy_float32_cross_check(),
    lambda: pins.test_mandelbrot_interiors_and_exterior(oracle.FP32),
    lambda: pins.test_conjugate_symmetry(oracle.FP32),
]


def _build_mutant(tmp_path, old, new):
    src = open(obuild.SRC).read()
    assert src.count(old) >= 1, old
    mutated = src.replace(old, new, 1)
    # the binary64 routine and the colour/histogram code stay as they are;
    # pixel-centre mutation applies to both precisions through render_rows.
    c = tmp_path / "m.c"
    c.write_text(mutated)
    so = tmp_path / "m.so"
    subprocess.check_call(["gcc", *obuild.CFLAGS, str(c), "-o", str(so), "-lm"])
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    so = _build_mutant(tmp_path, old, new)
    real = oracle._load()
    L = ctypes.CDLL(so)
    for fn in ("jlo_render", "jlo_escape_point", "jlo_colour", "jlo_hist"):
        f = getattr(L, fn)
        r = getattr(real, fn)
        f.argtypes, f.restype = r.argtypes, r.restype

    class Proxy:
        def __getattr__(self, k):
            return getattr(L, k)

    monkeypatch.setattr(oracle, "_lib", Proxy())
    caught = 0
    for chk in CHECKS:
        try:
            chk()
        except AssertionError:
            caught += 1
    assert caught >= 1, "mutant %s survived every pin" % name
