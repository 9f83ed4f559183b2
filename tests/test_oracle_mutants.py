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


# ---- generic maps (jl_oracle_maps.c / map_iter.inc) -----------------------
from tests import test_oracle_maps as mpins  # noqa: E402

MAP_MUTANTS = {
    "mul_sign": ("map_iter.inc", "            wx = ac - bd;", "            wx = ac + bd;"),
    "mul_cross": ("map_iter.inc", "            wy = ad + bc;", "            wy = ad - bc;"),
    "square_no_doubling": ("map_iter.inc", "REAL tw = wx + wx;", "REAL tw = wx;"),
    "top_bit_high": ("map_iter.inc", "while ((d >> (top + 1)) != 0)", "while ((d >> top) != 0)"),
    "skip_multiply": ("map_iter.inc", "if ((d >> b) & 1) {", "if (!((d >> b) & 1)) {"),
    "horner_sign": ("map_iter.inc", "REAL mr = ac - bd;", "REAL mr = ac + bd;"),
    "horner_index": ("map_iter.inc", "pr = mr + a[2 * k];", "pr = mr + a[2 * k + 2];"),
    "quotient_sign": ("map_iter.inc", "REAL ni = s3 - s4;", "REAL ni = s3 + s4;"),
    "quotient_norm": ("map_iter.inc", "REAL q2 = q2r + q2i;", "REAL q2 = q2r - q2i;"),
    "bailout_strict": ("map_iter.inc", "if (!(r <= bail))", "if (!(r < bail))"),
    "drop_c": ("map_iter.inc", "x = fx + cr;", "x = fx;"),
    "z0_ignored": ("jl_oracle_maps.c", "n = map_escape_f64(jb->m, jb->m->z0r, jb->m->z0i, xd, yd, jb->max_iter);",
                   "n = map_escape_f64(jb->m, 0.0, 0.0, xd, yd, jb->max_iter);"),
}

MAP_CHECKS = [
    lambda: mpins.test_power2_equals_quadratic(oracle.FP64, oracle.JULIA),
    lambda: mpins.test_rational_forms_of_the_quadratic(oracle.FP64, oracle.MANDELBROT),
    lambda: mpins.test_power_c0_closed_form(oracle.FP64, 3),
    lambda: mpins.test_power_c0_closed_form(oracle.FP64, 5),
    lambda: mpins.test_power_step_against_high_precision(oracle.FP64),
    lambda: mpins.test_rational_step_against_high_precision(oracle.FP64),
    lambda: mpins.test_fig4_as_printed_is_z4_plus_1(oracle.FP64),
    lambda: mpins.test_exact_orbits_and_bailout(oracle.FP64),
    lambda: mpins.test_parameter_plane_starts_from_z0(oracle.FP64),
]


@pytest.mark.parametrize("name", sorted(MAP_MUTANTS))
def test_map_pins_catch_mutant(name, tmp_path, monkeypatch):
    fname, old, new = MAP_MUTANTS[name]
    for f in ("jl_oracle_maps.c", "map_iter.inc"):
        src = open(os.path.join(os.path.dirname(obuild.SRC), f)).read()
        if f == fname:
            assert src.count(old) >= 1, old
            src = src.replace(old, new, 1)
        (tmp_path / f).write_text(src)
    so = tmp_path / "m.so"
    subprocess.check_call(["gcc", *obuild.CFLAGS, "-I", str(tmp_path), obuild.SRC, str(tmp_path / "jl_oracle_maps.c"),
                           "-o", str(so), "-lm"])
    real = oracle._load()
    L = ctypes.CDLL(str(so))
    for fn in ("jlo_render", "jlo_escape_point", "jlo_colour", "jlo_hist", "jlo_render_map",
               "jlo_map_escape_point", "jlo_map_step"):
        f = getattr(L, fn)
        r = getattr(real, fn)
        f.argtypes, f.restype = r.argtypes, r.restype

    class Proxy:
        def __getattr__(self, k):
            return getattr(L, k)

    monkeypatch.setattr(oracle, "_lib", Proxy())
    caught = 0
    for chk in MAP_CHECKS:
        try:
            chk()
        except AssertionError:
            caught += 1
    assert caught >= 1, "mutant %s survived every map pin" % name


# ---- surrogate network (oracle/mlp.py) -------------------------------------
import importlib.util  # noqa: E402

from oracle import mlp as real_mlp  # noqa: E402
from tests import test_oracle_mlp as mlp_pins  # noqa: E402

MLP_MUTANTS = {
    "drop_relu1": ("h1 = _q(np.maximum(a1, 0.0), quant)", "h1 = _q(a1, quant)"),
    "drop_relu2": ("h2 = _q(np.maximum(a2, 0.0), quant)", "h2 = _q(a2, quant)"),
    "drop_bias1": ('.T + P["b1"]', ".T"),
    "drop_bias2": ('.T + P["b2"]', ".T"),
    "drop_bias3": ('.T + P["b3"]', ".T"),
    "sin_cos_swapped": ("[np.sin(2 * np.pi * t), np.cos(2 * np.pi * t)]",
                        "[np.cos(2 * np.pi * t), np.sin(2 * np.pi * t)]"),
    "no_two_pi": ("[np.sin(2 * np.pi * t), np.cos(2 * np.pi * t)]", "[np.sin(np.pi * t), np.cos(np.pi * t)]"),
    "c_parts_swapped": ("c32[:, None, 0] * B32[None, :, 0] + c32[:, None, 1] * B32[None, :, 1]",
                        "c32[:, None, 1] * B32[None, :, 0] + c32[:, None, 0] * B32[None, :, 1]"),
    "phase_in_float64": ("    t = t.astype(np.float64)\n", "    t = c32.astype(np.float64) @ B32.astype(np.float64).T\n"),
    "w2_transposed": ('a2 = h1 @ _q(P["W2"], quant).T', 'a2 = h1 @ _q(P["W2"], quant)'),
    "dz_not_rounded": ("dzq = _q(dz, quant)", "dzq = dz"),
    "dz2_not_rounded": ("dz2q = _q(dz2, quant)", "dz2q = dz2"),
    "bias_grad_rounded": ('"b3": dz.sum(axis=0)', '"b3": dzq.sum(axis=0)'),
    "no_mean_over_rows": ('dz = (f["p"] - T) / n', 'dz = (f["p"] - T)'),
    "mask_dropped": ('dz1 = dh1 * (f["h1"] > 0)', "dz1 = dh1"),
    "mask_wrong_layer": ('dz2 = dh2 * (f["h2"] > 0)', 'dz2 = dh2 * (f["h1"] > 0)'),
    "dw2_wrong_input": ('g["W2"] = dz2q.T @ f["h1"]', 'g["W2"] = dz2q.T @ f["h2"]'),
    "dh1_not_transposed": ('dh1 = dz2q @ _q(P["W2"], quant)', 'dh1 = dz2q @ _q(P["W2"], quant).T'),
    "adam_bias_correction": ("mh = mk / (1 - beta1 ** t)", "mh = mk / (1 - beta1 ** (t + 1))"),
    "adam_no_sqrt": ("(np.sqrt(vh) + eps)", "(vh + eps)"),
}

MLP_CHECKS = [mlp_pins.check_hand_forward, mlp_pins.check_hand_grads, mlp_pins.check_adam_constant_gradient,
              mlp_pins.check_features_binary32_phase]


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_mlp_pins_catch_mutant(name, tmp_path):
    old, new = MLP_MUTANTS[name]
    src = open(real_mlp.__file__).read()
    assert src.count(old) == 1, old
    path = tmp_path / "mlp_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("mlp_mutant", str(path))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    caught = 0
    for chk in MLP_CHECKS:
        try:
            chk(m)
        except (AssertionError, ValueError):
            caught += 1
    assert caught >= 1, "mutant %s survived every surrogate pin" % name
