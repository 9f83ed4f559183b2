"""C-ABI checks that need no GPU: libjl.so loads, exports every function that
include/*.h declares, and its host-side logic (argument validation, precision
rule, palette, variant table) behaves as documented."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_1611_03079_b300 import _lib, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(jl_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_1611_03079_b300 import build
    build.build()
    return _lib.lib()


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 8
    out = subprocess.check_output(["nm", "-D", "--defined-only", _lib.LIB_PATH]).decode()
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(L, n)
    # and the binding knows every one of them
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)


def test_select_precision_matches_oracle_rule(L):
    rng = np.random.default_rng(0)
    for _ in range(2000):
        cx, cy = rng.uniform(-2, 2, size=2)
        w = 10 ** rng.uniform(-14, 0.7)
        W = int(rng.integers(1, 4000))
        H = int(rng.integers(1, 3000))
        h = w * H / W
        rect = (cx - w / 2, cx + w / 2, cy - h / 2, cy + h / 2)
        if not (rect[0] < rect[1] and rect[2] < rect[3]):
            continue
        got = L.jl_select_precision(_lib.Rect(*rect), W, H)
        assert got == oracle.precision_for_view(rect, W, H)
    assert L.jl_select_precision(_lib.Rect(1.0, 0.0, 0.0, 1.0), 4, 4) == -1


def _render(L, **kw):
    args = dict(cr=0.0, ci=0.0, rect=(-2.0, 2.0, -2.0, 2.0), W=16, H=16, max_iter=100, prec=0, mode=0, ct=2,
                counts=1, rgba=None, pal=None, hist=None, stream=None)
    args.update(kw)
    return L.jl_render(args["cr"], args["ci"], _lib.Rect(*args["rect"]), args["W"], args["H"],
                       args["max_iter"], args["prec"], args["mode"], args["ct"], args["counts"], args["rgba"],
                       args["pal"], args["hist"], args["stream"])


@pytest.mark.parametrize("kw,frag", [
    (dict(W=0), "width"), (dict(H=70000), "width"), (dict(max_iter=0), "max_iter"),
    (dict(max_iter=65536), "max_iter"), (dict(rect=(1.0, -1.0, 0.0, 1.0)), "rect"),
    (dict(rect=(float("nan"), 1.0, 0.0, 1.0)), "rect"), (dict(mode=3), "mode"), (dict(prec=7), "precision"),
    (dict(ct=1, max_iter=256), "U8"), (dict(ct=0), "count_type"), (dict(ct=9), "count_type"),
    (dict(cr=float("inf")), "finite"), (dict(ct=0, counts=None), "no output"),
])
def test_argument_validation(L, kw, frag):
    rc = _render(L, **kw)
    assert rc == _lib.JL_EINVAL
    assert frag in L.jl_last_error().decode()


def test_default_palette(L):
    out = np.zeros((256, 4), np.uint8)
    assert L.jl_default_palette(out.ctypes.data) == 0
    assert (out[255] == [0, 0, 0, 255]).all()
    assert (out[:, 3] == 255).all()
    assert len({tuple(r) for r in out[:255]}) > 100


def test_variant_list(L):
    for prec in (0, 1):
        n = L.jl_variant_list(prec, None, 0)
        assert n >= 3
        buf = (ctypes.c_int32 * (2 * n))()
        assert L.jl_variant_list(prec, buf, n) == n
        pairs = [(buf[2 * i], buf[2 * i + 1]) for i in range(n)]
        assert pairs[0] == (0, 0)  # the static tile kernel
        # (0, T): the compacting tile kernel (binary32 only), parking threshold T
        compact = [u for p, u in pairs[1:] if p == 0]
        assert all(1 <= u <= 32 for u in compact) and (prec == 0 or not compact)
        assert all(p >= 1 and u >= 1 for p, u in pairs[1:] if p != 0)
    assert L.jl_variant_list(5, None, 0) == -1


def test_version(L):
    assert b"sm_103a" in L.jl_version()


def test_product_does_not_reference_oracle():
    """The product package never imports or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_1611_03079_b300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if path.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "jl_oracle" not in text and "jlo_" not in text, path


def test_tune_load_rejects_malformed(L, tmp_path):
    p = tmp_path / "bad.txt"
    p.write_text("0 0 0 3 3 128 0 1 1.0\n")  # (ppt 3, unroll 3) is not a variant
    assert L.jl_tune_load(str(p).encode()) == _lib.JL_EINVAL
    assert b"malformed" in L.jl_last_error()
    assert L.jl_tune_load(b"/nonexistent/x") == _lib.JL_EINVAL


def test_batch_create_validation(L):
    import ctypes
    f = _lib.Frame(0.0, 0.0, _lib.Rect(-2, 2, -2, 2), 16, 16, 100, 0, 0, 2, 0, -1, -1)
    h = ctypes.c_void_p()
    # counts offset given but no base pointer
    rc = L.jl_batch_create(ctypes.byref(f), 1, None, None, None, None, None, ctypes.byref(h))
    assert rc == _lib.JL_EINVAL and b"base pointer" in L.jl_last_error()
    # odd uint16 offset
    f.counts_offset = 1
    rc = L.jl_batch_create(ctypes.byref(f), 1, ctypes.c_void_p(256), None, None, None, None, ctypes.byref(h))
    assert rc == _lib.JL_EINVAL and b"even" in L.jl_last_error()
    rc = L.jl_batch_create(ctypes.byref(f), 0, None, None, None, None, None, ctypes.byref(h))
    assert rc == _lib.JL_EINVAL


def _map_call(L, m, **kw):
    import paper_1611_03079_b300 as jl
    spec = m if isinstance(m, _lib.Map) else jl.make_map(m)
    args = dict(cr=0.0, ci=0.0, rect=(-2.0, 2.0, -2.0, 2.0), W=16, H=16, max_iter=100, prec=0, mode=0, ct=2,
                counts=1)
    args.update(kw)
    return L.jl_render_map(ctypes.byref(spec), args["cr"], args["ci"], _lib.Rect(*args["rect"]), args["W"],
                           args["H"], args["max_iter"], args["prec"], args["mode"], args["ct"], args["counts"],
                           None, None, None, None)


def test_render_map_validation(L):
    """Generic-map arguments are rejected on the host, before any device use."""
    cases = [
        (wl.power_map(1), {}, "degree"), (wl.power_map(17), {}, "degree"),
        (dict(wl.power_map(3), bailout=0.0), {}, "bailout"),
        (dict(wl.power_map(3), bailout=float("inf")), {}, "bailout"),
        (dict(wl.power_map(3), z0=complex(float("nan"), 0)), {}, "z0"),
        (wl.rational_map([1, float("inf")], [1]), {}, "numerator"),
        (wl.rational_map([1], [complex(0, float("nan"))]), {}, "denominator"),
        (wl.power_map(3), dict(W=0), "width"), (wl.power_map(3), dict(max_iter=0), "max_iter"),
        (wl.fig4_map(), dict(mode=5), "mode"),
    ]
    for m, kw, frag in cases:
        assert _map_call(L, m, **kw) == _lib.JL_EINVAL, (m, kw)
        assert frag in L.jl_last_error().decode(), (frag, L.jl_last_error())
    bad = _lib.Map()
    bad.kind = 7
    assert _map_call(L, bad) == _lib.JL_EINVAL and "kind" in L.jl_last_error().decode()
    bad = _lib.Map()
    bad.kind, bad.num_degree, bad.den_degree, bad.bailout = 1, 9, 0, 4.0
    assert _map_call(L, bad) == _lib.JL_EINVAL and "degrees" in L.jl_last_error().decode()
    assert L.jl_render_map(None, 0.0, 0.0, _lib.Rect(-1, 1, -1, 1), 4, 4, 10, 0, 0, 2, 1, None, None, None,
                           None) == _lib.JL_EINVAL


def test_host_plan_validation(L):
    """Host plans reject bad depths and frames on the host, before any device
    use; the launch count of a NULL plan is -1."""
    f = _lib.Frame(0.0, 0.0, _lib.Rect(-2, 2, -2, 2), 16, 16, 100, 0, 0, 2, 0, -1, -1)
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(1024)
    for depth in (-1, 65):
        rc = L.jl_host_plan_create(ctypes.byref(f), 1, buf, None, None, None, depth, ctypes.byref(h))
        assert rc == _lib.JL_EINVAL and b"depth" in L.jl_last_error(), depth
        assert not h.value
    rc = L.jl_host_plan_create(ctypes.byref(f), 0, buf, None, None, None, 0, ctypes.byref(h))
    assert rc == _lib.JL_EINVAL
    # counts offset given but no base pointer
    rc = L.jl_host_plan_create(ctypes.byref(f), 1, None, None, None, None, 0, ctypes.byref(h))
    assert rc == _lib.JL_EINVAL and b"base pointer" in L.jl_last_error()
    assert L.jl_host_plan_run(None, None) == _lib.JL_EINVAL
    assert L.jl_host_plan_launches(None) == -1


def test_probe_validation(L):
    """Issue-rate probe kinds 0..2 only, and at least one iteration; checked
    on the host before any device use."""
    ops = ctypes.c_double(0)
    for kind, iters in ((-1, 10), (3, 10), (1, 0)):
        assert L.jl_probe_peak(kind, iters, ctypes.byref(ops), None, None) == _lib.JL_EINVAL, (kind, iters)
    assert b"packed binary32" in L.jl_last_error() or b"iters" in L.jl_last_error()
