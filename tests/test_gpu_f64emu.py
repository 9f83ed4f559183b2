"""The integer-pipe binary64 multiply, square and add against IEEE
round-to-nearest-even (numpy float64 on the host), bit for bit, on millions
of operands chosen to reach every path: exponent gaps 0..70, cancellation,
carries out of the significand, rounding ties, zeros of both signs, and the
edges of the normal range (where the routines must flag the case for the
hardware instead of answering)."""
import numpy as np
import pytest

import paper_1611_03079_b300 as jl

pytestmark = pytest.mark.gpu


def run(op, a, b):
    import torch
    ad = torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()
    bd = torch.from_numpy(np.ascontiguousarray(b, np.float64)).cuda()
    out = torch.empty_like(ad)
    sp = torch.empty(ad.numel(), dtype=torch.int32, device="cuda")
    jl._lib.check(jl._lib.lib().jl_selftest_f64(op, ad.data_ptr(), bd.data_ptr(), out.data_ptr(), sp.data_ptr(),
                                                ad.numel(), None))
    torch.cuda.synchronize()
    return out.cpu().numpy(), sp.cpu().numpy().astype(bool)


def rand_normal(rng, n, emin=-60, emax=60):
    m = rng.uniform(1.0, 2.0, n)
    e = rng.integers(emin, emax + 1, n)
    s = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    x = s * np.ldexp(m, e)
    # sprinkle significands with many trailing ones / zeros (rounding edges)
    k = rng.random(n) < 0.2
    u = x.view(np.uint64)
    u[k] = (u[k] | np.uint64(0x000FFFFFFFFFFF00)) & ~np.uint64(0xFF) | rng.integers(0, 256, k.sum()).astype(np.uint64)
    return u.view(np.float64)


def check(op, a, b, expect_fast=None):
    out, sp = run(op, a, b)
    with np.errstate(all="ignore"):
        ref = a * b if op == 0 else (a * a if op == 1 else a + b)
    ok = ~sp
    assert (out[ok].view(np.uint64) == ref[ok].view(np.uint64)).all(), \
        np.nonzero(out[ok].view(np.uint64) != ref[ok].view(np.uint64))[0][:5]
    if expect_fast is not None:
        assert not sp[expect_fast].any()
    return sp


@pytest.mark.parametrize("op", [0, 1])
def test_products(cuda, op):
    rng = np.random.default_rng(op)
    n = 2_000_000
    a = rand_normal(rng, n)
    b = rand_normal(rng, n)
    check(op, a, b, expect_fast=np.ones(n, bool))
    # zeros of both signs, and edges of the range (flagged, never wrong)
    z = np.array([0.0, -0.0, 1.5, -2.25, 1e-200, 1e200, 1e-160, 1e160, 2.2250738585072014e-308, 5e-324,
                  1.7976931348623157e308, np.inf])
    A, B = np.meshgrid(z, z)
    sp = check(op, A.ravel(), B.ravel())
    fast = np.isfinite(A.ravel()) & ((A.ravel() == 0) | (np.abs(A.ravel()) > 1e-300))
    assert not sp[(A.ravel() == 0) & (B.ravel() == 0)].any()


def test_sums(cuda):
    rng = np.random.default_rng(7)
    n = 2_000_000
    a = rand_normal(rng, n)
    gap = rng.integers(0, 71, n)
    b = rand_normal(rng, n, 0, 0) * np.ldexp(1.0, np.floor(np.log2(np.abs(a))).astype(int) - gap)
    check(2, a, b, expect_fast=np.ones(n, bool))
    # near-cancellation: b = -a (1 + k ulp)
    k = rng.integers(-4, 5, n)
    b2 = -(a.view(np.int64) + k).view(np.float64)
    check(2, a, b2, expect_fast=np.ones(n, bool))
    # exact ties: a has its last bit set, b = a * 2^-53 (half an ulp)
    a3 = (rand_normal(rng, n).view(np.uint64) | np.uint64(1)).view(np.float64)
    b3 = np.ldexp(np.abs(a3), -53) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    check(2, a3, b3, expect_fast=np.ones(n, bool))
    # zeros
    z = np.array([0.0, -0.0, 1.0, -1.0, 3.5e-5])
    A, B = np.meshgrid(z, z)
    sp = check(2, A.ravel(), B.ravel())
    assert not sp.any()
    out, _ = run(2, np.array([-0.0, 0.0, -0.0, 2.0]), np.array([-0.0, -0.0, 0.0, -2.0]))
    assert list(np.signbit(out)) == [True, False, False, False]


def test_iteration_range_is_fast(cuda):
    """Operands of the escape iteration (|values| <= 16, coordinates and C
    down to 1e-30 apart) never need the hardware fallback."""
    rng = np.random.default_rng(9)
    n = 1_000_000
    x = rng.uniform(-4, 4, n) * 10.0 ** rng.integers(-30, 1, n)
    y = rng.uniform(-4, 4, n) * 10.0 ** rng.integers(-30, 1, n)
    for op in (0, 1, 2):
        check(op, x, y, expect_fast=np.ones(n, bool))
