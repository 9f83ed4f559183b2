"""GPU checks of the learned surrogate: the tcgen05 product against numpy on
bfloat16-rounded operands, forward / gradients / Adam against the float64
oracle with the same bfloat16 rounding points, exact top-k, checkpoints."""
import ctypes

import numpy as np
import pytest

from oracle import mlp
from paper_1611_03079_b300 import _lib, workloads as wl

pytestmark = pytest.mark.gpu


def bf16_bits(x):
    """float array -> uint16 bfloat16 bits (round to nearest even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def to_dev_bf16(x):
    import torch
    return torch.from_numpy(bf16_bits(x).view(np.int16).copy()).cuda()


@pytest.mark.parametrize("M,N,K,at,bt", [
    (128, 16, 64, 0, 0), (128, 256, 64, 0, 0), (200, 112, 130, 0, 0), (300, 64, 256, 0, 1),
    (101, 256, 1024, 1, 1), (256, 64, 1024, 1, 1), (1024, 256, 101, 0, 1), (77, 48, 9, 1, 0),
])
def test_tc_gemm_matches_numpy(cuda, M, N, K, at, bt):
    import torch
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((K, N))
    Ast = A.T.copy() if at else A                 # at=1: stored K x M
    Bst = Bm if bt else Bm.T.copy()               # bt=0: stored N x K
    Ad, Bd = to_dev_bf16(Ast), to_dev_bf16(Bst)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = _lib.lib()
    _lib.check(L.jl_gemm_bf16(Ad.data_ptr(), Ast.shape[1], at, Bd.data_ptr(), Bst.shape[1], bt, M, N, K,
                              C.data_ptr(), N, st.data_ptr(), None))
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = mlp.bf16(A) @ mlp.bf16(Bm)
    got = C.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref).max()
    scale = (np.abs(mlp.bf16(A)) @ np.abs(mlp.bf16(Bm))).max()
    assert err <= 1e-5 * scale, (err, scale)


# ------------------------------------------------------------- the model ----
class Model:
    def __init__(self, params, B):
        self.L = _lib.lib()
        flat = np.concatenate([params[k].astype(np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
        assert flat.size == self.L.jl_model_num_params()
        self.h = ctypes.c_void_p()
        B = np.ascontiguousarray(B, np.float32)
        _lib.check(self.L.jl_model_create(B.ctypes.data, flat.ctypes.data, ctypes.byref(self.h)))

    def state(self):
        n = self.L.jl_model_num_params()
        p, m, v = (np.zeros(n, np.float32) for _ in range(3))
        s = ctypes.c_int32(0)
        _lib.check(self.L.jl_model_get_state(self.h, p.ctypes.data, m.ctypes.data, v.ctypes.data, ctypes.byref(s)))
        return p, m, v, s.value

    def close(self):
        self.L.jl_model_destroy(self.h)


def unflatten(flat):
    shapes = [("W1", (256, 64)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (101, 256)),
              ("b3", (101,))]
    out, o = {}, 0
    for k, s in shapes:
        n = int(np.prod(s))
        out[k] = np.asarray(flat[o:o + n], np.float64).reshape(s)
        o += n
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[k], np.float64).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def setup_model(seed=0):
    p = wl.mlp_init(seed)
    rng = np.random.default_rng(seed + 50)
    for k in ("b1", "b2", "b3"):
        p[k] = (rng.standard_normal(p[k].shape) * 0.1).astype(np.float32)
    return p, wl.fourier_matrix()


def targets(n, seed=1):
    rng = np.random.default_rng(seed)
    t = rng.random((n, 101)) ** 4
    return (t / t.sum(axis=1, keepdims=True)).astype(np.float32)


RTOL = 1e-2   # bfloat16 operands: the gradient tolerance of the survey's pins


def assert_close(name, got, ref, rtol, atol):
    """Element-wise |got - ref| <= atol + rtol |ref| (atol a scalar or an
    array of per-element bounds)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    bound = atol + rtol * np.abs(ref)
    bad = err > bound
    if bad.any():
        k = np.unravel_index(np.argmax(err - bound), err.shape)
        raise AssertionError("%s: %d of %d elements outside the bound; worst at %s: got %.6e ref %.6e bound %.3e"
                             % (name, int(bad.sum()), bad.size, k, got[k], ref[k], np.broadcast_to(bound, err.shape)[k]))


def forward_gpu(md, c, fn="jl_model_forward"):
    import torch
    n = c.shape[0]
    cd = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    probs = torch.zeros((n, 101), dtype=torch.float32, device="cuda")
    score = torch.zeros(n, dtype=torch.float32, device="cuda")
    _lib.check(getattr(md.L, fn)(md.h, cd.data_ptr(), n, probs.data_ptr(), score.data_ptr(), None))
    torch.cuda.synchronize()
    return probs.cpu().numpy(), score.cpu().numpy()


def check_forward(name, probs, score, ref):
    """Probabilities element-wise to 1e-2 relative (1e-7 absolute below, for
    bins whose probability underflows toward zero); entropy scores to 1e-2
    relative.  The remaining differences are rare bfloat16 rounding flips of
    features and activations (each moves a logit by about one bfloat16 unit
    of one term) and the hardware sine, cosine and exponential."""
    assert_close(name + " probs", probs, ref, RTOL, 1e-7)
    assert_close(name + " score", score, mlp.entropy(ref), RTOL, 1e-6)


def test_forward_matches_oracle(cuda):
    """Fused and per-layer forward on 1,000 values of C against the float64
    oracle with bfloat16 operands, element by element."""
    p, B = setup_model()
    md = Model(p, B)
    c = wl.survey_c(1000, seed=11)
    ref = mlp.forward({k: v.astype(np.float64) for k, v in p.items()}, c, B, quant=True)["p"]
    for fn in ("jl_model_forward", "jl_model_forward_layered"):
        probs, score = forward_gpu(md, c, fn)
        check_forward(fn, probs, score, ref)
    md.close()


def test_fused_forward_survey_sample(cuda):
    """The fused screening kernel over the 1,048,576 survey candidates (the
    bench's launch): 4,096 seeded rows against the oracle, element by element."""
    p, B = setup_model(5)
    md = Model(p, B)
    c = wl.survey_candidates()
    probs, score = forward_gpu(md, c)
    rows = np.sort(np.random.default_rng(7).choice(c.shape[0], 4096, replace=False))
    rows[-1] = c.shape[0] - 1                       # the last row of the ragged final tile
    ref = mlp.forward({k: v.astype(np.float64) for k, v in p.items()}, c[rows], B, quant=True)["p"]
    check_forward("fused 1M sample", probs[rows], score[rows], ref)
    md.close()


def well_conditioned(P, B, c, n, extra=0.0):
    """The first n rows of c whose ReLU arguments all lie farther from zero
    than two bfloat16 rounding flips of their largest term (plus `extra`)
    can move them.  Elsewhere a pre-activation within rounding distance of
    zero makes both mask bits correct answers, and the backward differs by
    that row's whole contribution; such rows are left out of the
    element-wise gradient comparisons."""
    f = mlp.forward(P, c, B, quant=True)
    W1q, W2q = np.abs(mlp.bf16(P["W1"])), np.abs(mlp.bf16(P["W2"]))
    keep = []
    for r in range(c.shape[0]):
        t1 = W1q * np.abs(f["phi"][r])[None, :]
        t2 = W2q * np.abs(f["h1"][r])[None, :]
        tau1 = 2.0 ** -6 * t1.max(axis=1) + 2.0 ** -14 * t1.sum(axis=1) + extra
        tau2 = 2.0 ** -6 * t2.max(axis=1) + 2.0 ** -14 * t2.sum(axis=1) + extra
        if (np.abs(f["a1"][r]) > tau1).all() and (np.abs(f["a2"][r]) > tau2).all():
            keep.append(r)
            if len(keep) == n:
                break
    assert len(keep) == n, "only %d well-conditioned rows" % len(keep)
    return np.ascontiguousarray(c[keep])


def _max_term(a, b):
    """max over rows r of |a[r, i]| |b[r, k]| (the largest term of a^T b)."""
    out = np.zeros((a.shape[1], b.shape[1]))
    for r in range(a.shape[0]):
        np.maximum(out, np.outer(np.abs(a[r]), np.abs(b[r])), out=out)
    return out


def grad_bounds(t):
    """Per-element absolute tolerances of the gradients: 2^-6 of the largest
    term of each sum (a bfloat16 rounding flip moves an operand by at most
    2^-7 of itself -- one unit in the last of its 8 significand bits -- and
    each term has two bfloat16 operands that may both flip: the error and
    the activation or feature) plus 2^-14 of the sum of the terms'
    magnitudes (binary32 accumulation and small upstream differences)."""
    q = 2.0 ** -6
    s = 2.0 ** -14
    out = {}
    for W, b, d, dq, h in (("W3", "b3", "dz", "dzq", "h2"), ("W2", "b2", "dz2", "dz2q", "h1"),
                           ("W1", "b1", "dz1", "dz1q", "phi")):
        out[W] = q * _max_term(t[dq], t[h]) + s * (np.abs(t[dq]).T @ np.abs(t[h]))
        out[b] = q * np.abs(t[d]).max(axis=0) + s * np.abs(t[d]).sum(axis=0)
    return out


def gpu_grads(md, c, T):
    import torch
    n = c.shape[0]
    cd, Td = torch.from_numpy(np.ascontiguousarray(c)).cuda(), torch.from_numpy(np.ascontiguousarray(T)).cuda()
    loss = ctypes.c_float(0)
    g = np.zeros(md.L.jl_model_num_params(), np.float32)
    _lib.check(md.L.jl_model_grads(md.h, cd.data_ptr(), Td.data_ptr(), n, ctypes.byref(loss), g.ctypes.data, None))
    return loss.value, unflatten(g)


@pytest.mark.parametrize("n", [512, 300, 129, 1])
def test_gradients_match_oracle(cuda, n):
    """Loss and every gradient tensor element by element (n well-conditioned
    rows: whole 128-row tiles, a ragged last tile, a single row), against the
    oracle's backward with the same bfloat16 rounding points."""
    p, B = setup_model(1)
    P = {k: v.astype(np.float64) for k, v in p.items()}
    md = Model(p, B)
    c = well_conditioned(P, B, wl.survey_c(12000, seed=12 + n), n)
    T = targets(n, seed=1 + n)
    L_gpu, g = gpu_grads(md, c, T)
    L_ref, g_ref, t = mlp.grads(P, c, B, T, quant=True, terms=True)
    assert abs(L_gpu - L_ref) <= 1e-5 * abs(L_ref)
    bounds = grad_bounds(t)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert_close("grad " + k, g[k], g_ref[k], RTOL, bounds[k])
    md.close()


def adam_change_range(m, v, dm, dv, step, lr, eps=1e-8):
    """Range of the Adam change -lr m_hat / (sqrt(v_hat) + eps) over the box
    |m' - m| <= dm, |v' - v| <= dv (the change is monotone in each, so the
    extremes are at the corners)."""
    bc1, bc2 = 1 - 0.9 ** step, 1 - 0.999 ** step
    vals = [-lr * (mm / bc1) / (np.sqrt(vv / bc2) + eps)
            for mm in (m - dm, m + dm) for vv in (np.maximum(v - dv, 0.0), v + dv)]
    return np.minimum.reduce(vals), np.maximum.reduce(vals)


def test_adam_steps_match_oracle(cuda):
    """Two training steps (batch 512 each, well-conditioned rows) against the
    oracle's Adam, element by element.  The gradient tolerances propagate
    into bounds on the moments m = sum (1 - b1) b1^(t-s) g_s and
    v = sum (1 - b2) b2^(t-s) g_s^2, which are checked everywhere, and the
    parameter change -lr m_hat / (sqrt(v_hat) + eps) must lie in its range
    over those bounds.  Where |g| is within its tolerance of zero that range
    takes in both signs (either sign is a correct first step there);
    elsewhere it is narrow, and the test requires it to be narrow for most
    parameters.  Step 2 starts both sides from the oracle's parameters after
    step 1 (set on the GPU), so its gradient is evaluated at the same point."""
    import torch
    p, B = setup_model(2)
    P = {k: v.astype(np.float64) for k, v in p.items()}
    md = Model(p, B)
    lr, batch = 1e-3, 512
    mm = {k: np.zeros_like(v) for k, v in P.items()}
    vv = {k: np.zeros_like(v) for k, v in P.items()}
    dm = {k: np.zeros_like(v) for k, v in P.items()}
    dv = {k: np.zeros_like(v) for k, v in P.items()}
    q = P
    for step in (1, 2):
        if step == 2:
            flat = flatten(q).astype(np.float32)
            _lib.check(md.L.jl_model_set_state(md.h, flat.ctypes.data, None, None, None))
            q = unflatten(flat.astype(np.float64))       # the binary32 values the GPU starts from
        c = well_conditioned(q, B, wl.survey_c(12000, seed=12 + step), batch)
        T = targets(batch, seed=2 + step)
        _, g_ref, t = mlp.grads(q, c, B, T, quant=True, terms=True)
        gb = grad_bounds(t)
        q_next, mm, vv = mlp.adam_step(q, g_ref, mm, vv, step, lr=lr)
        cd, Td = torch.from_numpy(c).cuda(), torch.from_numpy(T).cuda()
        _lib.check(md.L.jl_train(md.h, cd.data_ptr(), Td.data_ptr(), batch, None, 1, batch, ctypes.c_float(lr),
                                 ctypes.c_float(lr), None, None))
        got, m, v, st = md.state()
        assert st == step
        got, m, v = unflatten(got), unflatten(m), unflatten(v)
        for k in P:
            tol_g = gb[k] + RTOL * np.abs(g_ref[k])
            dm[k] = 0.9 * dm[k] + 0.1 * tol_g
            dv[k] = 0.999 * dv[k] + 0.001 * (2 * np.abs(g_ref[k]) * tol_g + tol_g ** 2)
            assert_close("adam m %s step %d" % (k, step), m[k], mm[k], 1e-6, dm[k] + 1e-30)
            assert_close("adam v %s step %d" % (k, step), v[k], vv[k], 1e-6, dv[k] + 1e-30)
            lo, hi = adam_change_range(mm[k], vv[k], dm[k], dv[k], step, lr)
            d_gpu = got[k] - q[k]
            slack = 1e-7                                  # binary32 rounding of the parameter itself
            bad = (d_gpu < lo - slack) | (d_gpu > hi + slack)
            assert not bad.any(), ("adam change", k, step, int(bad.sum()), d_gpu[bad][:4], lo[bad][:4], hi[bad][:4])
            narrow = (hi - lo) < 0.1 * lr
            assert narrow.mean() > 0.5, ("adam change ranges too wide to test", k, step, narrow.mean())
        q = q_next
    md.close()


def test_adam_refreshes_transposed_copies(cuda):
    """The training step reads packed bfloat16 weight images (W1, W2, W3 and
    the transposes W2^T, W3^T) that Adam rewrites in place at every step.
    After training steps, gradients computed with Adam's images equal, bit
    for bit, the gradients after the images are rebuilt from the binary32
    parameters by the packing kernel (whose images the oracle comparisons
    above check)."""
    import torch
    p, B = setup_model(4)
    md = Model(p, B)
    n, batch = 3072, 1024
    c = wl.survey_c(n, seed=16)
    T = targets(n, seed=5)
    cd, Td = torch.from_numpy(c).cuda(), torch.from_numpy(T).cuda()
    _lib.check(md.L.jl_train(md.h, cd.data_ptr(), Td.data_ptr(), n, None, 1, batch, ctypes.c_float(1e-3),
                             ctypes.c_float(1e-3), None, None))
    c2, T2 = wl.survey_c(700, seed=17), targets(700, seed=6)
    _, ga = gpu_grads(md, c2, T2)
    params = md.state()[0]
    _lib.check(md.L.jl_model_set_state(md.h, params.ctypes.data, None, None, None))
    _, gb = gpu_grads(md, c2, T2)
    for k in ga:
        assert (ga[k] == gb[k]).all(), k
    md.close()


def test_topk_exact(cuda):
    import torch
    L = _lib.lib()
    rng = np.random.default_rng(4)
    cases = []
    for n, k in ((1000, 10), (100000, 1000), (1 << 20, 10486)):
        s = rng.random(n).astype(np.float32) * 4.6
        s[rng.choice(n, n // 10, replace=False)] = np.float32(2.5)  # many ties
        cases.append((s, k))
    cases.append((rng.random(5000).astype(np.float32), 5000))                    # k = n
    cases.append((np.full(70000, 1.75, np.float32), 1))                           # all equal: first index
    cases.append((np.full(70000, 1.75, np.float32), 16384))                       # all equal, k at its maximum
    # values sharing their top 22 bits: the rank is decided in the last digit level
    cases.append(((1.0 + rng.integers(0, 1024, 300000) * 2.0 ** -23).astype(np.float32), 16384))
    cases.append((np.zeros(40000, np.float32), 123))                              # all zero
    for s, k in cases:
        n = s.shape[0]
        sd = torch.from_numpy(s).cuda()
        idx = torch.zeros(k, dtype=torch.int32, device="cuda")
        val = torch.zeros(k, dtype=torch.float32, device="cuda")
        _lib.check(L.jl_topk(sd.data_ptr(), n, k, idx.data_ptr(), val.data_ptr(), None))
        torch.cuda.synchronize()
        ref = mlp.top_k(s, k)
        assert (idx.cpu().numpy() == ref).all()
        assert (val.cpu().numpy() == s[ref]).all()


def test_checkpoint_resume_bit_identical(cuda, tmp_path):
    import torch
    p, B = setup_model(3)
    n, batch = 2048, 512
    c = wl.survey_c(n, seed=14)
    T = targets(n, seed=4)
    cd, Td = torch.from_numpy(c).cuda(), torch.from_numpy(T).cuda()
    a = Model(p, B)
    _lib.check(a.L.jl_train(a.h, cd.data_ptr(), Td.data_ptr(), n, None, 1, batch, ctypes.c_float(1e-3), ctypes.c_float(1e-3), None, None))
    path = str(tmp_path / "ck.bin").encode()
    _lib.check(a.L.jl_model_save(a.h, path))
    _lib.check(a.L.jl_train(a.h, cd.data_ptr(), Td.data_ptr(), n, None, 1, batch, ctypes.c_float(1e-3), ctypes.c_float(1e-3), None, None))
    b = Model(p, B)
    b.L.jl_model_destroy(b.h)
    b.h = ctypes.c_void_p()
    _lib.check(b.L.jl_model_load(path, ctypes.byref(b.h)))
    _lib.check(b.L.jl_train(b.h, cd.data_ptr(), Td.data_ptr(), n, None, 1, batch, ctypes.c_float(1e-3), ctypes.c_float(1e-3), None, None))
    sa, sb = a.state(), b.state()
    for x, y in zip(sa[:3], sb[:3]):
        assert (x == y).all()
    assert sa[3] == sb[3] == 8
    a.close()
    b.close()


@pytest.mark.parametrize("n", [1, 127, 50001])
def test_fused_forward_matches_layered(cuda, n):
    """The fused screening kernel (one persistent launch) and the per-layer
    product kernels compute the same network."""
    import torch
    p, B = setup_model(5)
    md = Model(p, B)
    c = torch.from_numpy(wl.survey_c(n, seed=15)).cuda()
    out = {}
    for name, fn in (("fused", md.L.jl_model_forward), ("layered", md.L.jl_model_forward_layered)):
        P = torch.zeros((n, 101), dtype=torch.float32, device="cuda")
        S = torch.zeros(n, dtype=torch.float32, device="cuda")
        _lib.check(fn(md.h, c.data_ptr(), n, P.data_ptr(), S.data_ptr(), None))
        torch.cuda.synchronize()
        out[name] = (P.cpu().numpy(), S.cpu().numpy())
    assert np.abs(out["fused"][0] - out["layered"][0]).max() <= 1e-6
    assert np.abs(out["fused"][1] - out["layered"][1]).max() <= 5e-5
    if n <= 127:
        ref = mlp.forward({k: v.astype(np.float64) for k, v in p.items()}, c.cpu().numpy(), B, quant=True)["p"]
        check_forward("fused n=%d" % n, out["fused"][0], out["fused"][1], ref)
    md.close()
