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


def test_forward_matches_oracle(cuda):
    import torch
    p, B = setup_model()
    md = Model(p, B)
    c = wl.survey_c(1000, seed=11)
    cd = torch.from_numpy(c).cuda()
    probs = torch.zeros((1000, 101), dtype=torch.float32, device="cuda")
    score = torch.zeros(1000, dtype=torch.float32, device="cuda")
    _lib.check(md.L.jl_model_forward(md.h, cd.data_ptr(), 1000, probs.data_ptr(), score.data_ptr(), None))
    torch.cuda.synchronize()
    ref = mlp.forward({k: v.astype(np.float64) for k, v in p.items()}, c, B, quant=True)["p"]
    got = probs.cpu().numpy().astype(np.float64)
    l1 = np.abs(got - ref).sum(axis=1)
    assert l1.mean() < 2e-3 and l1.max() < 2e-2, (l1.mean(), l1.max())
    assert np.abs(score.cpu().numpy() - mlp.entropy(got)).max() < 1e-4
    md.close()


def test_gradients_match_oracle(cuda):
    import torch
    p, B = setup_model(1)
    md = Model(p, B)
    n = 512
    c = wl.survey_c(n, seed=12)
    T = targets(n)
    cd, Td = torch.from_numpy(c).cuda(), torch.from_numpy(T).cuda()
    loss = ctypes.c_float(0)
    g = np.zeros(md.L.jl_model_num_params(), np.float32)
    _lib.check(md.L.jl_model_grads(md.h, cd.data_ptr(), Td.data_ptr(), n, ctypes.byref(loss), g.ctypes.data, None))
    L_ref, g_ref = mlp.grads({k: v.astype(np.float64) for k, v in p.items()}, c, B, T, quant=True)
    assert abs(loss.value - L_ref) < 1e-4 * abs(L_ref)
    gg = unflatten(g)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        rel = np.linalg.norm(gg[k] - g_ref[k]) / np.linalg.norm(g_ref[k])
        assert rel < 2e-2, (k, rel)
    md.close()


def test_adam_steps_match_oracle(cuda):
    import torch
    p, B = setup_model(2)
    md = Model(p, B)
    n, batch = 2048, 1024
    c = wl.survey_c(n, seed=13)
    T = targets(n, seed=3)
    cd, Td = torch.from_numpy(c).cuda(), torch.from_numpy(T).cuda()
    curve = np.zeros(1, np.float32)
    _lib.check(md.L.jl_train(md.h, cd.data_ptr(), Td.data_ptr(), n, None, 1, batch, ctypes.c_float(1e-3),
                             ctypes.c_float(1e-3), curve.ctypes.data, None))
    got, m, v, step = md.state()
    assert step == 2
    q = {k: v_.astype(np.float64) for k, v_ in p.items()}
    mm = {k: np.zeros_like(v_) for k, v_ in q.items()}
    vv = {k: np.zeros_like(v_) for k, v_ in q.items()}
    for s in range(2):
        sl = slice(s * batch, (s + 1) * batch)
        _, g = mlp.grads(q, c[sl], B, T[sl], quant=True)
        q, mm, vv = mlp.adam_step(q, g, mm, vv, s + 1)
    ref = flatten(q)
    d0 = flatten({k: v_.astype(np.float64) for k, v_ in p.items()})
    # parameter change matches the oracle's change
    rel = np.linalg.norm((got - d0) - (ref - d0)) / np.linalg.norm(ref - d0)
    assert rel < 5e-2, rel
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
        assert np.abs(out["fused"][0] - ref).sum(axis=1).max() < 2e-2
    md.close()
