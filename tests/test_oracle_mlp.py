"""Pins for the surrogate oracle (oracle/mlp.py): gradients against finite
differences, Adam's first step in closed form, softmax / feature identities,
and bfloat16 rounding on hand-worked values."""
import numpy as np
import pytest

from oracle import mlp
from paper_1611_03079_b300 import workloads as wl


def small_params(seed=0, scale=1.0):
    p = wl.mlp_init(seed)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3"):
        p[k] = (rng.standard_normal(p[k].shape) * 0.1).astype(np.float32)
    return {k: v.astype(np.float64) * (scale if k.startswith("W") else 1.0) for k, v in p.items()}


def targets(n, seed=1):
    rng = np.random.default_rng(seed)
    t = rng.random((n, mlp.N_BINS)) ** 4
    return t / t.sum(axis=1, keepdims=True)


def test_gradients_match_finite_differences():
    """Central differences (step 1e-6) of the float64 loss against the
    analytic backward for a sample of entries of every parameter."""
    p = small_params()
    B = wl.fourier_matrix()
    c = wl.survey_c(6, seed=5).astype(np.float64)
    T = targets(6)
    L, g = mlp.grads(p, c, B, T)
    assert abs(L - mlp.loss(p, c, B, T)) < 1e-12
    rng = np.random.default_rng(3)
    h = 1e-6
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, 12, replace=False):
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k].reshape(-1)[idx] += h
            lp = mlp.loss(q, c, B, T)
            q[k].reshape(-1)[idx] -= 2 * h
            lm = mlp.loss(q, c, B, T)
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, idx, fd, an)


def test_softmax_and_loss_identities():
    p = small_params()
    B = wl.fourier_matrix()
    c = wl.survey_c(50, seed=6)
    f = mlp.forward(p, c, B)
    assert np.allclose(f["p"].sum(axis=1), 1.0, atol=1e-12)
    # the gradient wrt the logits vanishes when the target equals the prediction
    L, g = mlp.grads(p, c, B, f["p"])
    assert np.abs(g["b3"]).max() < 1e-15 and np.abs(g["W3"]).max() < 1e-15
    # cross-entropy of a distribution with itself is its entropy
    assert abs(L - mlp.entropy(f["p"]).mean()) < 1e-12


def test_features():
    B = wl.fourier_matrix()
    c = wl.survey_c(20, seed=7)
    phi = mlp.features(c, B)
    assert phi.shape == (20, 64)
    assert np.allclose(phi[:, :32] ** 2 + phi[:, 32:] ** 2, 1.0, atol=1e-14)
    z = mlp.features(np.zeros((1, 2)), B)
    assert (z[0, :32] == 0).all() and (z[0, 32:] == 1).all()
    # integer-period shift: C -> C + e with B e integer leaves phi unchanged
    Bi = np.array([[1.0, 0.0], [2.0, 3.0]])
    a = mlp.features(np.array([[0.1, 0.2]]), Bi)
    b = mlp.features(np.array([[1.1, 0.2]]), Bi)
    assert np.allclose(a[:, [0, 2]], b[:, [0, 2]], atol=1e-12)


def test_adam_first_step_closed_form():
    """First Adam step: m_hat = g and v_hat = g^2, so the update is
    -lr * g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    p = {"w": rng.standard_normal(100)}
    g = {"w": rng.standard_normal(100) * 1e-3}
    z = {"w": np.zeros(100)}
    q, m, v = mlp.adam_step(p, g, z, z, 1, lr=1e-3)
    assert np.allclose(q["w"] - p["w"], -1e-3 * g["w"] / (np.abs(g["w"]) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m["w"], 0.1 * g["w"]) and np.allclose(v["w"], 0.001 * g["w"] ** 2)


def test_bf16_rounding():
    one = 1.0
    # bf16 has 8 significand bits: spacing 2^-7 at 1
    assert mlp.bf16(one) == 1.0
    assert mlp.bf16(1 + 2 ** -8) == 1.0               # tie -> even (1.0)
    assert mlp.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6   # tie -> even (1 + 2^-6)
    assert mlp.bf16(1 + 2 ** -8 + 2 ** -20) == 1 + 2 ** -7
    assert mlp.bf16(-3.14159) == -3.140625
    x = np.random.default_rng(0).standard_normal(1000)
    y = mlp.bf16(x)
    assert (np.abs(y - x) <= np.abs(x) * 2 ** -8 + 1e-30).all()


def test_quantised_forward_is_close():
    p = small_params()
    B = wl.fourier_matrix()
    c = wl.survey_c(64, seed=8)
    a = mlp.forward(p, c, B)["p"]
    b = mlp.forward(p, c, B, quant=True)["p"]
    assert np.abs(a - b).sum(axis=1).max() < 0.05


def test_top_k_is_stable():
    s = np.array([0.5, 0.9, 0.9, 0.1, 0.9])
    assert list(mlp.top_k(s, 3)) == [1, 2, 4]
    assert list(mlp.top_k(s, 5)) == [1, 2, 4, 0, 3]


def test_training_reduces_loss():
    """A few Adam steps on a fixed batch lower the loss (sanity of the loop)."""
    p = small_params(scale=0.5)
    B = wl.fourier_matrix()
    c = wl.survey_c(32, seed=9)
    T = targets(32, seed=2)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(vv) for k, vv in p.items()}
    L0 = mlp.loss(p, c, B, T)
    for t in range(1, 21):
        _, g = mlp.grads(p, c, B, T)
        p, m, v = mlp.adam_step(p, g, m, v, t, lr=3e-3)
    assert mlp.loss(p, c, B, T) < 0.9 * L0
