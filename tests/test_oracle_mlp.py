"""Pins for the surrogate oracle (oracle/mlp.py): gradients against finite
differences, Adam's first step in closed form, softmax / feature identities,
and bfloat16 rounding on hand-worked values."""
import math

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
    # (dyadic C, so every binary32 phase is exact)
    Bi = np.array([[1.0, 0.0], [2.0, 3.0]])
    a = mlp.features(np.array([[0.125, 0.375]]), Bi)
    b = mlp.features(np.array([[1.125, 0.375]]), Bi)
    assert np.allclose(a[:, [0, 2]], b[:, [0, 2]], atol=1e-12)
    check_features_binary32_phase()


def check_features_binary32_phase(m=mlp):
    """The phase is rounded to binary32: C = (0.1, 0.3) and B row (3, 7) give
    t = fl(fl(3 * 0.1f) + fl(7 * 0.3f)) = 2.4000000953674316, not 2.4."""
    t32 = np.float32(np.float32(3) * np.float32(0.1)) + np.float32(np.float32(7) * np.float32(0.3))
    assert float(t32) == 2.4000000953674316
    f = m.features(np.array([[0.1, 0.3]]), np.array([[3.0, 7.0]]))
    assert f[0, 0] == math.sin(2 * math.pi * float(t32)) and f[0, 1] == math.cos(2 * math.pi * float(t32))


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


# ---------------------------------------------------------------------------
# A hand-worked network.  Every weight, bias and feature below is a small
# dyadic number (exact in bfloat16), so the features, pre-activations, hidden
# activations and logits are known exactly and written out here by hand; the
# oracle must reproduce them.  C = (1/4, 1/2) and B rows [1,0], [0,1], [1,1]
# put 2 pi B C at pi/2, pi and 3 pi/2, where sine and cosine are 0 or +-1.
# ---------------------------------------------------------------------------
HAND_C = np.array([[0.25, 0.5]])


def hand_network():
    B = np.zeros((32, 2))
    B[0] = [1, 0]
    B[1] = [0, 1]
    B[2] = [1, 1]
    W1, b1 = np.zeros((256, 64)), np.zeros(256)
    W1[0, 0], b1[0] = 1.0, 0.25          # sin(pi/2) = 1        -> a1 = 1.25
    W1[1, 33], b1[1] = 1.0, 0.5          # cos(pi) = -1         -> a1 = -0.5
    W1[2, 35] = 0.5                      # cos(0) = 1           -> a1 = 0.5
    b1[3] = -2.0                         #                         a1 = -2
    W1[4, 2] = -3.0                      # sin(3 pi/2) = -1     -> a1 = 3
    W1[5, 2], b1[5] = 1.0, 0.75          #                         a1 = -0.25
    W2, b2 = np.zeros((256, 256)), np.zeros(256)
    W2[0, 0], W2[0, 1] = 1.0, 1.0        # a2 = 1.25 + h1[1]
    W2[1, 2], W2[1, 3] = 2.0, 1.0        # a2 = 2 * 0.5 + h1[3]
    W2[2, 4], b2[2] = -1.0, 1.0          # a2 = -3 + 1
    W2[3, 4], b2[3] = 1.0, -1.0          # a2 = 3 - 1
    W2[4, 5], b2[4] = 4.0, 0.5           # a2 = 4 h1[5] + 0.5
    W3, b3 = np.zeros((101, 256)), np.zeros(101)
    W3[0, 0], b3[0] = 1.0, -0.25         # z = 1.25 - 0.25
    W3[1, 1], W3[1, 3] = 1.0, 0.5        # z = 1 + 0.5 * 2
    W3[2, 2] = 5.0                       # z = 5 h2[2]
    b3[3] = -1.0                         # z = -1
    W3[4, 4] = -2.0                      # z = -2 * 0.5
    W3[100, 3] = 0.25                    # z = 0.25 * 2
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3), B


# the values worked out by hand (indices not listed are 0)
HAND_A1 = {0: 1.25, 1: -0.5, 2: 0.5, 3: -2.0, 4: 3.0, 5: -0.25}
HAND_H1 = {0: 1.25, 2: 0.5, 4: 3.0}
HAND_A2 = {0: 1.25, 1: 1.0, 2: -2.0, 3: 2.0, 4: 0.5}
HAND_H2 = {0: 1.25, 1: 1.0, 3: 2.0, 4: 0.5}
HAND_Z = {0: 1.0, 1: 2.0, 3: -1.0, 4: -1.0, 100: 0.5}


def dense(d, n):
    v = np.zeros(n)
    for k, x in d.items():
        v[k] = x
    return v


def hand_probs():
    """softmax of the hand logits: 96 bins at e^0, the others listed."""
    S = math.e + math.e ** 2 + 96 + 2 / math.e + math.sqrt(math.e)
    return np.array([math.exp(HAND_Z.get(b, 0.0)) / S for b in range(101)])


def check_hand_forward(m=mlp):
    P, B = hand_network()
    for quant in (False, True):
        f = m.forward(P, HAND_C, B, quant=quant)
        phi = f["phi"][0]
        assert phi[0] == 1.0 and phi[2] == -1.0 and phi[33] == -1.0, quant
        assert (phi[3:32] == 0).all() and (phi[35:] == 1).all(), quant
        assert max(abs(phi[1]), abs(phi[32]), abs(phi[34])) < 1e-15, quant
        assert (f["a1"][0] == dense(HAND_A1, 256)).all(), quant
        assert (f["h1"][0] == dense(HAND_H1, 256)).all(), quant
        assert (f["a2"][0] == dense(HAND_A2, 256)).all(), quant
        assert (f["h2"][0] == dense(HAND_H2, 256)).all(), quant
        assert (f["z"][0] == dense(HAND_Z, 101)).all(), quant
        assert np.abs(f["p"][0] - hand_probs()).max() < 1e-16, quant


def test_hand_worked_forward():
    """Features, pre-activations, ReLU outputs, logits and softmax of the
    hand-worked network, with and without bfloat16 operands (every operand
    is on the bfloat16 grid, so both modes give the same values)."""
    check_hand_forward()


def test_zero_network_one_hot_bias():
    """All weights zero and b3 = t e_k: p_k = e^t / (e^t + 100), every other
    bin 1 / (e^t + 100), whatever C is."""
    P, B = hand_network()
    P = {k: np.zeros_like(v) for k, v in P.items()}
    P["b3"][17] = 3.0
    p = mlp.forward(P, wl.survey_c(5, seed=1), wl.fourier_matrix())["p"]
    d = math.exp(3.0) + 100
    assert np.abs(p[:, 17] - math.exp(3.0) / d).max() < 1e-15
    assert np.abs(np.delete(p, 17, axis=1) - 1 / d).max() < 1e-15


def hand_grads_expected(T, quant, n):
    """Backpropagation through the hand-worked network, written out by its
    sparsity pattern.  q() marks the operands the bfloat16 path rounds: the
    logit error dz, the masked hidden errors dz2, dz1 and the features."""
    q = mlp.bf16 if quant else (lambda x: np.asarray(x, np.float64))
    p = hand_probs()
    h1, h2 = dense(HAND_H1, 256), dense(HAND_H2, 256)
    # features by hand: sin at pi/2, pi, 3 pi/2 then 29 zeros; cos at the same angles then 29 ones
    phi = np.array([1.0, math.sin(math.pi), -1.0] + [0.0] * 29 +
                   [math.cos(math.pi / 2), -1.0, math.cos(3 * math.pi / 2)] + [1.0] * 29)
    g = {"W1": np.zeros((256, 64)), "b1": np.zeros(256), "W2": np.zeros((256, 256)), "b2": np.zeros(256),
         "W3": np.zeros((101, 256)), "b3": np.zeros(101)}
    for r in range(n):
        d = (p - T[r]) / n                       # dL/dz of row r
        e = q(d)
        g["b3"] += d
        g["W3"] += np.outer(e, h2)
        # dh2_j = sum_b e_b W3[b, j], masked where h2 = 0 (j = 2)
        dz2 = np.zeros(256)
        dz2[0] = e[0]
        dz2[1] = e[1]
        dz2[3] = 0.5 * e[1] + 0.25 * e[100]
        dz2[4] = -2.0 * e[4]
        f = q(dz2)
        g["b2"] += dz2
        g["W2"] += np.outer(f, h1)
        # dh1_k = sum_i f_i W2[i, k], masked where h1 = 0 (k = 1, 3, 5)
        dz1 = np.zeros(256)
        dz1[0] = f[0]
        dz1[2] = 2.0 * f[1]
        dz1[4] = f[3] - f[2]
        g["b1"] += dz1
        g["W1"] += np.outer(q(dz1), q(phi))
    L = -np.mean([(T[r] * np.log(p)).sum() for r in range(n)])
    return L, g


def hand_targets():
    T = np.zeros((2, 101))
    T[0, 1], T[0, 0], T[0, 100] = 0.5, 0.25, 0.25
    T[1, 4], T[1, 3], T[1, 50] = 0.625, 0.125, 0.25
    return T


def check_hand_grads(m=mlp):
    P, B = hand_network()
    T = hand_targets()
    c = np.repeat(HAND_C, 2, axis=0)
    for quant in (False, True):
        L, g = m.grads(P, c, B, T, quant=quant)
        Le, ge = hand_grads_expected(T, quant, 2)
        assert abs(L - Le) < 1e-14, quant
        for k in ge:
            assert np.abs(g[k] - ge[k]).max() <= 1e-15 * max(1.0, np.abs(ge[k]).max()), (k, quant)
    # bfloat16 rounding of the error terms really changes the products here
    _, g0 = m.grads(P, c, B, T, quant=False)
    _, g1 = m.grads(P, c, B, T, quant=True)
    assert np.abs(g0["W3"] - g1["W3"]).max() > 1e-6 and np.abs(g0["W1"] - g1["W1"]).max() > 1e-6
    assert (g0["b3"] == g1["b3"]).all()          # bias gradients are not rounded


def test_hand_worked_gradients():
    """Loss and every gradient of the hand-worked network, two rows, with and
    without the bfloat16 rounding points (dz, dz2, dz1 rounded before their
    products; bias gradients from the unrounded errors)."""
    check_hand_grads()


def check_adam_constant_gradient(m=mlp):
    """With the same gradient at every step the bias corrections cancel
    exactly: m_hat = g and v_hat = g^2 at every t, so every step moves each
    parameter by -lr g / (|g| + eps)."""
    rng = np.random.default_rng(1)
    g = {"w": rng.standard_normal(50) * 1e-2}
    p = {"w": rng.standard_normal(50)}
    mm = {"w": np.zeros(50)}
    vv = {"w": np.zeros(50)}
    step = -1e-3 * g["w"] / (np.abs(g["w"]) + 1e-8)
    for t in range(1, 8):
        q, mm, vv = m.adam_step(p, g, mm, vv, t)
        assert np.allclose(q["w"] - p["w"], step, rtol=1e-9, atol=0), t
        p = q


def test_adam_constant_gradient():
    check_adam_constant_gradient()


def test_softmax_entropy_topk_against_library():
    """softmax against scipy.special.softmax, entropy against
    scipy.stats.entropy, top-k against a full stable sort."""
    import scipy.special
    import scipy.stats
    rng = np.random.default_rng(5)
    z = rng.standard_normal((40, 101)) * 4
    assert np.abs(mlp.softmax(z) - scipy.special.softmax(z, axis=1)).max() < 1e-15
    p = scipy.special.softmax(z, axis=1)
    p[3, :50] = 0
    p[3] /= p[3].sum()
    assert np.abs(mlp.entropy(p) - scipy.stats.entropy(p, axis=1)).max() < 1e-13
    s = rng.integers(0, 20, 500).astype(np.float32)
    ref = sorted(range(500), key=lambda i: (-float(s[i]), i))
    assert list(mlp.top_k(s, 500)) == ref
