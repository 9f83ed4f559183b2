"""Oracle for the learned screening surrogate (TEST INFRASTRUCTURE ONLY).

The surrogate maps a parameter C to the normalised escape-count histogram of
its Julia frame, so that many C can be screened before any is rendered (the
paper's motivation: sample the parameter space quickly and comprehensively,
Sec. 1, and use the Mandelbrot set as a roadmap for C, Sec. 3).  Network:

    phi(C) = [sin(2 pi B C), cos(2 pi B C)]        B: 32 x 2, fixed (B C in binary32)
    h1 = relu(phi W1^T + b1)                          64 -> 256
    h2 = relu(h1 W2^T + b2)                           256 -> 256
    p  = softmax(h2 W3^T + b3)                        256 -> 101
    loss = mean over rows of  -sum_b t_b log p_b      (t: target histogram)
    Adam(lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on float32 master weights

Everything here is float64 numpy.  With quant=True the operands of every
matrix product (phi, h1, h2, the weights, and the backward products' dZ,
dZ2, dZ1) are first rounded to bfloat16 (round to nearest, ties to even), which
is where the GPU path rounds; sums, biases, masks, softmax and gradients stay
in float64 (the GPU keeps them in binary32).
"""
import numpy as np

N_FREQ, HIDDEN, N_BINS = 32, 256, 101


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) through binary32, returned as
    float64.  Finite inputs only."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def features(c, B):
    """phi(C): (n, 64) = [sin(2 pi t), cos(2 pi t)] with t = C B^T; c (n, 2),
    B (32, 2).  C and B are binary32 values and the phase t_j = B_j0 cr +
    B_j1 ci is formed in binary32 (each product and the sum rounded, no fused
    multiply-add), the precision the network accumulates in; the features
    are rounded to bfloat16 next, and that rounding must be decided from the
    same t on both sides.  Sine and cosine are then evaluated in float64."""
    c32 = np.asarray(c, np.float32)
    B32 = np.asarray(B, np.float32)
    t = c32[:, None, 0] * B32[None, :, 0] + c32[:, None, 1] * B32[None, :, 1]   # binary32 throughout
    t = t.astype(np.float64)
    return np.concatenate([np.sin(2 * np.pi * t), np.cos(2 * np.pi * t)], axis=1)


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def _q(x, quant):
    return bf16(x) if quant else np.asarray(x, np.float64)


def forward(params, c, B, quant=False):
    """Returns a dict with phi, a1, h1, a2, h2, z, p (all float64)."""
    P = {k: np.asarray(v, np.float64) for k, v in params.items()}
    phi = _q(features(c, B), quant)
    a1 = phi @ _q(P["W1"], quant).T + P["b1"]
    h1 = _q(np.maximum(a1, 0.0), quant)
    a2 = h1 @ _q(P["W2"], quant).T + P["b2"]
    h2 = _q(np.maximum(a2, 0.0), quant)
    z = h2 @ _q(P["W3"], quant).T + P["b3"]
    return dict(phi=phi, a1=a1, h1=h1, a2=a2, h2=h2, z=z, p=softmax(z))


def loss(params, c, B, T, quant=False):
    f = forward(params, c, B, quant)
    return float(-(np.asarray(T, np.float64) * np.log(f["p"])).sum(axis=1).mean())


def grads(params, c, B, T, quant=False, terms=False):
    """Loss and gradients of every parameter (backpropagation, float64).
    With terms=True also returns the forward values and the backward error
    terms (dz, dz2, dz1 and their rounded forms) as a third result."""
    P = {k: np.asarray(v, np.float64) for k, v in params.items()}
    f = forward(params, c, B, quant)
    n = f["p"].shape[0]
    T = np.asarray(T, np.float64)
    L = float(-(T * np.log(f["p"])).sum(axis=1).mean())
    dz = (f["p"] - T) / n
    dzq = _q(dz, quant)
    g = {"W3": dzq.T @ f["h2"], "b3": dz.sum(axis=0)}
    dh2 = dzq @ _q(P["W3"], quant)
    dz2 = dh2 * (f["h2"] > 0)
    dz2q = _q(dz2, quant)
    g["W2"] = dz2q.T @ f["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2q @ _q(P["W2"], quant)
    dz1 = dh1 * (f["h1"] > 0)
    dz1q = _q(dz1, quant)
    g["W1"] = dz1q.T @ f["phi"]
    g["b1"] = dz1.sum(axis=0)
    if terms:
        return L, g, dict(f, dz=dz, dzq=dzq, dz2=dz2, dz2q=dz2q, dz1=dz1, dz1q=dz1q)
    return L, g


def adam_step(params, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t = 1 for the first step); returns new (params, m, v)."""
    out_p, out_m, out_v = {}, {}, {}
    for k in params:
        gk = np.asarray(g[k], np.float64)
        mk = beta1 * np.asarray(m[k], np.float64) + (1 - beta1) * gk
        vk = beta2 * np.asarray(v[k], np.float64) + (1 - beta2) * gk * gk
        mh = mk / (1 - beta1 ** t)
        vh = vk / (1 - beta2 ** t)
        out_p[k] = np.asarray(params[k], np.float64) - lr * mh / (np.sqrt(vh) + eps)
        out_m[k], out_v[k] = mk, vk
    return out_p, out_m, out_v


def entropy(p):
    """Shannon entropy (nats) of each row of a histogram."""
    p = np.asarray(p, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return -(np.where(p > 0, p * np.log(p), 0.0)).sum(axis=1)


def top_k(scores, k):
    """Indices of the k largest scores, ties broken by the smaller index
    (stable), in descending score order."""
    s = np.asarray(scores)
    order = np.lexsort((np.arange(s.size), -s.astype(np.float64)))
    return order[:k]
