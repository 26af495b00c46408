"""FP64 reference of the learned PCG warm start's network (test infrastructure only).

The network maps per-point feature channels to a predicted Backward Euler increment: four 3-D
convolutions with 3 x 3 x 3 kernels, zero padding ("same" size) and ReLU after the first three:

    h1 = relu(conv(x, W1) + b1), h2 = relu(conv(h1, W2) + b2), h3 = relu(conv(h2, W3) + b3),
    y  = conv(h3, W4) + b4,

conv(x, W)[o, k, j, i] = sum_c sum_{a,b,d in {-1,0,1}} W[o, c, a+1, b+1, d+1] x[c, k+a, j+b, i+d]
(cross-correlation; x is zero outside the array).  Arrays are (channels, n_phi, n_theta, n_r).
The loss is the mean squared error over a mask.  The paper has no network; this is the
definition the GPU kernels are checked against, written from the formulas above.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)]


def shifted(x: np.ndarray, a: int, b: int, d: int) -> np.ndarray:
    """shifted(x)[c, k, j, i] = x[c, k+a, j+b, i+d], zero outside."""
    out = np.zeros_like(x)
    C, K, J, I = x.shape
    ks = slice(max(0, -a), min(K, K - a)); kd = slice(max(0, a), min(K, K + a))
    js = slice(max(0, -b), min(J, J - b)); jd = slice(max(0, b), min(J, J + b))
    is_ = slice(max(0, -d), min(I, I - d)); id_ = slice(max(0, d), min(I, I + d))
    out[:, ks, js, is_] = x[:, kd, jd, id_]
    return out


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    Cout = W.shape[0]
    y = np.zeros((Cout,) + x.shape[1:])
    for (a, bb, d) in OFFSETS:
        xs = shifted(x, a, bb, d)
        y += np.einsum("oc,ckji->okji", W[:, :, a + 1, bb + 1, d + 1], xs)
    if b is not None:
        y += b[:, None, None, None]
    return y


def forward(params, x):
    """params = [(W1, b1), ..., (W4, b4)]; returns (y, cache)."""
    cache = [x]
    h = x
    for li, (W, b) in enumerate(params):
        z = conv(h, W, b)
        cache.append(z)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
    return h, cache


def backward(params, cache, dy):
    """Gradients of sum(dy * y) wrt every W, b and the input."""
    grads = [None] * len(params)
    g = dy
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        z = cache[li + 1]
        if li < len(params) - 1:
            g = g * (z > 0.0)
        h_in = cache[li] if li == 0 else np.maximum(cache[li], 0.0)
        dW = np.zeros_like(W)
        for (a, bb, d) in OFFSETS:
            dW[:, :, a + 1, bb + 1, d + 1] = np.einsum("okji,ckji->oc", g, shifted(h_in, a, bb, d))
        db = g.sum(axis=(1, 2, 3))
        # input gradient: transpose of the correlation
        gx = np.zeros_like(h_in)
        for (a, bb, d) in OFFSETS:
            gx += shifted(np.einsum("oc,okji->ckji", W[:, :, a + 1, bb + 1, d + 1], g), -a, -bb, -d)
        grads[li] = (dW, db)
        g = gx
    return grads, g


def mse(y: np.ndarray, target: np.ndarray, mask: np.ndarray):
    """Loss = sum(mask (y - t)^2) / sum(mask) and its gradient wrt y."""
    n = float(mask.sum())
    r = (y - target) * mask
    return float((r * r).sum() / n), 2.0 * r / n


def init_params(rng, channels=(6, 16, 16, 16, 1)):
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        bound = np.sqrt(6.0 / (cin * 27))
        params.append((rng.uniform(-bound, bound, (cout, cin, 3, 3, 3)), np.zeros(cout)))
    return params
