"""Plain FP64 CPU oracle for the selector network (16 -> 64 -> 64 -> 4, ReLU).

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` and the selector's checking code in tests);
the library's inference and training kernels never use it and share no code with it.

The network maps per-problem features x (16) to three logits for the factor precision
(FP16 / BF16 / FP32) and one regression output, log10 of the inner PCGTLS tolerance:
    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  out = W3 h2 + b3.
Per-sample loss: cross-entropy of softmax(out[0:3]) against the class label y, plus
lambda * mask * (out[3] - t)^2. The batch loss is the mean over samples.

``fp16=True`` rounds every weight to IEEE half precision (round to nearest even) before use,
the stored precision of the network; gradients are then taken with respect to the master
weights through that rounding (the rounding is treated as the identity).

Flat parameter layout (5508 values): W1[64][16], b1[64], W2[64][64], b2[64], W3[4][64], b3[4].
Gradients are pinned by central finite differences in tests (with fp16=False).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT, N_CLS = 16, 64, 4, 3
SHAPES = [("W1", (64, 16)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (4, 64)),
          ("b3", (4,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(P: np.ndarray, fp16: bool = False) -> dict:
    P = np.asarray(P, dtype=np.float64)
    if fp16:
        P = P.astype(np.float32).astype(np.float16).astype(np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = P[o:o + k].reshape(shp)
        o += k
    return out


def forward(P, X, fp16: bool = False):
    """Outputs (nsamp x 4) and the hidden activations."""
    w = unpack(P, fp16)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    out = h2 @ w["W3"].T + w["b3"]
    return out, (h1, h2)


def loss_and_grad(P, X, y, t, mask, lam: float, fp16: bool = False):
    """Mean loss and its gradient (flat, 5508) by explicit backpropagation."""
    w = unpack(P, fp16)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    out, (h1, h2) = forward(P, X, fp16)
    z = out[:, :N_CLS]
    zm = z.max(axis=1, keepdims=True)
    e = np.exp(z - zm)
    s = e.sum(axis=1, keepdims=True)
    p = e / s
    y = np.asarray(y, dtype=np.int64)
    t = np.asarray(t, dtype=np.float64)
    mask = np.asarray(mask, dtype=np.float64)
    dt = out[:, 3] - t
    loss = (zm[:, 0] + np.log(s[:, 0]) - z[np.arange(n), y]) + lam * mask * dt * dt
    dout = np.zeros_like(out)
    dout[:, :N_CLS] = p
    dout[np.arange(n), y] -= 1.0
    dout[:, 3] = 2.0 * lam * mask * dt
    dout /= n
    g = {"W3": dout.T @ h2, "b3": dout.sum(axis=0)}
    dh2 = (dout @ w["W3"]) * (h2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ w["W2"]) * (h1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    flat = np.concatenate([g[name].ravel() for name, _ in SHAPES])
    return float(loss.mean()), flat
