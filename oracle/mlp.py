"""Plain FP64 reference of the surrogate MLP — TEST INFRASTRUCTURE ONLY.

Network: x -> h1 = GELU(W1 x + b1) -> h2 = GELU(W2 h1 + b2) -> h3 = GELU(W3 h2 + b3)
-> y = W4 h3 + b4, with GELU(t) = t * Phi(t) (Phi the standard normal CDF).
The products use the weights rounded to bfloat16 (round to nearest even), as
the model is defined; activations and accumulation are FP64 here.  Backward is
the chain rule written out; Adam is the bias-corrected update of Kingma & Ba.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def bf16_round(w: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    u = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(t):
    return 0.5 * t * (1.0 + erf(t / np.sqrt(2.0)))


def gelu_grad(t):
    return 0.5 * (1.0 + erf(t / np.sqrt(2.0))) + t * np.exp(-0.5 * t * t) / np.sqrt(2.0 * np.pi)


def forward(weights, biases, X):
    """Returns (y, cache); weights[l] has shape [out, in] (FP32 master values)."""
    a = np.asarray(X, dtype=np.float64)
    cache = []
    L = len(weights)
    for l in range(L):
        Wb = bf16_round(weights[l])
        p = a @ Wb.T + np.asarray(biases[l], dtype=np.float64)
        cache.append((a, p))
        a = gelu(p) if l < L - 1 else p
    return a, cache


def backward(weights, cache, dY):
    """Gradients of sum(dY * y) with respect to the weights and biases."""
    L = len(weights)
    g = np.asarray(dY, dtype=np.float64)
    gw, gb = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        a, p = cache[l]
        if l < L - 1:
            g = g * gelu_grad(p)
        gw[l] = g.T @ a
        gb[l] = g.sum(axis=0)
        g = g @ bf16_round(weights[l])
    return gw, gb


def mse(y, t):
    """Loss mean((y - t)^2) and its gradient 2 (y - t) / y.size."""
    d = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(w, g, m, v, lr, b1, b2, eps, step):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    w = w - lr * (m / (1 - b1**step)) / (np.sqrt(v / (1 - b2**step)) + eps)
    return w, m, v
