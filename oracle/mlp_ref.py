"""FP64 CPU reference of the learned-guess MLP (forward, backward, Adam).

TEST INFRASTRUCTURE: used only by tests to check the CUDA training and inference
kernels.  Plain numpy, float64, the textbook formulas:

    h_0 = x,  z_l = h_{l-1} W_l^T + b_l,  h_l = silu(z_l) (l < L),  out = z_L
    loss = 1/(2B) sum_b sum_o (out_bo - t_bo)^2
    silu(z) = z sigmoid(z),  silu'(z) = sigmoid(z) (1 + z (1 - sigmoid(z)))

Weights W_l have shape [out, in] (row n holds the weights of output unit n).
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(params, x):
    """params: list of (W [out,in], b [out]); returns (out, cache)."""
    h = np.asarray(x, np.float64)
    cache = [(h, None)]
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        h = silu(z) if l < L - 1 else z
        cache.append((h, z))
    return h, cache


def loss_and_grads(params, x, t):
    """MSE loss 1/(2B) sum (out - t)^2 and its gradients w.r.t. every W, b."""
    out, cache = forward(params, x)
    B = x.shape[0]
    d = (out - t) / B
    loss = 0.5 * np.sum((out - t) ** 2) / B
    grads = [None] * len(params)
    L = len(params)
    for l in range(L - 1, -1, -1):
        h_prev = cache[l][0]
        z = cache[l + 1][1]
        dz = d if l == L - 1 else d * silu_grad(z)
        grads[l] = (dz.T @ h_prev, dz.sum(axis=0))
        d = dz @ params[l][0]
    return loss, grads


def adam_step(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; state: dict with 't', 'm', 'v' lists."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    if "m" not in state:
        state["m"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        state["v"] = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    new = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        out = []
        for i, (p, g) in enumerate(((W, gW), (b, gb))):
            m = state["m"][l][i] * b1 + (1 - b1) * g
            v = state["v"][l][i] * b2 + (1 - b2) * g * g
            state["m"][l] = tuple(m if j == i else state["m"][l][j] for j in range(2))
            state["v"][l] = tuple(v if j == i else state["v"][l][j] for j in range(2))
            out.append(p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps))
        new.append(tuple(out))
    return new


def bf16_round(a):
    """Round float64 values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
