"""FP64 reference of the warm-start network (oracle; test infrastructure).

A multilayer perceptron maps a member's parameter theta to a prediction of
its scaled solution state: layers d_in -> h -> ... -> h -> d_out, GELU after
every hidden layer, a linear output layer.  Loss: mean squared error over the
(unmasked) outputs of a batch.  Optimiser: Adam.  The GPU's BF16 kernels are
compared with this module's gradients on the same (BF16-rounded) inputs.

Conventions: a layer holds W (out x in) and b (out); for a batch X
(rows = samples) the layer computes Z = X W^T + b.  GELU(z) = z Phi(z) with
Phi the standard normal distribution function, GELU'(z) = Phi(z) + z phi(z).

``bf16_points=True`` rounds to BF16 where a BF16 network stores values that
feed a product: each hidden activation GELU(Z), and each layer's dZ before
the products dW = dZ^T A and dA = dZ W (the bias gradient sums the unrounded
dZ).  Inputs and weights are rounded by the caller (``bf16_round``).  Every
other step stays in FP64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def init_params(rng, sizes):
    """[(W, b), ...] with W ~ N(0, 1/fan_in), b = 0 (float64)."""
    out = []
    for fin, fout in zip(sizes[:-1], sizes[1:]):
        out.append((rng.standard_normal((fout, fin)) / math.sqrt(fin), np.zeros(fout)))
    return out


def forward(params, X, bf16_points=False):
    """Returns (output, cache) with cache = [(input, Z), ...] per layer."""
    cache = []
    A = np.asarray(X, dtype=np.float64)
    for li, (W, b) in enumerate(params):
        Z = A @ W.T + b
        cache.append((A, Z))
        if li < len(params) - 1:
            A = gelu(Z)
            if bf16_points:
                A = bf16_round(A)
        else:
            A = Z
    return A, cache


def loss_and_grads(params, X, T, mask=None, bf16_points=False):
    """MSE = mean over samples and unmasked outputs of (Y - T)^2, and its
    gradients [(dW, db), ...] by the chain rule through every layer."""
    Y, cache = forward(params, X, bf16_points)
    M = np.ones(Y.shape[1]) if mask is None else np.asarray(mask, dtype=np.float64)
    cnt = Y.shape[0] * M.sum()
    R = (Y - T) * M
    loss = float(np.sum(R * R) / cnt)
    dA = 2.0 * R / cnt
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        A_in, Z = cache[li]
        dZ = dA if li == len(params) - 1 else dA * gelu_grad(Z)
        W, _ = params[li]
        dZp = bf16_round(dZ) if bf16_points else dZ
        grads[li] = (dZp.T @ A_in, dZ.sum(axis=0))
        dA = dZp @ W
    return loss, grads


def adam(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step with bias correction; ``state`` (a dict, empty at the
    start) keeps the step count and the first and second moment estimates."""
    if not state:
        state["t"] = 0
        state["m"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        state["v"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    state["t"] += 1
    t = state["t"]
    new = []
    for li, (layer, grad) in enumerate(zip(params, grads)):
        pair = []
        for k in range(2):
            g = grad[k]
            m = beta1 * state["m"][li][k] + (1.0 - beta1) * g
            v = beta2 * state["v"][li][k] + (1.0 - beta2) * g * g
            state["m"][li][k], state["v"][li][k] = m, v
            mh = m / (1.0 - beta1 ** t)
            vh = v / (1.0 - beta2 ** t)
            pair.append(layer[k] - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(pair))
    return new


def bf16_round(a):
    """Round float values to bfloat16 (round to nearest even), returned as
    float64: the GPU kernels read inputs and weights in this precision."""
    a32 = np.asarray(a, dtype=np.float32)
    bits = a32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)
