"""Float64 forward and backward of the surrogate network -- TEST INFRASTRUCTURE ONLY.

Layers 1024 -> 256 -> 256 -> 256 -> 64; hidden activation GELU in its tanh
form (Hendrycks and Gimpel 2016): gelu(z) = z (1 + tanh(u)) / 2 with
u = sqrt(2 / pi) (z + 0.044715 z^3); output linear; loss = mean over the
valid (label >= 0) entries of (y - label)^2.  Parameters are one flat vector:
per layer the weights [out][in] row-major, then the biases.  Gradients by
hand-written backpropagation in numpy; shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

SIZES = [(1024, 256), (256, 256), (256, 256), (256, 64)]


def unpack(params):
    params = np.asarray(params, np.float64)
    out, o = [], 0
    for fin, fout in SIZES:
        W = params[o:o + fin * fout].reshape(fout, fin)
        o += fin * fout
        b = params[o:o + fout]
        o += fout
        out.append((W, b))
    assert o == params.size
    return out


_C = np.sqrt(2.0 / np.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(_C * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C * (1.0 + 3.0 * 0.044715 * z * z)


def forward(params, X):
    layers = unpack(params)
    h = np.asarray(X, np.float64)
    cache = []
    for i, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if i < len(layers) - 1 else z
    return h, cache


def loss_and_grad(params, X, L):
    """Masked mean-squared error and its gradient with respect to params."""
    layers = unpack(params)
    Y, cache = forward(params, X)
    L = np.asarray(L, np.float64)
    mask = L >= 0
    cnt = max(int(mask.sum()), 1)
    d = np.where(mask, Y - L, 0.0)
    loss = float((d * d).sum() / cnt)
    g = 2.0 * d / cnt  # dLoss / dY
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        W, b = layers[i]
        h_in, z = cache[i]
        if i < len(layers) - 1:
            g = g * gelu_grad(z)  # through the GELU of layer i
        grads.append((g.T @ h_in, g.sum(axis=0)))
        g = g @ W
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.ravel())
        flat.append(gb)
    return loss, np.concatenate(flat)


def bf16(x):
    """Round to bfloat16 (round to nearest, ties to even) through float32, as
    a float32 value stored in bfloat16 is; returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def loss_and_grad_bf16(params, X, L):
    """The same masked MSE and gradient with the network's storage in
    bfloat16, as the network is specified (BF16 weights, FP32
    accumulation): weights, each layer's pre-activation kept for the backward
    pass and its activation, the output gradient and each back-propagated
    gradient are rounded to bfloat16 where they are stored; every sum is
    exact (float64).  Also returns, per parameter, the sum of the magnitudes
    of the products the gradient adds up (sum_r |g_r| |h_r|, and sum_r |g_r|
    for a bias), the scale of the rounding error any summation order of
    those products can make."""
    layers = [(bf16(W), b) for W, b in unpack(params)]
    h = np.asarray(X, np.float64)
    cache = []
    for i, (W, b) in enumerate(layers):
        z = h @ W.T + b
        if i < len(layers) - 1:
            cache.append((h, bf16(z)))
            h = bf16(gelu(z))
        else:
            cache.append((h, None))
            h = z
    Y = h
    L = np.asarray(L, np.float64)
    mask = L >= 0
    cnt = max(int(mask.sum()), 1)
    d = np.where(mask, Y - L, 0.0)
    loss = float((d * d).sum() / cnt)
    g = bf16(2.0 * d / cnt)  # dLoss / dY as stored
    grads, scales = [], []
    for i in range(len(layers) - 1, -1, -1):
        W, b = layers[i]
        h_in, _ = cache[i]
        grads.append((g.T @ h_in, g.sum(axis=0)))
        scales.append((np.abs(g).T @ np.abs(h_in), np.abs(g).sum(axis=0)))
        if i == 0:
            break
        g = bf16((g @ W) * gelu_grad(cache[i - 1][1]))  # through the GELU of layer i - 1, stored
    flat, sflat = [], []
    for (gW, gb), (sW, sb) in zip(reversed(grads), reversed(scales)):
        flat += [gW.ravel(), gb]
        sflat += [sW.ravel(), sb]
    return loss, np.concatenate(flat), np.concatenate(sflat)
