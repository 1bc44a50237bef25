"""CPU oracle of the surrogate MLP's forward and backward pass.

TEST INFRASTRUCTURE ONLY.  Plain numpy in FP64.  With ``bf16=True`` it rounds,
to the nearest BF16 (ties to even), exactly the values the GPU path stores in
BF16: the inputs, the weights, every hidden activation a_l = gelu(z_l), and the
output-side gradients dz_l before they enter the weight- and input-gradient
products.  Pre-activations, the output, the loss, the bias gradients and the
accumulation of every product stay in high precision.
    z_l = a_{l-1} W_l + b_l,  a_l = gelu(z_l)   (hidden layers)
    y_hat = z_L,  loss = mean((y_hat - y)^2)
    dz_L = 2 (y_hat - y) / numel,  dW_l = a_{l-1}^T dz_l,  db_l = sum_rows dz_l
    dz_{l-1} = (dz_l W_l^T) * gelu'(z_{l-1})
The activation is GELU in its tanh form (Hendrycks and Gimpel, 2016, Sec. 2):
    gelu(z) = z/2 (1 + tanh(u)),  u = sqrt(2/pi) (z + 0.044715 z^3)
    gelu'(z) = (1 + tanh(u))/2 + z/2 (1 - tanh(u)^2) sqrt(2/pi) (1 + 3 * 0.044715 z^2)
(the surrogate is not in the paper; its activation is this design's choice).
"""
from __future__ import annotations

import math

import numpy as np

_C1 = math.sqrt(2.0 / math.pi)
_A = 0.044715


def bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even) and return it as FP64."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64).reshape(f.shape)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C1 * (z + _A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(_C1 * (z + _A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C1 * (1.0 + 3.0 * _A * z * z)


def unpack(params: np.ndarray, sizes):
    """Flat FP32 layout: for each layer W [fan_in x fan_out] row-major, then b."""
    out, off = [], 0
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        W = params[off:off + fi * fo].reshape(fi, fo)
        off += fi * fo
        b = params[off:off + fo]
        off += fo
        out.append((np.asarray(W, np.float64), np.asarray(b, np.float64)))
    assert off == params.size
    return out


def forward(params, sizes, x, bf16_round=True):
    r = bf16 if bf16_round else (lambda v: np.asarray(v, np.float64))
    layers = unpack(np.asarray(params), sizes)
    a = r(x)
    acts, zs = [a], []
    for l, (W, b) in enumerate(layers):
        z = a @ r(W) + b
        if l < len(layers) - 1:
            zs.append(z)
            a = r(gelu(z))
            acts.append(a)
        else:
            return z, acts, zs


def loss_and_grad(params, sizes, x, y, bf16_round=True):
    r = bf16 if bf16_round else (lambda v: np.asarray(v, np.float64))
    layers = unpack(np.asarray(params), sizes)
    yhat, acts, zs = forward(params, sizes, x, bf16_round)
    d = yhat - y
    loss = float(np.mean(d * d))
    dz = 2.0 * d / d.size
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        dzr = r(dz)
        gW = acts[l].T @ dzr
        gb = dz.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            dz = (dzr @ r(W).T) * gelu_grad(zs[l - 1])
    flat = np.concatenate([np.concatenate([g[0].reshape(-1), g[1]]) for g in grads])
    return loss, flat, yhat


def init_params(sizes, seed=0) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (FP32)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        lim = 1.0 / math.sqrt(fi)
        parts += [rng.uniform(-lim, lim, fi * fo), np.zeros(fo)]
    return np.concatenate(parts).astype(np.float32)
