"""Plain FP64 reference of the emulator network's loss and gradients.

TEST INFRASTRUCTURE ONLY (the tests are the only callers).

The network: inputs scaled to [-1, 1] by a box (in FP32, as the device scales
them), linear layers z = a W + b, SiLU a = z / (1 + exp(-z)) on hidden layers,
a linear output layer, and the loss L = mean over rows and outputs of
(y_hat - (y - mu) / sd)^2.  Backpropagation by the chain rule: dL/dy_hat =
2 (y_hat - y_s) / (rows * outputs), dz = da * SiLU'(z), dW = a_prev^T dz,
db = sum over rows of dz, da_prev = dz W^T.  The gradient with respect to the
FP32 master weight is the one with respect to the rounded weight.

Rounding (rounding=True): every operand of the three products is rounded to
bfloat16 (round to nearest even of its FP32 value) as the device's tensor
cores take them: the weights as stored, and the activations a, the output
gradient dz and the inputs of each product as they are staged; the products
and sums are then exact here (FP64), where the device accumulates in FP32.
The bias gradient is the plain FP32-valued sum of dz.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x):
    """FP32 -> nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unpack(params, widths):
    """Parameter vector -> [(W [in][out], b [out]), ...]."""
    out, off = [], 0
    for l in range(len(widths) - 1):
        i, o = widths[l], widths[l + 1]
        W = params[off:off + i * o].reshape(i, o)
        off += i * o
        b = params[off:off + o]
        off += o
        out.append((W, b))
    return out


def scale_inputs(x, lo, hi):
    """2 (x - lo) / (hi - lo) - 1 in FP32 operations, as the device scales them."""
    x, lo, hi = (np.asarray(v, dtype=np.float32) for v in (x, lo, hi))
    return (np.float32(2.0) * (x - lo) / (hi - lo) - np.float32(1.0)).astype(np.float32)


def loss_and_grad(params, widths, x, y, lo, hi, mu, sd, rounding=True):
    """FP64 loss and gradient (same layout as params); rounding=False keeps every
    operand exact (for finite-difference checks of the backpropagation)."""
    rnd = bf16_round if rounding else (lambda w: np.asarray(w, dtype=np.float64))
    params = np.asarray(params, dtype=np.float32 if rounding else np.float64)
    layers = unpack(params, widths)
    if rounding:
        a = scale_inputs(x, lo, hi).astype(np.float64)
    else:
        a = 2.0 * (np.asarray(x, np.float64) - lo) / (np.asarray(hi, np.float64) - lo) - 1.0
    acts, zs = [a], []
    for l, (W, b) in enumerate(layers):
        z = rnd(acts[-1]) @ rnd(W) + b.astype(np.float64)
        zs.append(z)
        if l + 1 < len(layers):
            acts.append(z / (1.0 + np.exp(-z)))
    ys = (np.asarray(y, np.float64) - mu) / sd
    n = ys.size
    diff = zs[-1] - ys
    loss = float((diff ** 2).sum() / n)
    d = 2.0 * diff / n
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        if l + 1 < len(layers):
            z = zs[l]
            s = 1.0 / (1.0 + np.exp(-z))
            d = d * s * (1.0 + z * (1.0 - s))
        dr = rnd(d)
        grads.append((rnd(acts[l]).T @ dr, d.sum(0)))
        d = dr @ rnd(W).T
    grads.reverse()
    return loss, np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def predict(params, widths, x, lo, hi, mu, sd):
    params = np.asarray(params, dtype=np.float32)
    a = scale_inputs(x, lo, hi).astype(np.float64)
    layers = unpack(params, widths)
    for l, (W, b) in enumerate(layers):
        z = bf16_round(a) @ bf16_round(W) + b.astype(np.float64)
        a = z / (1.0 + np.exp(-z)) if l + 1 < len(layers) else z
    return a * sd + mu
