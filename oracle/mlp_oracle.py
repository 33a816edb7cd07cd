"""FP64 reference of the T5 scoring network (test infrastructure only).

Only tests/ and the benchmark's CPU-baseline leg use this module; it never
imports the device package.

Network (an optional learned T5 selection; the paper itself uses hand-set
cuts, Section 2.1): 48 inputs (38 features, zero padded) ->
64 -> 64 -> 32 -> 1, ReLU on the hidden layers, sigmoid on the output. The
device evaluates it with BF16 weights and BF16 layer inputs, accumulating in
FP32; this reference applies the same BF16 rounding (round to nearest even)
to the weights and to every layer input and accumulates in FP64, so the two
agree to FP32 accumulation error. Loss: mean binary cross-entropy.

Parameter vector layout (FP32 master copy, 9409 values):
  W1[64][48], b1[64], W2[64][64], b2[64], W3[32][64], b3[32], W4[32], b4[1]
(W[o][i] multiplies input i into output o).
"""
from __future__ import annotations

import numpy as np

N_IN, H1, H2, H3 = 48, 64, 64, 32
SHAPES = [("W1", (H1, N_IN)), ("b1", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)), ("W3", (H3, H2)), ("b3", (H3,)),
          ("W4", (H3,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even); returns float64."""
    a = np.asarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))
    r = ((u + bias) & np.uint64(0xFFFF0000)).astype(np.uint32)
    nan = np.isnan(a)
    r = np.where(nan, np.uint32(0x7FC00000), r)
    return r.view(np.float32).astype(np.float64)


def forward(theta, X, rounding=True):
    """Scores (sigmoid outputs) and the activations the gradient needs.

    rounding=False gives the same network in plain FP64 (for finite differences).
    """
    p = unpack(theta)
    r = bf16 if rounding else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3 = r(p["W1"]), r(p["W2"]), r(p["W3"])
    x0 = r(np.asarray(X, np.float32) if rounding else np.asarray(X, np.float64))
    z1 = x0 @ W1.T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    x1 = r(h1.astype(np.float32)) if rounding else h1
    z2 = x1 @ W2.T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    x2 = r(h2.astype(np.float32)) if rounding else h2
    z3 = x2 @ W3.T + p["b3"]
    h3 = np.maximum(z3, 0.0)
    z4 = h3 @ p["W4"] + p["b4"][0]
    s = 1.0 / (1.0 + np.exp(-z4))
    return s, dict(x0=x0, z1=z1, x1=x1, z2=z2, x2=x2, z3=z3, h3=h3, z4=z4, W1=W1, W2=W2, W3=W3, W4=p["W4"])


def loss(theta, X, y, rounding=True):
    s, c = forward(theta, X, rounding)
    z = c["z4"]
    y = np.asarray(y, np.float64)
    # mean BCE from the logit: log(1 + e^z) - y z, written stably
    return float(np.mean(np.maximum(z, 0) - y * z + np.log1p(np.exp(-np.abs(z)))))


def grad(theta, X, y, rounding=True):
    """Gradient of the mean BCE with respect to the parameter vector.

    The chain rule runs through the BF16-rounded weights (the device multiplies
    with them); rounding of activations is treated as the identity for the
    derivative (straight-through), as on the device.
    """
    s, c = forward(theta, X, rounding)
    y = np.asarray(y, np.float64)
    B = len(y)
    dz4 = (s - y) / B
    g = {}
    g["W4"] = c["h3"].T @ dz4
    g["b4"] = np.array([dz4.sum()])
    dz3 = np.outer(dz4, c["W4"]) * (c["z3"] > 0)
    g["W3"] = dz3.T @ c["x2"]
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ c["W3"]) * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["x1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ c["W2"]) * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["x0"]
    g["b1"] = dz1.sum(0)
    return pack(g)


def adam(theta, m, v, gr, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); returns new (theta, m, v). step counts from 1."""
    m = b1 * m + (1 - b1) * gr
    v = b2 * v + (1 - b2) * gr * gr
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
