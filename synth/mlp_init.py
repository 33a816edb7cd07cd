"""Seeded initial parameters of the T5 scoring network (input producer).

He-normal weights (standard deviation sqrt(2 / fan_in)), zero biases, drawn
with numpy's PCG64; laid out as W1[64][48], b1[64], W2[64][64], b2[64],
W3[32][64], b3[32], W4[32], b4 (9409 float32 values).
"""
import numpy as np

SHAPES = [((64, 48), True), ((64,), False), ((64, 64), True), ((64,), False), ((32, 64), True), ((32,), False),
          ((32,), True), ((1,), False)]


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for shape, is_w in SHAPES:
        if is_w:
            fan_in = shape[-1] if len(shape) == 2 else shape[0]
            parts.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), shape).ravel())
        else:
            parts.append(np.zeros(shape).ravel())
    return np.concatenate(parts).astype(np.float32)
