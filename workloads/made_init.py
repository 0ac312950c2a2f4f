"""Seeded initial parameters of the MADE proposal network (input generator).

He-uniform weights W ~ U(-sqrt(6/fan_in), sqrt(6/fan_in)), zero biases, packed in
the order W1[h,n], b1[h], W2[h,h], b2[h], W3[h,h], b3[h], W4[n,h], b4[n].
"""
from __future__ import annotations

import numpy as np


def made_init(n: int, h: int = 256, seed: int = 7) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for (o, i) in ((h, n), (h, h), (h, h), (n, h)):
        lim = np.sqrt(6.0 / i)
        parts.append(rng.uniform(-lim, lim, size=(o, i)).ravel())
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def epoch_orders(n_data: int, epochs: int, seed: int = 7):
    """Data permutation of every training epoch."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    return [rng.permutation(n_data).astype(np.int32) for _ in range(epochs)]
