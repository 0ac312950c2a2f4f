"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).  Written from the published
definition: a 4x32-bit counter and a 2x32-bit key; ten rounds, each multiplying
counter words 0 and 2 by the round constants, XOR-mixing the high halves with
the key and the other counter words, then bumping the key by the Weyl
constants.  The paper does not fix an RNG; this library uses Philox for every
random number the method draws (sample draws and range-finder test matrices),
keyed so that results are reproducible on any device.

Vectorised over numpy uint64 arrays holding 32-bit values.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words (as uint64 arrays) for counters/keys."""
    c0, c1, c2, c3, k0, k1 = (np.asarray(x, dtype=np.uint64) & MASK for x in (c0, c1, c2, c3, k0, k1))
    for rnd in range(10):
        p0 = M0 * c0               # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
        if rnd < 9:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
    return c0, c1, c2, c3


def u53(hi, lo):
    """Uniform double in [0, 1) from the upper 53 bits of the 64-bit word hi:lo."""
    x = ((np.asarray(hi, dtype=np.uint64) << np.uint64(32)) | np.asarray(lo, dtype=np.uint64)) >> np.uint64(11)
    return x.astype(np.float64) * (2.0 ** -53)


def split_seed(seed: int) -> tuple[int, int]:
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def draw_uniforms(seed: int, sample_ids, site_ids):
    """Uniform used to draw qubit ``site`` of sample ``sample``.

    counter = (sample lo, sample hi, site, 0), key = seed; u from output words 0,1.
    """
    k0, k1 = split_seed(seed)
    s = np.asarray(sample_ids, dtype=np.uint64)
    v = np.asarray(site_ids, dtype=np.uint64)
    s, v = np.broadcast_arrays(s, v)
    w0, w1, _, _ = philox4x32_10(s & MASK, s >> np.uint64(32), v, np.zeros_like(v), k0, k1)
    return u53(w0, w1)


STAGE_SAMPLE, STAGE_ENV_KET, STAGE_ENV_BRA, STAGE_AMPLITUDE = 0, 1, 2, 3


def test_matrix(seed: int, stage: int, row: int, site: int, n: int, k: int) -> np.ndarray:
    """Complex n x k range-finder test matrix, entries with Re, Im uniform in [-1, 1).

    counter = (i, j, row * 4096 + site, 0x80000000 | stage), key = seed; Re from
    output words 0,1 and Im from words 2,3.  Shared by every sample.
    """
    k0, k1 = split_seed(seed)
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(k, dtype=np.uint64)[None, :]
    i, j = np.broadcast_arrays(i, j)
    c2 = np.full(i.shape, row * 4096 + site, dtype=np.uint64)
    c3 = np.full(i.shape, 0x80000000 | stage, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32_10(i, j, c2, c3, k0, k1)
    return (2.0 * u53(w0, w1) - 1.0) + 1j * (2.0 * u53(w2, w3) - 1.0)
