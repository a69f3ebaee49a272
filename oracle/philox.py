"""Philox4x32-10 counter-based generator and Box-Muller normals (test infrastructure).

Written from the definition in Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
easy as 1, 2, 3" (SC'11): a 4 x 32-bit counter and a 2 x 32-bit key; each of 10 rounds
multiplies counter words 0 and 2 by 0xD2511F53 and 0xCD9E8D57 (64-bit products split into
high and low halves), then the new counter is (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
the key is bumped by (0x9E3779B9, 0xBB67AE85) between rounds.

Element i of a stream: counter (i // 2 low word, high word, 0, 0), key = (seed low, high);
u1 = (x0 + 1/2) 2^-32, u2 = (x1 + 1/2) 2^-32, radius sqrt(-2 ln u1), angle 2 pi u2;
even i -> radius * cos, odd i -> radius * sin.
"""

import numpy as np

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) for c in (c0, c1, c2, c3))
    k0, k1 = int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0)), lo1, (hi0 ^ c3 ^ np.uint64(k1)), lo0
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def uniforms(seed, count):
    q = np.arange((count + 1) // 2, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(q & MASK, q >> np.uint64(32), 0, 0, seed & 0xFFFFFFFF,
                                 (seed >> 32) & 0xFFFFFFFF)
    return x0, x1


def gaussian(seed, count):
    x0, x1 = uniforms(seed, count)
    u1 = (x0.astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (x1.astype(np.float64) + 0.5) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    out = np.empty(2 * len(x0))
    out[0::2] = rad * np.cos(ang)
    out[1::2] = rad * np.sin(ang)
    return out[:count]
