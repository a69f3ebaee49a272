"""Pins of the oracle's Philox4x32-10 generator and Box-Muller normals (oracle/philox.py).

The generator is pinned to the known-answer values published with the Random123 library of
Salmon, Moraes, Dror & Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC'11) for
Philox4x32 with 10 rounds: an all-zero counter and key, an all-ones counter and key, and the
counter/key taken from the hexadecimal digits of pi. A wrong multiplier, Weyl constant,
word permutation or round count changes every output word of these three blocks.

The normals are pinned by what the Box-Muller transform fixes whatever the uniform source
(Box & Muller 1958): mean 0, variance 1, a Kolmogorov-Smirnov distance to the standard
normal CDF within its 1e-6-level critical value, uncorrelated neighbours (the cos / sin
pair of one counter), and the stream layout (element 2q and 2q + 1 come from counter q).
"""

import math

import numpy as np
import pytest

from oracle import philox as X

# (counter words, key words) -> output words, Philox4x32-10 known-answer values
KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF), (0xFFFFFFFF, 0xFFFFFFFF),
     (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,expect", KAT)
def test_philox_known_answers(ctr, key, expect):
    out = X.philox4x32_10(*ctr, *key)
    assert tuple(int(v) for v in out) == expect


def test_philox_vectorised_equals_scalar_calls():
    # the array form used for streams gives the same words as one call per counter
    q = np.array([0, 1, 2, 12345, 2**32 - 1], dtype=np.uint64)
    words = X.philox4x32_10(q, q + np.uint64(7), 0, 0, 11, 13)
    for i, qi in enumerate(q):
        one = X.philox4x32_10(int(qi), int(qi) + 7, 0, 0, 11, 13)
        assert all(int(words[w][i]) == int(one[w]) for w in range(4))


def test_stream_layout_counter_and_key():
    seed = 0x0123456789ABCDEF
    x0, x1 = X.uniforms(seed, 10)
    for q in range(5):
        ref = X.philox4x32_10(q, 0, 0, 0, seed & 0xFFFFFFFF, seed >> 32)
        assert int(x0[q]) == int(ref[0]) and int(x1[q]) == int(ref[1])
    # an odd count drops the last sine, keeping the prefix
    g9, g10 = X.gaussian(seed, 9), X.gaussian(seed, 10)
    assert np.array_equal(g9, g10[:9])


def _normal_cdf(x):
    return 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def test_gaussian_moments_and_ks():
    n = 1 << 20
    g = X.gaussian(210112164, n)
    assert np.all(np.isfinite(g))
    # mean and variance of N(0, 1): standard errors 1/sqrt(n) and sqrt(2/n)
    assert abs(g.mean()) < 5.0 / math.sqrt(n)
    assert abs(g.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    # fourth moment 3 (excess kurtosis 0): standard error sqrt(96/n)
    assert abs((g ** 4).mean() - 3.0) < 5.0 * math.sqrt(96.0 / n)
    # Kolmogorov-Smirnov distance on a 2^16 subsample (erf per point); critical value at
    # level 1e-6 is about 2.7 / sqrt(m)
    m = 1 << 16
    xs = np.sort(g[:m])
    F = _normal_cdf(xs)
    i = np.arange(1, m + 1)
    d = max(np.max(i / m - F), np.max(F - (i - 1) / m))
    assert d < 2.7 / math.sqrt(m), d
    # the cos / sin pair of one counter is uncorrelated, and so are consecutive counters
    assert abs(np.corrcoef(g[0::2], g[1::2])[0, 1]) < 5.0 / math.sqrt(n / 2)
    assert abs(np.corrcoef(g[0:-2:2], g[2::2])[0, 1]) < 5.0 / math.sqrt(n / 2)


def test_uniforms_are_strictly_inside_unit_interval():
    x0, x1 = X.uniforms(7, 1 << 16)
    for x in (x0, x1):
        u = (x.astype(np.float64) + 0.5) * 2.0 ** -32
        assert u.min() > 0.0 and u.max() < 1.0
        # uniform words: the top bit is set about half the time
        assert abs((x >> np.uint64(31)).mean() - 0.5) < 0.02


def test_seeds_give_independent_streams():
    a, b = X.gaussian(1, 1 << 16), X.gaussian(2, 1 << 16)
    assert abs(np.corrcoef(a, b)[0, 1]) < 5.0 / math.sqrt(1 << 16)
