"""Seed derivation: one master seed, SplitMix64 substreams per (config, index, purpose).

SplitMix64 is the 64-bit mixing generator of Steele, Lea & Flood (OOPSLA 2014):
state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds and a final xor-shift.
Each substream seed feeds a numpy PCG64 generator.
"""

import numpy as np

MASTER_SEED = 210112164

_MASK = (1 << 64) - 1

# purposes of random draws
PURPOSE = {"field": 1, "xstar": 2, "sketch": 3, "net_init": 4, "draw": 5, "train": 6,
           "probe": 7, "sample": 8}


def _splitmix64(state):
    state = (state + 0x9E3779B97F4A7C15) & _MASK
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return state, z ^ (z >> 31)


def substream_seed(config: int, index: int, purpose: str, master: int = MASTER_SEED) -> int:
    """64-bit seed for the stream (config, index, purpose) derived from ``master``."""
    s = master & _MASK
    out = 0
    for word in (config, index, PURPOSE[purpose]):
        s, z = _splitmix64(s ^ (word & _MASK))
        out ^= z
        s = z
    return out


def rng_for(config: int, index: int, purpose: str, master: int = MASTER_SEED):
    return np.random.Generator(np.random.PCG64(substream_seed(config, index, purpose, master)))
