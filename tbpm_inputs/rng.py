"""Counter-based SplitMix64 stream used for every seeded input.

The i-th draw of stream ``seed`` is the SplitMix64 output after i+1 state
increments (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state = seed + (i+1)*0x9E3779B97F4A7C15 (mod 2^64),
then the published 64-bit finaliser. Uniforms in [0, 1) keep the top 53 bits.
Nothing here performs any step of the propagation method.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx) -> np.ndarray:
    """uint64 draws number ``idx`` (array-like of non-negative ints) of stream ``seed``."""
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (i + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, idx) -> np.ndarray:
    """float64 uniforms in [0, 1) from the top 53 bits of ``splitmix64``."""
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
