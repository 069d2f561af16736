"""Counter-based Gaussian start block (test infrastructure only).

The paper draws Pi ~ N(0,1)^{d x k} (Algorithms 1 and 2, step 1) but names no
generator.  The GPU library and this oracle each implement the same one from its
published definition, so a seed alone fixes Pi on both sides:

* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output i of the stream seeded
  with s is mix(s + (i + 1) * 0x9E3779B97F4A7C15 mod 2^64), where mix is the
  variant-13 finaliser: z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
  z *= 0x94D049BB133111EB; z ^= z >> 31.
* Box-Muller (1958): u1 = ((x1 >> 11) + 1) 2^-53 in (0, 1], u2 = (x2 >> 11) 2^-53
  in [0, 1); r = sqrt(-2 ln u1), theta = 2 pi u2; the pair gives r cos(theta) and
  r sin(theta).

Element (j, c) of the row-major d x k block has index e = j k + c; pair p = e // 2
uses outputs 2p and 2p + 1; even e takes the cosine, odd e the sine.  The value
is computed in FP64 and rounded once to FP32.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, i: int) -> int:
    """Output i (0-based) of the SplitMix64 stream seeded with ``seed``."""
    z = (seed + (i + 1) * GAMMA) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def gaussian_pair(seed: int, p: int):
    """The two FP64 normals of pair p."""
    x1 = splitmix64(seed, 2 * p)
    x2 = splitmix64(seed, 2 * p + 1)
    u1 = ((x1 >> 11) + 1) * (2.0 ** -53)
    u2 = (x2 >> 11) * (2.0 ** -53)
    r = math.sqrt(-2.0 * math.log(u1))
    theta = 6.283185307179586 * u2
    return r * math.cos(theta), r * math.sin(theta)


def start_block(seed: int, d: int, k: int) -> np.ndarray:
    """Pi (d x k, row-major, FP32) from ``seed``."""
    total = d * k
    out = np.empty(total, dtype=np.float64)
    for p in range((total + 1) // 2):
        c, s = gaussian_pair(seed, p)
        out[2 * p] = c
        if 2 * p + 1 < total:
            out[2 * p + 1] = s
    return out.astype(np.float32).reshape(d, k)
