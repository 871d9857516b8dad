"""Counter-based SplitMix64 stream and Box-Muller normals.

SplitMix64 is the generator of Steele, Lea and Flood, "Fast splittable
pseudorandom number generators" (OOPSLA 2014): the k-th output of stream
``seed`` is ``mix64(seed + (k + 1) * 0x9E3779B97F4A7C15)`` with the
published 64-bit finaliser (shifts 30, 27, 31 and the two odd multipliers).
Uniforms take the top 53 bits; normals use the Box-Muller transform
(Box and Muller, Ann. Math. Statist. 29, 1958) on consecutive pairs.

Everything here is vectorised NumPy on uint64 with wrap-around arithmetic, so
the same (seed, counter) gives the same number on any host.  Nothing in this
module knows about the preconditioner.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser applied elementwise to uint64 words."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class SplitMix64:
    """A stream identified by ``seed``; draws advance an internal counter."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def raw(self, count: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + count, dtype=np.uint64)
        self.counter += count
        with np.errstate(over="ignore"):
            return mix64(self.seed + k * GAMMA)

    def uniform(self, count: int) -> np.ndarray:
        """Uniforms in [0, 1) from the top 53 bits."""
        return (self.raw(count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, count: int) -> np.ndarray:
        """Standard normals by Box-Muller on pairs of uniforms."""
        pairs = (count + 1) // 2
        u = self.uniform(2 * pairs).reshape(pairs, 2)
        r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))  # 1 - u in (0, 1]
        t = 2.0 * np.pi * u[:, 1]
        out = np.empty(2 * pairs)
        out[0::2] = r * np.cos(t)
        out[1::2] = r * np.sin(t)
        return out[:count]

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Integers uniform on [lo, hi] inclusive (multiply-shift on 53-bit uniforms)."""
        span = hi - lo + 1
        return lo + np.floor(self.uniform(count) * span).astype(np.int64)
