"""Counter-based random streams for the synthetic workloads.

Every number is SplitMix64's output function (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser
constants are Vigna's published SplitMix64) applied to ``base + k * GAMMA`` for
a running counter ``k``, so a stream is fully defined by ``(seed, stream)`` and
gives the same integers on every platform: only integer arithmetic is used to
draw ids.  This module holds no join arithmetic; it only draws numbers.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def mix64(z):
    """SplitMix64 finaliser; a bijection on uint64 (scalar or array)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _mix_int(x: int) -> int:
    x &= _MASK64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _MASK64
    return x ^ (x >> 31)


class Rng:
    """One seeded stream.  ``Rng(seed, stream)`` for independent sub-streams."""

    def __init__(self, seed: int, stream: int = 0):
        self.base = _mix_int(_mix_int(seed * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) ^ (stream & _MASK64))
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.ctr + 1, self.ctr + 1 + n, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return mix64(np.uint64(self.base) + k * GAMMA)

    def u32(self, n: int) -> np.ndarray:
        return (self.u64(n) >> np.uint64(32)).astype(np.uint32)

    def below(self, n: int, m) -> np.ndarray:
        """Integers in [0, m) (m scalar or array, 1 <= m <= 2**32), multiply-shift."""
        hi = self.u64(n) >> np.uint64(32)
        m = np.asarray(m, dtype=np.uint64)
        return ((hi * m) >> np.uint64(32)).astype(np.int64)

    def between(self, n: int, lo, hi) -> np.ndarray:
        """Integers in [lo, hi] inclusive."""
        lo = np.asarray(lo, dtype=np.int64)
        hi = np.asarray(hi, dtype=np.int64)
        return lo + self.below(n, (hi - lo + 1))

    def unit(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable")


def zipf_ranks(rng: Rng, n: int, domain: int, s: float) -> np.ndarray:
    """n ranks in [0, domain) with P(rank = r) proportional to (r+1)^-s.

    Inverse-CDF sampling; s == 0 is the uniform distribution.
    """
    if s == 0.0:
        return rng.below(n, domain)
    w = np.arange(1, domain + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    r = np.searchsorted(cdf, rng.unit(n), side="right")
    return np.minimum(r, domain - 1).astype(np.int64)
