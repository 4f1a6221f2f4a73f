"""Counter-based splitmix64 streams (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), vectorised with numpy.

This module only draws random numbers for the synthetic inputs (graph shapes,
degrees, trip counts, payload round counts, arrival gaps).  It contains none
of the task-graph method's arithmetic: no payload, no condition hash, no
digest.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    """The splitmix64 output function applied elementwise (uint64, wrapping)."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def mix64_scalar(x: int) -> int:
    """Scalar splitmix64 finaliser, used to derive independent stream seeds."""
    x &= _MASK64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _MASK64
    return x ^ (x >> 31)


class Stream:
    """One splitmix64 sequence: value i is mix64(seed + (i + 1) * gamma).

    Streams are split by tag: Stream(seed, tag) starts from a seed derived from
    (seed, tag), so independent draws (degrees, predecessors, trips, ...) of
    one workload never share values.
    """

    def __init__(self, seed: int, tag: int = 0):
        self.state = mix64_scalar((int(seed) * 0x100000001B3 + 0x51ED2701 * (int(tag) + 1)) & _MASK64)
        self.pos = 0

    def u64(self, count: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            i = np.arange(self.pos + 1, self.pos + 1 + count, dtype=np.uint64)
            z = np.uint64(self.state) + i * _GAMMA
            out = _mix64(z)
        self.pos += count
        return out

    def below(self, count: int, span) -> np.ndarray:
        """Integers in [0, span) (span scalar or array, span <= 2**32), by the
        multiply-high range reduction of the top 32 bits."""
        r = self.u64(count) >> np.uint64(32)
        span = np.asarray(span, dtype=np.uint64)
        return ((r * span) >> np.uint64(32)).astype(np.int64)

    def integers(self, count: int, lo, hi) -> np.ndarray:
        """Integers uniform in [lo, hi] inclusive."""
        lo = np.asarray(lo, dtype=np.int64)
        hi = np.asarray(hi, dtype=np.int64)
        return lo + self.below(count, (hi - lo + 1))

    def uniform(self, count: int) -> np.ndarray:
        """Doubles uniform in [0, 1) from the top 53 bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
