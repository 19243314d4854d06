"""SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) with the two derived draws the input recipe uses.

uniform():  (x >> 11) * 2**-53, in [0, 1).
gauss():    Box-Muller from two consecutive uniforms, cosine branch only:
            sqrt(-2 ln(1 - u1)) * cos(2 pi u2).

The k-th output (k = 1, 2, ...) is mix(seed + k * 0x9E3779B97F4A7C15), so bulk draws are
computed with wrapping uint64 array arithmetic and give exactly the scalar sequence.
"""
import math

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix_np(z):
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def gauss(self) -> float:
        u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)

    # ---- bulk versions (identical sequence) ----
    def uniforms(self, n: int) -> np.ndarray:
        if n <= 0:
            return np.zeros(0, dtype=np.float64)
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + k * np.uint64(_GAMMA)
            x = _mix_np(z)
        self.state = (self.state + n * _GAMMA) & _MASK
        return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def gausses(self, n: int) -> np.ndarray:
        u = self.uniforms(2 * n).reshape(n, 2)
        return np.sqrt(-2.0 * np.log(1.0 - u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])
