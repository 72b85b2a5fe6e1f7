"""SplitMix64: a counter-based 64-bit generator (Steele, Lea and Flood, OOPSLA 2014).

state_{k+1} = state_k + 0x9E3779B97F4A7C15; output = mix(state_{k+1}) with the
published 30/27/31 xor-shift-multiply finaliser.  Doubles take the top 53 bits.
"""
import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * _M1) & _MASK
        z = ((z ^ (z >> 27)) * _M2) & _MASK
        return z ^ (z >> 31)

    def next_double(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def _mix_array(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles in [lo, hi): element k is the (k+1)-th output of SplitMix64(seed)."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + k * np.uint64(_GAMMA)
    u = (_mix_array(z) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return lo + (hi - lo) * u


def seeded_field(seed: int, shape, lo=-1.0, hi=1.0) -> np.ndarray:
    """A seeded uniform field of the given shape (used for apply timing and parity inputs)."""
    n = int(np.prod(shape))
    return uniform(seed, n, lo, hi).reshape(shape)
