"""Counter-based splitmix64 (Steele, Lea and Flood, OOPSLA 2014).

Output ``i`` (i = 0, 1, ...) of the stream with seed ``s`` is
``mix(s + (i + 1) * 0x9E3779B97F4A7C15 mod 2**64)`` where ``mix`` is the
published splitmix64 finaliser.  Uniform doubles use the top 53 bits.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n, offset=0):
    """Return outputs offset .. offset+n-1 of the splitmix64 stream ``seed`` as uint64."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_01(seed, n, offset=0):
    """Uniform doubles in [0, 1): (x >> 11) * 2**-53."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed, n, offset=0):
    """Uniform doubles in [-1, 1): 2 * uniform_01 - 1 (exact in binary64)."""
    return uniform_01(seed, n, offset) * 2.0 - 1.0
