"""Counter-based random numbers: a pure function of (seed, stream, index).

The mixer is the splitmix64 finaliser (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) applied to a
linear combination of the three counters.  All arithmetic is modulo 2**64 on
numpy uint64 arrays, so it is identical on every platform.
"""

import numpy as np

_G1 = np.uint64(0x9E3779B97F4A7C15)
_G2 = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(seed, stream, index):
    """64-bit hash of (seed, stream, index); broadcasts over numpy arrays."""
    s = np.asarray(seed, dtype=np.uint64)
    t = np.asarray(stream, dtype=np.uint64)
    i = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = s * _G1 + (t + np.uint64(1)) * _G2 + i
        z = z ^ (z >> np.uint64(30))
        z = z * _M1
        z = z ^ (z >> np.uint64(27))
        z = z * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def unit_float(seed, stream, index):
    """Uniform float64 in [0, 1) from the top 53 bits of mix64."""
    z = mix64(seed, stream, index)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_int(seed, stream, index, lo, hi):
    """Integer in [lo, hi] inclusive: lo + (mix64 mod (hi - lo + 1))."""
    z = mix64(seed, stream, index)
    span = np.uint64(hi - lo + 1)
    return (z % span).astype(np.int64) + lo
