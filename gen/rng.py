"""Counter-based random numbers: the SplitMix64 sequence, vectorised.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; 64-bit output function as published by S. Vigna)
keeps a 64-bit state that advances by the odd constant gamma = 0x9E3779B97F4A7C15
and returns a bijective mix of the state.  The i-th output (i = 0, 1, ...) of
the sequence seeded with s is therefore mix(s + (i + 1) * gamma), which makes
it counter-based: any element can be computed independently, so a whole array
is one vectorised expression and the values never depend on the numpy version
or the machine.

Streams: a (seed, stream) pair is turned into a 64-bit starting state by
mixing, so the per-purpose streams (solution vector, coefficients, velocity,
...) do not overlap in practice.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (uint64 arithmetic wraps modulo 2^64)."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _start_state(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        s = _mix(s + _GAMMA * np.uint64(stream & 0xFFFF))
        return s[0]


def splitmix64_stream(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 sequence of (seed, stream)."""
    s0 = _start_state(seed, stream)
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix(s0 + k * _GAMMA)


def uniform01(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """53-bit uniform doubles in [0, 1): (x >> 11) * 2^-53."""
    x = splitmix64_stream(seed, stream, count, offset)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
