"""Counter-based random numbers for the synthetic inputs.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the i-th output of stream `seed` is the SplitMix64
finaliser applied to seed + (i + 1) * golden_gamma.  Being counter based, any
element of any field can be regenerated on its own, and the streams are the
same on every host (x86 here, aarch64 on the GPU hosts).

This module draws numbers only; it holds none of the tiling method's
arithmetic.
"""
from __future__ import annotations

import zlib

import numpy as np

BASE_SEED = 20170403

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def subseed(base: int, *names) -> int:
    """Derive a 64-bit stream id from a base seed and a tuple of labels."""
    s = int(base) & _MASK64
    for name in names:
        h = zlib.crc32(str(name).encode())
        s = (s * 0x100000001B3 + h + 0x9E3779B9) & _MASK64
        s ^= s >> 29
    return s


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 outputs for the given counters of stream `seed` (uint64)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(int(seed) & _MASK64) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, shape, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """float64 samples of U[lo, hi) with 53 random bits each, C order."""
    n = int(np.prod(shape)) if len(shape) else 1
    z = splitmix64(seed, np.arange(n, dtype=np.uint64))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (lo + (hi - lo) * u).reshape(shape)


def log_uniform(seed: int, shape, lo: float, hi: float) -> np.ndarray:
    """exp(U[log lo, log hi)), e.g. conductivities spanning decades."""
    u = uniform(seed, shape)
    return np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)


def exponential(seed: int, n: int, rate: float) -> np.ndarray:
    """Inter-arrival gaps of a Poisson process with the given rate."""
    u = uniform(seed, (n,))
    return -np.log1p(-u) / rate
