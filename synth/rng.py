"""Counter-based random numbers for the seeded synthetic lattice fields.

Every value is a pure function of (seed, stream, counter), so any slice of a
field can be regenerated independently (and in any chunking) with identical
results.  The bit generator is SplitMix64 (G. Steele, D. Lea, C. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), used here in
counter mode: the 64-bit state for draw ``k`` is ``key + (k + 1) * GAMMA`` and
the output is the SplitMix64 finaliser applied to that state.  With
``key = seed`` and ``k = 0, 1, ...`` this is exactly the sequential SplitMix64
stream, which the tests pin against the published first outputs for seed
1234567.

Normals come from the Box-Muller transform (Box and Muller, Ann. Math.
Statist. 29, 1958) on pairs of uniforms in (0, 1).

This module holds no lattice arithmetic; it only turns counters into numbers.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)


def _finalise(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (uint64 arrays wrap modulo 2**64)."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of an independent stream: stream 0 keeps the raw seed."""
    with np.errstate(over="ignore"):
        if stream == 0:
            return np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        z = np.array([(seed ^ (stream * 0xD1B54A32D192ED03)) & 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
        return _finalise(z + GAMMA)[0]


def raw_u64(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """64-bit outputs for the given counters of stream ``stream``."""
    key = stream_key(seed, stream)
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _finalise(key + (c + np.uint64(1)) * GAMMA)


def uniform(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in the open interval (0, 1): the top 53 bits, offset by 1/2 ulp."""
    z = raw_u64(seed, stream, counters)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def complex_normal(seed: int, stream: int, first: int, count: int,
                   variance: float = 1.0) -> np.ndarray:
    """``count`` complex normals z with E|z|^2 = ``variance``.

    Complex number j (j = first .. first+count-1) uses uniform counters 2j and
    2j+1; its real and imaginary parts are the two Box-Muller outputs, each
    with variance ``variance / 2``.
    """
    j = np.arange(first, first + count, dtype=np.uint64)
    u1 = uniform(seed, stream, np.uint64(2) * j)
    u2 = uniform(seed, stream, np.uint64(2) * j + np.uint64(1))
    rad = np.sqrt(-2.0 * np.log(u1) * (variance / 2.0))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang) + 1j * (rad * np.sin(ang))
