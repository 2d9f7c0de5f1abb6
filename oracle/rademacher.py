"""Counter-based Rademacher probes: the oracle's own implementation.

The paper draws the sketch S and the residual probes from i.i.d. +-1 entries
(the sketch-sampling step of Algorithms 2 and 3; Sec. 2.2 and
Sec. 3.2) but does not name a generator.  Both sides of the parity check
implement this one from the published SplitMix64 definition (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):

    mix(z) = z3 with  z1 = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9
                      z2 = (z1 ^ (z1 >> 27)) * 0x94d049bb133111eb
                      z3 = z2 ^ (z2 >> 31)            (all mod 2^64)
    the i-th output (i = 0, 1, ...) of the generator seeded with s is
        mix(s + (i + 1) * GOLDEN),  GOLDEN = 0x9e3779b97f4a7c15.

Probe entry (row, col) of stream ``stream`` for ``seed``:

    key   = mix(seed + (stream + 1) * GOLDEN)          # a per-stream seed
    bits  = mix(key + (col * 2^32 + row + 1) * GOLDEN)  # output #(col*2^32+row)
    value = +1 if bits >> 63 == 0 else -1

Stream 0 is the sketch S, stream 1 the residual probes G.  ``row`` is the
row index of the matrix as given by the caller.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def splitmix64_mix(z):
    """The SplitMix64 output finaliser on uint64 (scalar or array), wrapping mod 2^64."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_sequence(seed: int, count: int) -> np.ndarray:
    """First ``count`` outputs of the SplitMix64 generator seeded with ``seed``."""
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64_mix(np.uint64(seed) + i * GOLDEN)


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return splitmix64_mix(np.uint64(seed) + np.uint64(stream + 1) * GOLDEN)[()]


def rademacher_bits(seed: int, stream: int, n: int, ncols: int, col0: int = 0) -> np.ndarray:
    """Raw 64-bit outputs, shape (n, ncols), for columns col0 .. col0+ncols-1."""
    key = stream_key(seed, stream)
    rows = np.arange(n, dtype=np.uint64)[:, None]
    cols = np.arange(col0, col0 + ncols, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        ctr = (cols << np.uint64(32)) + rows + np.uint64(1)
        return splitmix64_mix(key + ctr * GOLDEN)


def gaussian_block(seed: int, stream: int, n: int, ncols: int, col0: int = 0) -> np.ndarray:
    """n x ncols standard normal entries from the same counters (Box-Muller).

    For entry (row, col) with counter output z (as in rademacher_bits) and
    w = mix(z) (the output finaliser applied once more):
        u1 = ((z >> 11) + 1) * 2^-53   in (0, 1]
        u2 = (w >> 11) * 2^-53         in [0, 1)
        g  = sqrt(-2 log u1) cos(2 pi u2).
    """
    z = rademacher_bits(seed, stream, n, ncols, col0)
    with np.errstate(over="ignore"):
        w = splitmix64_mix(z)
    u1 = ((z >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0**-53
    u2 = (w >> np.uint64(11)).astype(np.float64) * 2.0**-53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def rademacher_block(seed: int, stream: int, n: int, ncols: int, col0: int = 0) -> np.ndarray:
    """n x ncols matrix of +-1.0 (float64)."""
    bits = rademacher_bits(seed, stream, n, ncols, col0)
    return np.where((bits >> np.uint64(63)) == 0, 1.0, -1.0)
