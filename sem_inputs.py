"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the solver: it only turns (seed, index)
pairs into pseudo-random numbers, so that the oracle and the GPU library are
fed byte-identical data.  The generator is SplitMix64 (G. L. Steele, D. Lea,
C. H. Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
used in counter mode: draw number i of stream `seed` is the SplitMix64 output
mixing function applied to  seed * G + (i + 1) * G  (mod 2^64), G the golden
gamma 0x9E3779B97F4A7C15.  The top 53 bits give a double in [0, 1).

Inputs the solver consumes:
  * uniform_nodal(seed, shape, lo, hi)  - i.i.d. nodal values, e.g. the random
    right-hand side U[-1, 1] at GLL nodes or the random initial guess U[0, 1]
    of the convergence studies (index = row-major position in the node grid).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 output for draw `index` (uint64 array) of stream `seed`."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GAMMA + (idx + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from stream `seed` (53-bit mantissa)."""
    z = splitmix64(seed, np.arange(n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_nodal(seed: int, shape, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Array of `shape` with i.i.d. U[lo, hi) entries, row-major draw order."""
    n = int(np.prod(shape))
    return (lo + (hi - lo) * uniform01(seed, n)).reshape(shape)


def geometric_edges(n: int, first_width: float, length: float = 1.0) -> np.ndarray:
    """n + 1 element edges on [0, length] whose widths grow geometrically from
    `first_width` (the ratio is found by bisection so that the widths sum to
    `length`).  Mesh geometry only: an input of the stretched-mesh workloads."""
    if first_width * n >= length:
        raise ValueError("first_width too large for a growing mesh")
    lo, hi = 1.0, 2.0
    while first_width * (hi**n - 1) / (hi - 1) < length:
        hi *= 2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        tot = first_width * n if mid == 1.0 else first_width * (mid**n - 1) / (mid - 1)
        lo, hi = (mid, hi) if tot < length else (lo, mid)
    r = 0.5 * (lo + hi)
    w = first_width * r ** np.arange(n)
    e = np.concatenate([[0.0], np.cumsum(w)])
    e *= length / e[-1]
    return e


def nu_contrast(c: float):
    """nu(x, y) = 1 + (c - 1)(1/2 + 1/2 sin(2 pi x) cos(2 pi y)) (contrast c)."""
    return lambda x, y: 1.0 + (c - 1.0) * (0.5 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y))


def nu_paper(amplitude: float, shift: float):
    """nu(x, y) = 1 + a sin(2 pi (x - s)) sin(2 pi (y - s))."""
    return lambda x, y: 1.0 + amplitude * np.sin(2 * np.pi * (x - shift)) * np.sin(2 * np.pi * (y - shift))
