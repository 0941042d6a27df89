"""splitmix64 (Steele, Lea and Flood, OOPSLA 2014), as a counter-based generator.

The d-th output of the generator seeded with s is mix(s + (d + 1) * gamma) with
gamma = 0x9E3779B97F4A7C15 and mix the published three-step finaliser.  The
eigenvalue-estimate start vector takes v[d] = 2 * u53(d) - 1 with u53 the top
53 bits of the d-th output scaled to [0, 1).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(d, seed: int = 0) -> np.ndarray:
    """d-th output(s) of splitmix64 seeded with ``seed`` (uint64 arithmetic mod 2^64)."""
    d = np.asarray(d, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (d + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def start_vector(n: int, seed: int = 0) -> np.ndarray:
    """Deterministic start vector in [-1, 1): v[d] = 2 * (splitmix64(d) >> 11) * 2^-53 - 1."""
    z = splitmix64(np.arange(n, dtype=np.uint64), seed)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0
