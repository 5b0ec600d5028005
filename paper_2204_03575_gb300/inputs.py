"""Seeded synthetic inputs shared by the CUDA path, the oracle-based tests and the bench.

This module holds no arithmetic of the Cahn-Hilliard method: it only draws the
random initial fluctuations and the per-run sizes of the batched workload.

Initial states follow the experiments section (Section 4): each volume fraction
starts at a base value plus uniformly distributed fluctuations of +/-0.01.  The
uniform variates are drawn from the counter-based SplitMix64 generator (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
evaluated on a counter so that any node's value can be computed on its own:

    u(seed, field, node) = (splitmix64(seed ^ (field << 40) ^ node) >> 11) * 2**-53

field 0 is the polymer, field 1 the NFA.  The device side of the library
(``ch_state_init``) implements the same generator from the same definition.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x) -> np.ndarray:
    """One SplitMix64 output for each 64-bit counter value in ``x``."""
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, field: int, n: int) -> np.ndarray:
    """u in [0, 1) for nodes 0..n-1 of one field (53 random bits each)."""
    ctr = np.uint64(seed) ^ (np.uint64(field) << np.uint64(40)) ^ np.arange(n, dtype=np.uint64)
    return (splitmix64(ctr) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def initial_state(n_nodes: int, phi_p0: float, phi_nfa0: float, noise: float = 0.01,
                  seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Nodal phi_p, phi_nfa = base + noise * (2u - 1), fp64."""
    up = uniform(seed, 0, n_nodes)
    un = uniform(seed, 1, n_nodes)
    return phi_p0 + noise * (2.0 * up - 1.0), phi_nfa0 + noise * (2.0 * un - 1.0)


BATCH_SIZES = (64, 96, 128, 192, 256)


def batch_runs(nruns: int = 64, seed: int = 0, lo: float = 0.20, hi: float = 0.45):
    """Per-run (nx, ny, phi_p0, phi_nfa0) of the batched workload.

    Run r draws from the counter stream seed ^ (0xB47C << 40) ^ (r << 8) ^ k:
    k=0,1 pick nx, ny from BATCH_SIZES (independently), k=2,3 the two bases,
    uniform in [lo, hi).
    """
    out = []
    for r in range(nruns):
        base = np.uint64(seed) ^ (np.uint64(0xB47C) << np.uint64(40)) ^ (np.uint64(r) << np.uint64(8))
        u = (splitmix64(base ^ np.arange(4, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        nx = BATCH_SIZES[int(u[0] * len(BATCH_SIZES))]
        ny = BATCH_SIZES[int(u[1] * len(BATCH_SIZES))]
        out.append((nx, ny, lo + (hi - lo) * u[2], lo + (hi - lo) * u[3]))
    return out
