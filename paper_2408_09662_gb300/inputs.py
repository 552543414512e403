"""Seeded synthetic inputs for the benchmark workloads (numpy PCG64).

Random numbers only: this module holds none of the method's arithmetic, so the
CUDA path, the oracle, the tests and the benchmark can all draw their inputs
from it.  Arrays are [rows, N], instance-fastest (row k of instance i at
[k, i]), float64.
"""
from __future__ import annotations

import numpy as np


def cartpole(N: int, seed: int = 0) -> np.ndarray:
    """Rows: x, th, xd, thd ~ U[-1, 1]; f ~ U[-10, 10]."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(-1.0, 1.0, size=(4, N))
    f = rng.uniform(-10.0, 10.0, size=(1, N))
    return np.vstack([q, f])


def normal(rows: int, N: int, seed: int = 1) -> np.ndarray:
    """Standard normal inputs (the random-program workload draws seed 1)."""
    return np.random.default_rng(seed).standard_normal(size=(rows, N))


def uniform(rows: int, N: int, lo: float, hi: float, seed: int = 0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=(rows, N))
