"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds none of the search's arithmetic: only uniform random +-1 draws of given shapes
from numpy's PCG64 generator, and the length lists of the paper's workloads (odd
L = 201..303, Table 1).  Skew-symmetric inputs are built from these draws by
whichever side consumes them.
"""
from __future__ import annotations

import numpy as np


def random_pm1(shape, seed: int) -> np.ndarray:
    """Uniform i.i.d. +-1 values as int8."""
    rng = np.random.default_rng(seed)
    return (1 - 2 * rng.integers(0, 2, size=shape, dtype=np.int8)).astype(np.int8)


def random_free_vars(batch: int, L: int, seed: int) -> np.ndarray:
    """[batch, n] uniform +-1 free variables, n = (L+1)/2, for odd L."""
    if L % 2 == 0:
        raise ValueError("odd L only")
    return random_pm1((batch, (L + 1) // 2), seed)


def table1_lengths() -> list[int]:
    """The 52 odd lengths of Table 1."""
    return list(range(201, 304, 2))


def structured_pm1(kind: str, L: int) -> np.ndarray:
    """Degenerate +-1 sequences used as edge cases: all +1, alternating, half/half."""
    if kind == "ones":
        return np.ones(L, dtype=np.int8)
    if kind == "alternating":
        return np.array([1 if i % 2 == 0 else -1 for i in range(L)], dtype=np.int8)
    if kind == "halves":
        return np.array([1 if i < L // 2 else -1 for i in range(L)], dtype=np.int8)
    raise ValueError(kind)
