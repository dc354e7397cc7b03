"""Seeded synthetic inputs shared by the GPU path and the oracle in tests.

Holds none of the method's arithmetic: only reproducible random spin planes.
"""
import numpy as np


def random_spins(L: int, seed: int, p_up: float = 0.5) -> np.ndarray:
    """int8 +/-1 plane of L*L sites, each +1 with probability p_up."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random(L * L) < p_up, 1, -1).astype(np.int8)


def single_plus(L: int, site: int) -> np.ndarray:
    s = -np.ones(L * L, dtype=np.int8)
    s[site] = 1
    return s
