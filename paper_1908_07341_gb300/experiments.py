"""Experiments of the paper's Section 3 built on the batched kernel.

critical_curve_sweep  Section 3.1: mean and variance of the magnetisation of
                      sigma over a (q, J) grid from an all -1 start, and the J
                      of the variance peak per q against J_c(q) (Eq. J_di_q).

Everything that runs on the GPU goes through the C ABI (shk_batch_*); this
module only sets up the grid and reduces the exact integer statistics.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from .batch import Batch, derived


def critical_J(q):
    """J_c(q) = atanh(sqrt(tanh^2 q + 1) - tanh q), Eq. J_di_q."""
    t = np.tanh(np.asarray(q, dtype=np.float64))
    return np.arctanh(np.sqrt(t * t + 1.0) - t)


def grid_points(n: int, upper: float) -> np.ndarray:
    """n interior points of the open interval (0, upper): (i + 1) upper / (n + 1)."""
    return (np.arange(n) + 1.0) * upper / (n + 1.0)


def critical_curve_sweep(L: int = 224, n_grid: int = 80, q_max: float = 2.0, J_max: float = 2.0,
                         warmup: int = 300_000, measured: int = 300_000, seed: int = 1,
                         steps_per_launch: int = 8, block_threads: int = 256, tile_sites: int = 1 << 18,
                         device="cuda") -> dict:
    """One lattice per grid point (q_i, J_j), all spins -1 at the start,
    `warmup` steps, then the statistics of `measured` more steps.  Returns the
    grids of <m>, Var m and <|m|>, the J of the largest Var m for every q, and
    the timing."""
    q = grid_points(n_grid, q_max)
    J = grid_points(n_grid, J_max)
    Q, JJ = np.meshgrid(q, J, indexing="ij")
    n = n_grid * n_grid
    total = warmup + measured
    if total % steps_per_launch:
        raise ValueError("warmup + measured must be a multiple of steps_per_launch")
    b = Batch(np.full(n, L, dtype=np.int32), Q.ravel(), JJ.ravel(), np.full(n, seed, dtype=np.uint64),
              np.arange(n, dtype=np.uint32), device=device)
    b.configure(steps_per_launch, block_threads, tile_sites).init("down")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(total, burn_in=warmup)
    stats = b.read_stats()
    wall = time.perf_counter() - t0
    b.close()
    d = derived(stats, np.full(n, L), Q.ravel(), JJ.ravel())
    var_m = d["var_m"].reshape(n_grid, n_grid)
    peak_J = J[np.argmax(var_m, axis=1)]
    return {"L": L, "q": q, "J": J, "mean_m": d["m"].reshape(n_grid, n_grid), "var_m": var_m,
            "abs_m": d["abs_m"].reshape(n_grid, n_grid), "peak_J": peak_J, "J_c": critical_J(q),
            "stats": stats, "wall_s": wall,
            "site_updates": float(n) * 2.0 * L * L * total,
            "rate": float(n) * 2.0 * L * L * total / wall}
