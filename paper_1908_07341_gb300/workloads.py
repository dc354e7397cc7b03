"""Seeded synthetic workloads (inputs only: no arithmetic of the method).

phase_diagram_batch reproduces the batched configuration: 1024 lattices, side
L_k drawn log-uniformly from {32, 64, ..., 2048} by a seeded generator, cell
k of a 32 x 32 (q, J) grid with q in [0.05, 3.0] and J in [0.05, 1.5], seed 4,
lattice id k, random starts, 10^4 steps with the first half as burn-in.
"""
from __future__ import annotations

import numpy as np


def phase_diagram_batch(n_side: int = 32, seed: int = 4, q_range=(0.05, 3.0), J_range=(0.05, 1.5),
                        L_choices=(32, 64, 128, 256, 512, 1024, 2048)) -> dict:
    n = n_side * n_side
    k = np.arange(n)
    i, j = k // n_side, k % n_side
    q = q_range[0] + i * (q_range[1] - q_range[0]) / (n_side - 1)
    J = J_range[0] + j * (J_range[1] - J_range[0]) / (n_side - 1)
    rng = np.random.default_rng(seed)
    L = np.asarray(L_choices, dtype=np.int32)[rng.integers(0, len(L_choices), size=n)]
    return {"L": L, "q": q, "J": J, "seed": np.full(n, seed, dtype=np.uint64),
            "lattice_id": k.astype(np.uint32), "init_seed": seed, "steps": 10_000, "burn_in": 5_000}


def serving_stream(n_jobs: int = 10_000, rate_per_s: float = 200.0, seed: int = 5, L_range=(64, 4096),
                   q_range=(0.05, 3.0), J_range=(0.05, 1.5), steps_range=(1_000, 100_000)) -> dict:
    """The serving configuration: Poisson arrivals (mean rate rate_per_s), L
    log-uniform in L_range rounded to a multiple of 32, q and J uniform, steps
    log-uniform in steps_range, seed 5 and lattice id = job index for every
    job, random starts, burn-in half the steps."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_jobs))
    L = np.exp(rng.uniform(np.log(L_range[0]), np.log(L_range[1]), size=n_jobs))
    L = np.clip((np.rint(L / 32) * 32).astype(np.int64), 32, None)
    q = rng.uniform(*q_range, size=n_jobs)
    J = rng.uniform(*J_range, size=n_jobs)
    steps = np.rint(np.exp(rng.uniform(np.log(steps_range[0]), np.log(steps_range[1]), size=n_jobs)))
    steps = steps.astype(np.int64)
    jobs = [dict(L=int(L[i]), q=float(q[i]), J=float(J[i]), seed=seed, lattice_id=i, n_steps=int(steps[i]),
                 burn_in=int(steps[i]) // 2, init="random", init_seed=seed) for i in range(n_jobs)]
    return {"jobs": jobs, "arrivals": arrivals, "site_updates": float((2.0 * L.astype(np.float64) ** 2 * steps).sum())}
