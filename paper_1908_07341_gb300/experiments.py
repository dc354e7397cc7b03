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
                         var_threshold: float = 0.03, device="cuda") -> dict:
    """One lattice per grid point (q_i, J_j), all spins -1 at the start,
    `warmup` steps, then the statistics of `measured` more steps.  Returns the
    grids of <m>, Var m and <|m|>, the J of the largest Var m for every q, the
    first J with Var m >= var_threshold for every q (the cells the paper's
    figures mark), and the timing."""
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
    # the paper's figures mark the cells with Var m >= 0.03; the first such J per q
    above = var_m >= var_threshold
    first_J = np.where(above.any(axis=1), J[np.argmax(above, axis=1)], np.nan)
    return {"L": L, "q": q, "J": J, "mean_m": d["m"].reshape(n_grid, n_grid), "var_m": var_m,
            "abs_m": d["abs_m"].reshape(n_grid, n_grid), "peak_J": peak_J, "J_c": critical_J(q),
            "var_threshold": var_threshold, "first_J_above_threshold": first_J,
            "stats": stats, "wall_s": wall,
            "site_updates": float(n) * 2.0 * L * L * total,
            "rate": float(n) * 2.0 * L * L * total / wall}


# ---- Section 3.2: coalescence times near the critical curve ----------------

def coalescence_scan(q_values, J_offsets=(-0.1, -0.05, 0.0, 0.05, 0.1), n_samples: int = 64, L: int = 32,
                     max_steps: int = 1 << 20, seed: int = 11, dynamics: str = "shaken", J_values=None) -> dict:
    """Mean coalescence time of the all + / all - chains (independent lattice
    ids per sample) at J = J_c(q) + offset for every q (or at the given
    J_values, one per q), all points in one launch."""
    from .lattice import coalescence_times
    q_values = np.asarray(q_values, dtype=np.float64)
    if J_values is None:
        Jg = critical_J(q_values)[:, None] + np.asarray(J_offsets)[None, :]
    else:
        Jg = np.asarray(J_values, dtype=np.float64).reshape(q_values.size, -1)
    Qg = np.broadcast_to(q_values[:, None], Jg.shape)
    n_pts = Jg.size
    Ls = np.full(n_pts * n_samples, L, dtype=np.int32)
    qs = np.repeat(Qg.ravel(), n_samples)
    Js = np.repeat(Jg.ravel(), n_samples)
    ids = np.arange(n_pts * n_samples, dtype=np.uint32)
    t0 = time.perf_counter()
    T = coalescence_times(Ls, qs, Js, np.uint64(seed), ids, max_steps, dynamics=dynamics).astype(np.float64)
    wall = time.perf_counter() - t0
    T = T.reshape(Jg.shape + (n_samples,))
    reached = T <= max_steps
    mean = np.where(reached.all(axis=-1), T.mean(axis=-1), np.nan)
    return {"L": L, "dynamics": dynamics, "q": q_values, "J": Jg, "mean_T": mean,
            "sem_T": T.std(axis=-1, ddof=1) / np.sqrt(n_samples), "log_mean_T": np.log(mean),
            "not_reached": (~reached).sum(axis=-1), "wall_s": wall}


# ---- Section 3.2: perfect samples, shaken vs checkerboard (square Gibbs) ---

def _sample_observables(samples: torch.Tensor, L: int) -> tuple[np.ndarray, np.ndarray]:
    """Magnetisation per site and C_nn = sum_x s_x (s_{x up} + s_{x right})
    of bit-packed samples (host-side analysis of a few small planes)."""
    from .lattice import unpack_bits
    host = samples.cpu().numpy()
    m = np.empty(host.shape[0])
    c = np.empty(host.shape[0], dtype=np.int64)
    for i in range(host.shape[0]):
        s = unpack_bits(host[i, : L * L // 8], L).reshape(L, L).astype(np.int64)
        m[i] = s.mean()
        c[i] = int(np.sum(s * (np.roll(s, -1, axis=0) + np.roll(s, -1, axis=1))))
    return m, c


def gibbs_comparison(J_values=(0.38, 0.40, 0.42, 0.44, 0.46), q_values=(0.5, 1.0, 1.5, 2.0, 2.5, 3.0),
                     n_samples: int = 256, L: int = 32, k_max: int = 18, seed: int = 21) -> dict:
    """Sample mean and standard deviation of m and of the square-lattice
    energy H_G = -J C_nn over coupling-from-the-past draws of the shaken
    dynamics (every q) and of the checkerboard heat bath, whose stationary law
    is the square-lattice Gibbs measure; also the mean number of steps 2^k of
    the successful attempts."""
    from .lattice import cftp
    J_values = np.asarray(J_values, dtype=np.float64)
    rows = []
    t0 = time.perf_counter()
    for dyn, qs in (("checkerboard", [0.0]), ("shaken", list(q_values))):
        for q in qs:
            n = J_values.size * n_samples
            Js = np.repeat(J_values, n_samples)
            ids = np.arange(n, dtype=np.uint32)
            ks, samples = cftp(np.full(n, L), np.full(n, q), Js, np.uint64(seed), ids, k_max=k_max, dynamics=dyn)
            m, c = _sample_observables(samples, L)
            for a, J in enumerate(J_values):
                sl = slice(a * n_samples, (a + 1) * n_samples)
                ok = ks[sl] >= 0
                H = -J * c[sl][ok]
                rows.append({"dynamics": dyn, "q": None if dyn == "checkerboard" else float(q), "J": float(J),
                             "n": int(ok.sum()), "mean_m": float(m[sl][ok].mean()) if ok.any() else None,
                             "sd_m": float(m[sl][ok].std(ddof=1)) if ok.sum() > 1 else None,
                             "mean_abs_m": float(np.abs(m[sl][ok]).mean()) if ok.any() else None,
                             "mean_H": float(H.mean()) if ok.any() else None,
                             "sd_H": float(H.std(ddof=1)) if ok.sum() > 1 else None,
                             "mean_steps": float(np.mean(2.0 ** ks[sl][ok])) if ok.any() else None})
    return {"L": L, "rows": rows, "wall_s": time.perf_counter() - t0}


# ---- Section 3.3 (Correlations, Table 1): diagonal spin-spin correlations --

TABLE1_POINTS = ((0.05, 1.7), (0.05, 1.855), (0.2, 1.05), (0.2, 1.175), (0.4, 0.82), (0.4, 0.86), (0.6, 0.67),
                 (0.6, 0.7), (0.65, 0.65), (0.663, 0.663), (0.8, 0.58), (0.8, 0.61), (1.0, 0.52), (1.0, 0.55),
                 (2.5, 0.43), (2.5, 0.46))


def diagonal_correlations_table(points=TABLE1_POINTS, lags=(1, 2, 4, 8, 16), L: int = 32, burn_in: int = 20_000,
                                n_samples: int = 2_000, gap: int = 10, seed: int = 31) -> dict:
    """<sigma_x sigma_{x+(l,l)}> (SW-NE) and <sigma_x sigma_{x+(l,-l)}> (NW-SE)
    on an L x L torus, averaged over the torus and over n_samples states taken
    every `gap` steps after `burn_in` steps from a random start."""
    from .lattice import Lattice, diag_correlations
    lags = list(lags)
    out = []
    t0 = time.perf_counter()
    for idx, (q, J) in enumerate(points):
        lat = Lattice(L).set_params(q, J).set_seed(seed, idx).init("random", seed)
        lat.run(burn_in)
        acc = torch.zeros(2 * len(lags), dtype=torch.int64, device=lat.device)
        for _ in range(n_samples):
            lat.run(gap)
            diag_correlations(lat.plane(0), L, lags, out=acc)
        sums = acc.cpu().numpy().astype(np.float64) / (n_samples * L * L)
        out.append({"q": q, "J": J, "supercritical": bool(J > critical_J(q)),
                    "sw_ne": sums[: len(lags)].tolist(), "nw_se": sums[len(lags):].tolist()})
        lat.close()
    return {"L": L, "lags": lags, "rows": out, "burn_in": burn_in, "n_samples": n_samples, "gap": gap,
            "wall_s": time.perf_counter() - t0}


def _jsonable(x):
    if isinstance(x, dict):
        return {k: _jsonable(v) for k, v in x.items() if k != "stats"}
    if isinstance(x, (list, tuple)):
        return [_jsonable(v) for v in x]
    if isinstance(x, np.ndarray):
        return _jsonable(x.tolist())
    if isinstance(x, (np.floating, float)):
        return None if not np.isfinite(x) else float(x)
    if isinstance(x, np.integer):
        return int(x)
    return x


def main(argv=None) -> None:
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Section 3 experiments on the GPU")
    ap.add_argument("which", choices=["critical-curve", "coalescence", "coalescence-hex", "coalescence-square",
                                      "gibbs", "correlations"])
    ap.add_argument("--out", default=None)
    ap.add_argument("--warmup", type=int, default=300_000)
    ap.add_argument("--measured", type=int, default=300_000)
    ap.add_argument("--grid", type=int, default=80)
    ap.add_argument("--L", type=int, default=None)
    ap.add_argument("--samples", type=int, default=None)
    a = ap.parse_args(argv)
    if a.which == "critical-curve":
        r = critical_curve_sweep(L=a.L or 224, n_grid=a.grid, warmup=a.warmup, measured=a.measured)
    elif a.which == "coalescence":
        r = coalescence_scan(grid_points(8, 2.0), n_samples=a.samples or 64, L=a.L or 32)
    elif a.which == "coalescence-hex":      # J = q: the isotropic hexagonal lattice
        qj = np.array([0.3, 0.4, 0.5, 0.55, 0.6, 0.6585, 0.7, 0.8])
        r = coalescence_scan(qj, n_samples=a.samples or 64, L=a.L or 32, J_values=qj[:, None])
    elif a.which == "coalescence-square":   # shaken at several q against the checkerboard chain
        Jv = np.array([0.3, 0.35, 0.4, 0.42, 0.44])
        qv = np.array([0.5, 1.0, 2.0, 3.0])
        sh = coalescence_scan(qv, n_samples=a.samples or 64, L=a.L or 32, J_values=np.tile(Jv, (qv.size, 1)))
        cb = coalescence_scan(np.zeros(1), n_samples=a.samples or 64, L=a.L or 32, J_values=Jv[None, :],
                              dynamics="checkerboard")
        r = {"shaken": sh, "checkerboard": cb}
    elif a.which == "gibbs":
        r = gibbs_comparison(n_samples=a.samples or 256, L=a.L or 32)
    else:
        r = diagonal_correlations_table(n_samples=a.samples or 2000, L=a.L or 32)
    text = json.dumps(_jsonable(r), indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    print(text[:4000])


if __name__ == "__main__":
    main()
