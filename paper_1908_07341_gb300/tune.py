"""Autotuner for the launch shapes of the half-step sweeps.

Every variant draws exactly the same spins (the random numbers depend only on
the site, the half-step and the seed), so the choice is purely about speed.
The tuner times each variant with CUDA events on the caller's stream over a
few launches of shk_halfstep on scratch planes of the requested size, sets the
fastest process-wide through the C ABI, and caches the choice per
(GPU name, layout, size class) in a JSON file (an entry made for another list
of variants is timed again).
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import _lib
from .lattice import alloc_plane, halfstep, init_plane, layout_code, thresholds

_CACHE_PATH = os.environ.get(
    "SHK_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "shaken_gb300", "tune.json"))
_lock = threading.Lock()


def variant_names(layout) -> list[str]:
    code = layout_code(layout)
    so = _lib.lib()
    return [so.shk_sweep_variant_name(code, v).decode() for v in range(so.shk_sweep_variant_count(code))]


def get_variant(layout) -> int:
    return int(_lib.lib().shk_get_sweep_variant(layout_code(layout)))


def set_variant(layout, variant: int) -> None:
    _lib.check(_lib.lib().shk_set_sweep_variant(layout_code(layout), int(variant)))


def size_class(L: int) -> str:
    """Sizes whose best launch shape is expected to agree: powers of two."""
    return f"L<={1 << max(5, (int(L) - 1).bit_length())}"


def time_variants(layout, L: int, launches: int = 20, reps: int = 5) -> dict[int, float]:
    """Mean milliseconds per half-step launch of every variant at side L,
    measured on back-to-back launches replayed from a captured CUDA graph (so
    host-side launch overhead is excluded).  Unless specialisation is off, each
    variant is timed in its specialised form (compiled, blocking, before the
    warm-up launches)."""
    code = layout_code(layout)
    n = _lib.lib().shk_sweep_variant_count(code)
    a, b = alloc_plane(L, layout), alloc_plane(L, layout)
    init_plane(layout, a, L, "random", init_seed=1)
    T = thresholds(1.0, 0.35)
    acc = torch.zeros(_lib.NOBS, dtype=torch.int64, device=a.device)
    before = get_variant(layout)
    mode_before = int(_lib.lib().shk_get_specialize())
    if mode_before != 0:
        _lib.check(_lib.lib().shk_set_specialize(2))
    out = {}

    def enqueue(stream):
        for k in range(launches):
            half = k & 1
            halfstep(code, half, a if half == 0 else b, b if half == 0 else a, L, T, 7, 0, k, acc, stream)

    try:
        for v in range(n):
            set_variant(layout, v)
            enqueue(torch.cuda.current_stream())          # warm-up, outside the graph
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                enqueue(torch.cuda.current_stream())
            g.replay()
            torch.cuda.synchronize()
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record()
            for _ in range(reps):
                g.replay()
            e.record()
            torch.cuda.synchronize()
            out[v] = s.elapsed_time(e) / (reps * launches)
            del g
    finally:
        set_variant(layout, before)
        _lib.lib().shk_set_specialize(mode_before)
    return out


def _load_cache() -> dict:
    try:
        with open(_CACHE_PATH) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(cache: dict) -> None:
    try:
        os.makedirs(os.path.dirname(_CACHE_PATH), exist_ok=True)
        tmp = _CACHE_PATH + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, _CACHE_PATH)
    except OSError:
        pass


def autotune(layout, L: int, use_cache: bool = True, stream=None) -> int:
    """Picks and sets the fastest sweep variant for (layout, L); returns it."""
    if layout_code(layout) == _lib.INT8 and L % 32 != 0:
        return get_variant(layout)      # the generic int8 path has a single shape
    key = f"{torch.cuda.get_device_name()}|{layout_code(layout)}|{size_class(L)}"
    with _lock:
        cache = _load_cache() if use_cache else {}
        if key in cache and cache[key].get("names") == variant_names(layout):
            best = int(cache[key]["variant"])
        else:
            times = time_variants(layout, L)
            best = min(times, key=times.get)
            cache = _load_cache()
            cache[key] = {"variant": best, "ms": times, "names": variant_names(layout)}
            _store_cache(cache)
        set_variant(layout, best)
    return best


def autotune_batch(batch, steps_per_launch=(2, 4, 8, 16), block_threads=(256, 512),
                   tile_sites=(1 << 16, 1 << 17, 1 << 18, 1 << 19), launches: int = 3,
                   init_kind="random", init_seed: int = 0) -> dict:
    """Times every (steps per launch, block size, tile size) on a few launches
    of the given batch and configures the fastest.  The batch is left
    re-initialised (kind, init_seed) with its step counter at 0.  Returns
    {"best": (k, block, tile_sites), "ms_per_step": {...}}."""
    results = {}
    stream = batch.stream
    for k in steps_per_launch:
        for blk in block_threads:
            for ts in tile_sites:
                try:
                    batch.configure(k, blk, ts)
                except _lib.ShakenError:
                    continue            # tile does not fit in shared memory
                batch.init(init_kind, init_seed)
                batch.run(k)            # warm-up launch (graph capture)
                s = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                s.record(stream)
                batch.run(k * launches)
                e.record(stream)
                torch.cuda.synchronize()
                results[(k, blk, ts)] = s.elapsed_time(e) / (k * launches)
    best = min(results, key=results.get)
    batch.configure(*best)
    batch.init(init_kind, init_seed)
    return {"best": best, "ms_per_step": {f"{k}/{b}/{t}": v for (k, b, t), v in results.items()}}
