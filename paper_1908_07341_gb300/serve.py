"""Python face of the serving C ABI (shk_server_*): continuous batching of
simulation jobs, plus a driver that replays a timed arrival stream.

The scheduler (admission by slots and HBM budget, the arena allocator, the
per-tick launch and retirement) is native code in the library; this module
only marshals jobs and results and keeps the wall clock for latencies.
"""
from __future__ import annotations

import ctypes
import json
import time

import numpy as np
import torch

from . import _lib
from ._lib import lib

_INITS = {"up": _lib.INIT_ALL_UP, "down": _lib.INIT_ALL_DOWN, "random": _lib.INIT_RANDOM}


class Job(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("q", ctypes.c_double), ("J", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("lattice_id", ctypes.c_uint32), ("init_kind", ctypes.c_int),
                ("init_seed", ctypes.c_uint64), ("n_steps", ctypes.c_uint64), ("burn_in", ctypes.c_uint64),
                ("deadline_ticks", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("job_id", ctypes.c_uint64), ("status", ctypes.c_int), ("steps_done", ctypes.c_uint64),
                ("stats", ctypes.c_int64 * _lib.NSTATS), ("last_obs", ctypes.c_int64 * _lib.NOBS),
                ("sigma_hash", ctypes.c_uint64), ("submit_tick", ctypes.c_uint64),
                ("admit_tick", ctypes.c_uint64), ("done_tick", ctypes.c_uint64)]


def _check(status, handle):
    if status != _lib.OK:
        msg = lib().shk_server_last_error(handle) or lib().shk_last_error(None) or b""
        raise _lib.ShakenError(status, msg.decode(errors="replace"))


def fnv1a64(data: bytes) -> int:
    """The hash shk_result.sigma_hash uses (for comparing with other runs)."""
    h = 0xcbf29ce484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


class Server:
    def __init__(self, max_slots: int, arena_bytes: int, hbm_budget: int | None = None, device="cuda",
                 stream=None, result_log: str | None = None):
        """result_log: optional path; every result poll() returns is also
        appended to it as one JSON line."""
        self.result_log = result_log
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = int(lib().shk_server_bytes(int(max_slots), int(arena_bytes)))
        if nbytes == 0:
            raise ValueError("max_slots must be positive")
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        budget = int(arena_bytes if hbm_budget is None else hbm_budget)
        _check(lib().shk_server_create(int(max_slots), budget, self.buffer.data_ptr(), nbytes,
                                       int(self.stream.cuda_stream), ctypes.byref(h)), None)
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().shk_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, steps_per_launch=2, launches_per_tick=16, block_threads=256, tile_sites=1 << 18,
                  max_pending=1 << 20):
        _check(lib().shk_server_configure(self._h, int(steps_per_launch), int(launches_per_tick),
                                          int(block_threads), int(tile_sites), int(max_pending)), self._h)
        return self

    def submit(self, L, q, J, seed, lattice_id, n_steps, burn_in=0, init="random", init_seed=0,
               deadline_ticks=0) -> int:
        """Queues a job; deadline_ticks > 0 retires it with SHK_ETIMEOUT if it
        is not finished within that many ticks of its submission."""
        job = Job(int(L), float(q), float(J), int(seed) & (2 ** 64 - 1), int(lattice_id),
                  _INITS.get(init, init), int(init_seed), int(n_steps), int(burn_in), int(deadline_ticks))
        jid = ctypes.c_uint64()
        _check(lib().shk_server_submit(self._h, ctypes.byref(job), ctypes.byref(jid)), self._h)
        return int(jid.value)

    def cancel(self, job_id: int) -> None:
        _check(lib().shk_server_cancel(self._h, int(job_id)), self._h)

    def tick(self):
        a, p = ctypes.c_int(), ctypes.c_int()
        _check(lib().shk_server_tick(self._h, ctypes.byref(a), ctypes.byref(p)), self._h)
        return a.value, p.value

    def poll(self, max_results: int = 4096) -> list[dict]:
        buf = (Result * max_results)()
        n = ctypes.c_int()
        _check(lib().shk_server_poll(self._h, buf, max_results, ctypes.byref(n)), self._h)
        out = []
        for r in buf[: n.value]:
            out.append({"job_id": r.job_id, "status": r.status, "steps_done": r.steps_done,
                        "stats": np.array(r.stats[:], dtype=np.int64),
                        "last_obs": np.array(r.last_obs[:], dtype=np.int64), "sigma_hash": r.sigma_hash,
                        "submit_tick": r.submit_tick, "admit_tick": r.admit_tick, "done_tick": r.done_tick})
        if self.result_log and out:
            with open(self.result_log, "a") as f:
                for r in out:
                    f.write(json.dumps({k: (v.tolist() if isinstance(v, np.ndarray) else int(v))
                                        for k, v in r.items()}) + "\n")
        return out

    def read_job(self, job_id: int, L: int, plane: int = 0) -> tuple[np.ndarray, int]:
        """Spins (int8 +/-1, L x L) of a running job of side L between ticks,
        and the full steps it has completed."""
        out = np.zeros(int(L) * int(L), dtype=np.int8)
        steps = ctypes.c_uint64()
        _check(lib().shk_server_read_job(self._h, int(job_id), int(plane), out.ctypes.data, out.size,
                                         ctypes.byref(steps)), self._h)
        return out.reshape(int(L), int(L)), int(steps.value)

    def stats(self):
        t, u = ctypes.c_uint64(), ctypes.c_size_t()
        _check(lib().shk_server_stats(self._h, ctypes.byref(t), ctypes.byref(u)), self._h)
        return {"tick": int(t.value), "used_bytes": int(u.value)}


def replay_stream(server: Server, jobs: list[dict], arrivals, clock=time.perf_counter) -> dict:
    """Submits each job when the wall clock reaches its arrival time (seconds
    from the start), ticks the server while it has work, and records for every
    job the latency from arrival to the end of the tick that finished it."""
    order = np.argsort(np.asarray(arrivals))
    arrivals = np.asarray(arrivals, dtype=np.float64)
    t0 = clock()
    nxt, n = 0, len(jobs)
    id_to_idx, results = {}, {}
    busy = False
    while len(results) < n:
        now = clock() - t0
        while nxt < n and arrivals[order[nxt]] <= now:
            i = int(order[nxt])
            jid = server.submit(**jobs[i])
            id_to_idx[jid] = i
            nxt += 1
        if busy or nxt > len(results):
            active, pending = server.tick()
            done_at = clock() - t0
            for r in server.poll():
                i = id_to_idx[r["job_id"]]
                r["arrival_s"] = float(arrivals[i])
                r["done_s"] = done_at
                r["latency_s"] = done_at - float(arrivals[i])
                results[i] = r
            busy = active > 0 or pending > 0
        elif nxt < n:
            time.sleep(max(0.0, min(0.01, arrivals[order[nxt]] - (clock() - t0))))
    wall = clock() - t0
    lat = np.array([results[i]["latency_s"] for i in range(n)])
    return {"results": [results[i] for i in range(n)], "wall_s": wall,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean())}
