"""Python face of the batched-lattice C ABI (shk_batch_*).

A batch advances many independent bit-packed lattices of uneven side L, each
with its own (q, J), seed and lattice id, in one persistent kernel; a run is
one CUDA graph launch whose while node repeats the kernel.  The statistics
are exact int64 sums; ``derived`` turns them into the usual per-lattice
averages in FP64.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import lib

_INITS = {"up": _lib.INIT_ALL_UP, "down": _lib.INIT_ALL_DOWN, "random": _lib.INIT_RANDOM}
STAT_NAMES = ["sum_M", "sum_M2", "sum_absM", "sum_SJ", "sum_Sq", "sum_SJ2", "sum_Sq2", "sum_SJSq",
              "sum_Cnn", "sum_Cnn2", "count"]


def _check(status, handle):
    if status != _lib.OK:
        msg = lib().shk_batch_last_error(handle) or lib().shk_last_error(None) or b""
        raise _lib.ShakenError(status, msg.decode(errors="replace"))


class Batch:
    def __init__(self, L, q, J, seed, lattice_id, device="cuda", stream=None):
        self.L = np.ascontiguousarray(L, dtype=np.int32)
        self.n = int(self.L.size)
        self.q = np.ascontiguousarray(np.broadcast_to(q, (self.n,)), dtype=np.float64)
        self.J = np.ascontiguousarray(np.broadcast_to(J, (self.n,)), dtype=np.float64)
        self.seed = np.ascontiguousarray(np.broadcast_to(seed, (self.n,)), dtype=np.uint64)
        self.lattice_id = np.ascontiguousarray(np.broadcast_to(lattice_id, (self.n,)), dtype=np.uint32)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = int(lib().shk_batch_bytes(self.n, self.L.ctypes.data))
        if nbytes == 0:
            raise ValueError("invalid lattice sizes (need 32 <= L <= 65536, L % 32 == 0)")
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        _check(lib().shk_batch_create(self.n, self.L.ctypes.data, self.q.ctypes.data, self.J.ctypes.data,
                                      self.seed.ctypes.data, self.lattice_id.ctypes.data,
                                      self.buffer.data_ptr(), nbytes, int(self.stream.cuda_stream),
                                      ctypes.byref(h)), None)
        self._h = h
        self.steps_per_launch = 8

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().shk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def configure(self, steps_per_launch=8, block_threads=256, tile_sites=1 << 18) -> "Batch":
        _check(lib().shk_batch_configure(self._h, int(steps_per_launch), int(block_threads), int(tile_sites)),
               self._h)
        self.steps_per_launch = int(steps_per_launch)
        return self

    def init(self, kind="random", init_seed: int = 0) -> "Batch":
        _check(lib().shk_batch_init(self._h, _INITS.get(kind, kind), int(init_seed)), self._h)
        return self

    def run(self, n_steps: int, burn_in: int = 0) -> None:
        _check(lib().shk_batch_run(self._h, int(n_steps), int(burn_in)), self._h)

    @property
    def step(self) -> int:
        v = ctypes.c_uint64()
        _check(lib().shk_batch_get_step(self._h, ctypes.byref(v)), self._h)
        return int(v.value)

    def read_stats(self) -> np.ndarray:
        out = np.zeros((self.n, _lib.NSTATS), dtype=np.int64)
        _check(lib().shk_batch_read_stats(self._h, out.ctypes.data), self._h)
        return out

    def read_observables(self) -> np.ndarray:
        out = np.zeros((self.n, _lib.NOBS), dtype=np.int64)
        _check(lib().shk_batch_read_observables(self._h, out.ctypes.data), self._h)
        return out

    def read_spins(self, idx: int, plane: int = 0) -> np.ndarray:
        L = int(self.L[idx])
        out = np.zeros(L * L, dtype=np.int8)
        _check(lib().shk_batch_read_spins(self._h, int(idx), int(plane), out.ctypes.data), self._h)
        return out.reshape(L, L)


def stats_from_observables(obs: np.ndarray) -> np.ndarray:
    """The eleven exact sums of shk_batch from per-step rows of the five
    observables (used to compare a batch with single-lattice runs)."""
    o = np.asarray(obs, dtype=np.int64)
    M, Sq, SJ, C = o[:, 0], o[:, 2], o[:, 3], o[:, 4]
    return np.array([M.sum(), (M * M).sum(), np.abs(M).sum(), SJ.sum(), Sq.sum(), (SJ * SJ).sum(),
                     (Sq * Sq).sum(), (SJ * Sq).sum(), C.sum(), (C * C).sum(), len(o)], dtype=np.int64)


def derived(stats: np.ndarray, L, q, J) -> dict:
    """Per-lattice FP64 averages from the exact sums: <m>, <|m|>, <m^2>, Var m,
    susceptibility chi = N (<m^2> - <m>^2), <H>, Var H with
    H = -(J S_J + q S_q), and the square-lattice energy -J <C_nn>."""
    s = np.asarray(stats, dtype=np.float64)
    N = np.asarray(L, dtype=np.float64) ** 2
    q = np.asarray(q, dtype=np.float64)
    J = np.asarray(J, dtype=np.float64)
    n = np.maximum(s[:, 10], 1.0)
    m = s[:, 0] / n / N
    m2 = s[:, 1] / n / N ** 2
    absm = s[:, 2] / n / N
    EJ, Eq = s[:, 3] / n, s[:, 4] / n
    H = -(J * EJ + q * Eq)
    H2 = J * J * s[:, 5] / n + 2 * J * q * s[:, 7] / n + q * q * s[:, 6] / n
    return {"m": m, "abs_m": absm, "m2": m2, "var_m": m2 - m * m, "chi": N * (m2 - m * m),
            "H": H, "var_H": H2 - H * H, "E_square": -J * s[:, 8] / n}
