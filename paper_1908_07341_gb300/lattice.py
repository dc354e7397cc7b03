"""Python face of the C ABI: a lattice handle over a torch-owned device buffer.

PyTorch supplies device memory and the CUDA stream; the library does all the
work.  Names follow the paper: sigma lives on Lambda_1 (plane 0), tau on
Lambda_2 (plane 1); (q, J) are the beta-rescaled couplings.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, lib

_LAYOUTS = {"bitpack": _lib.BITPACK, "int8": _lib.INT8, _lib.BITPACK: _lib.BITPACK, _lib.INT8: _lib.INT8}
_INITS = {"up": _lib.INIT_ALL_UP, "down": _lib.INIT_ALL_DOWN, "random": _lib.INIT_RANDOM}


def layout_code(layout) -> int:
    try:
        return _LAYOUTS[layout]
    except KeyError:
        raise ValueError(f"unknown layout {layout!r}; use 'bitpack' or 'int8'") from None


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def thresholds(q: float, J: float) -> np.ndarray:
    """The six integer thresholds T[k], k = 3*[s=+1] + n (host computation)."""
    out = np.zeros(6, dtype=np.uint32)
    check(lib().shk_thresholds(float(q), float(J), out.ctypes.data))
    return out


def plane_bytes(L: int, layout="bitpack") -> int:
    return int(lib().shk_plane_bytes(int(L), layout_code(layout)))


def lattice_bytes(L: int, layout="bitpack") -> int:
    return int(lib().shk_lattice_bytes(int(L), layout_code(layout)))


def alloc_plane(L: int, layout="bitpack", device="cuda") -> torch.Tensor:
    n = plane_bytes(L, layout)
    if n == 0:
        raise ValueError(f"invalid L={L} for layout {layout}")
    return torch.empty(n, dtype=torch.uint8, device=device)


def halfstep(layout, half: int, src: torch.Tensor, dst: torch.Tensor, L: int, T, seed: int,
             lattice_id: int, hs: int, obs_accum: torch.Tensor | None = None, stream=None) -> None:
    """One half-step over a whole plane (A: sigma -> tau, B: tau -> sigma)."""
    Tn = np.ascontiguousarray(T, dtype=np.uint32)
    for t in (src, dst):
        if not t.is_cuda:
            raise ValueError("planes must be CUDA tensors")
    if obs_accum is not None and (obs_accum.dtype != torch.int64 or obs_accum.numel() < _lib.NOBS):
        raise ValueError("obs_accum must be an int64 CUDA tensor of at least 5 entries")
    check(lib().shk_halfstep(layout_code(layout), int(half), src.data_ptr(), dst.data_ptr(), int(L),
                             Tn.ctypes.data, int(seed) & (2**64 - 1), int(lattice_id), int(hs),
                             obs_accum.data_ptr() if obs_accum is not None else None,
                             _stream_ptr(stream)))


def init_plane(layout, plane: torch.Tensor, L: int, kind="random", init_seed: int = 0,
               lattice_id: int = 0, plane_index: int = 0, stream=None) -> None:
    check(lib().shk_init_plane(layout_code(layout), plane.data_ptr(), int(L), _INITS.get(kind, kind),
                               int(init_seed), int(lattice_id), int(plane_index), _stream_ptr(stream)))


def diag_correlations(plane: torch.Tensor, L: int, lags, stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """SW-NE and NW-SE spin sums of a bit-packed device plane for each lag
    (int64 device tensor of 2 * len(lags): SW-NE first).  With `out` the sums
    are added to it (accumulation over samples)."""
    lg = np.ascontiguousarray(lags, dtype=np.int32)
    if out is None:
        out = torch.zeros(2 * lg.size, dtype=torch.int64, device=plane.device)
    elif out.dtype != torch.int64 or out.numel() < 2 * lg.size or not out.is_contiguous():
        raise ValueError("out must be a contiguous int64 tensor of 2 * len(lags) entries")
    check(lib().shk_diag_correlations(plane.data_ptr(), int(L), lg.ctypes.data, int(lg.size), out.data_ptr(),
                                      _stream_ptr(stream)))
    return out


_DYN = {"shaken": 0, "checkerboard": 1}


def _pair_arrays(L, q, J, seed, lattice_id):
    Ls = np.ascontiguousarray(L, dtype=np.int32).reshape(-1)
    n = Ls.size
    qs = np.ascontiguousarray(np.broadcast_to(q, (n,)), dtype=np.float64)
    Js = np.ascontiguousarray(np.broadcast_to(J, (n,)), dtype=np.float64)
    ss = np.ascontiguousarray(np.broadcast_to(seed, (n,)), dtype=np.uint64)
    ids = np.ascontiguousarray(np.broadcast_to(lattice_id, (n,)), dtype=np.uint32)
    return Ls, qs, Js, ss, ids


def coalescence_times(L, q, J, seed, lattice_id, max_steps: int, device="cuda", stream=None,
                      dynamics: str = "shaken") -> np.ndarray:
    """Coalescence time of the all + and all - chains of every pair (see
    shk_coalescence_times); max_steps + 1 where they did not meet.  dynamics:
    "shaken" or "checkerboard" (q ignored)."""
    Ls, qs, Js, ss, ids = _pair_arrays(L, q, J, seed, lattice_id)
    n = Ls.size
    nbytes = int(lib().shk_coalescence_scratch_bytes(n))
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=device)
    out = np.zeros(n, dtype=np.uint64)
    check(lib().shk_coalescence_times(_DYN[dynamics], n, Ls.ctypes.data, qs.ctypes.data, Js.ctypes.data,
                                      ss.ctypes.data, ids.ctypes.data, int(max_steps), scratch.data_ptr(), nbytes,
                                      out.ctypes.data, _stream_ptr(stream)))
    return out


def cftp(L, q, J, seed, lattice_id, k_max: int = 16, device="cuda", stream=None, dynamics: str = "shaken"):
    """Perfect samples by coupling from the past (see shk_cftp).  Returns
    (k, samples): k per pair (-1: not coalesced by k_max) and a uint8 device
    tensor of shape (n, max L^2 / 8) holding each bit-packed sigma."""
    Ls, qs, Js, ss, ids = _pair_arrays(L, q, J, seed, lattice_id)
    n = Ls.size
    stride = max(4, int(Ls.max()) ** 2 // 8)
    samples = torch.empty((n, stride), dtype=torch.uint8, device=device)
    nbytes = int(lib().shk_cftp_scratch_bytes(n))
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=device)
    ks = np.zeros(n, dtype=np.int32)
    check(lib().shk_cftp(_DYN[dynamics], n, Ls.ctypes.data, qs.ctypes.data, Js.ctypes.data, ss.ctypes.data,
                         ids.ctypes.data, int(k_max), samples.data_ptr(), stride, scratch.data_ptr(), nbytes,
                         ks.ctypes.data, _stream_ptr(stream)))
    return ks, samples


def checkerboard_thresholds(J: float) -> np.ndarray:
    out = np.zeros(5, dtype=np.uint32)
    check(lib().shk_checkerboard_thresholds(float(J), out.ctypes.data))
    return out


def checkerboard_run(plane: torch.Tensor, L: int, J: float, seed: int, lattice_id: int, t0: int, n_steps: int,
                     obs: bool = True, stream=None):
    """n_steps checkerboard heat-bath steps in place on a bit-packed device
    plane; returns the (n_steps, 2) int64 device rows of (M, C_nn) if obs."""
    out = torch.empty((int(n_steps), 2), dtype=torch.int64, device=plane.device) if obs else None
    check(lib().shk_checkerboard_run(plane.data_ptr(), int(L), float(J), int(seed) & (2 ** 64 - 1),
                                     int(lattice_id), int(t0), int(n_steps),
                                     out.data_ptr() if out is not None else None, _stream_ptr(stream)))
    return out


SPECIALIZE_OFF, SPECIALIZE_BACKGROUND, SPECIALIZE_BLOCKING = 0, 1, 2


def specialize(mode: int | None = None) -> int:
    """Run-time specialisation of the sweeps (thresholds compiled in as
    constants): sets the process-wide mode when given (0 off, 1 compile in the
    background, the default; 2 compile at first use and wait) and returns the
    mode now in force."""
    if mode is not None:
        check(lib().shk_set_specialize(int(mode)))
    return int(lib().shk_get_specialize())


def specialize_status() -> dict:
    """Entries compiled, failed and still queued, host seconds spent
    compiling, and the last failure's log."""
    c, f, qd, secs = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    log = ctypes.create_string_buffer(8192)
    check(lib().shk_specialize_status(ctypes.byref(c), ctypes.byref(f), ctypes.byref(qd), ctypes.byref(secs),
                                      log, len(log)))
    return {"compiled": c.value, "failed": f.value, "queued": qd.value, "compile_s": secs.value,
            "log": log.value.decode(errors="replace")}


def wait_specialized(timeout_s: float = 60.0) -> dict:
    """Waits (polling, bounded) until no specialised compile is queued."""
    import time
    t0 = time.perf_counter()
    st = specialize_status()
    while st["queued"] > 0 and time.perf_counter() - t0 < timeout_s:
        time.sleep(0.02)
        st = specialize_status()
    return st


def unpack_bits(words: np.ndarray, L: int) -> np.ndarray:
    """Host view of a bit-packed plane as int8 +/-1 of shape (L, L)."""
    w = np.ascontiguousarray(words).view(np.uint32)[: L * L // 32]
    bits = (w[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1
    return (2 * bits.astype(np.int8) - 1).reshape(L, L)


def pack_bits(spins: np.ndarray) -> np.ndarray:
    """int8 +/-1 array (L*L entries, L % 32 == 0) to bit-packed uint32 words."""
    s = (np.asarray(spins).reshape(-1, 32) > 0).astype(np.uint32)
    return (s << np.arange(32, dtype=np.uint32)[None, :]).sum(axis=1, dtype=np.uint64).astype(np.uint32)


class Lattice:
    """One L x L shaken-dynamics lattice pair (sigma, tau) resident on the GPU."""

    def __init__(self, L: int, layout="bitpack", device="cuda", stream=None):
        self.L = int(L)
        self.layout = layout_code(layout)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = lattice_bytes(self.L, self.layout)
        if nbytes == 0:
            raise ValueError(f"invalid L={L} for layout {layout}")
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        check(lib().shk_lattice_create(self.L, self.layout, self.buffer.data_ptr(), nbytes,
                                       int(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    # -- handle plumbing
    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("lattice closed")
        return self._h

    def _check(self, status):
        check(status, self._h)

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().shk_lattice_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration
    def set_params(self, q: float, J: float) -> "Lattice":
        self._check(lib().shk_set_params(self.handle, float(q), float(J)))
        self.q, self.J = float(q), float(J)
        return self

    def set_seed(self, seed: int, lattice_id: int = 0) -> "Lattice":
        self._check(lib().shk_set_seed(self.handle, int(seed) & (2**64 - 1), int(lattice_id)))
        return self

    def init(self, kind="random", init_seed: int = 0) -> "Lattice":
        self._check(lib().shk_lattice_init(self.handle, _INITS.get(kind, kind), int(init_seed)))
        return self

    @property
    def step(self) -> int:
        v = ctypes.c_uint64()
        self._check(lib().shk_get_step(self.handle, ctypes.byref(v)))
        return int(v.value)

    @step.setter
    def step(self, t: int) -> None:
        self._check(lib().shk_set_step(self.handle, int(t)))

    # -- dynamics
    def run(self, n_steps: int, obs: torch.Tensor | bool | None = None):
        """Runs n full steps; with obs=True returns a (n, 5) int64 device tensor
        of per-step observables, with a tensor writes into it."""
        out = None
        if obs is True:
            out = torch.empty((int(n_steps), _lib.NOBS), dtype=torch.int64, device=self.device)
        elif isinstance(obs, torch.Tensor):
            if obs.dtype != torch.int64 or obs.numel() < n_steps * _lib.NOBS or not obs.is_contiguous():
                raise ValueError("obs must be a contiguous int64 tensor of n_steps*5 entries")
            out = obs
        self._check(lib().shk_run(self.handle, int(n_steps), out.data_ptr() if out is not None else None))
        return out

    def read_observables(self) -> np.ndarray:
        out = np.zeros(_lib.NOBS, dtype=np.int64)
        self._check(lib().shk_read_observables(self.handle, out.ctypes.data))
        return out

    def read_spins(self, plane: int = 0) -> np.ndarray:
        out = np.zeros(self.L * self.L, dtype=np.int8)
        self._check(lib().shk_read_spins(self.handle, int(plane), out.ctypes.data))
        return out.reshape(self.L, self.L)

    def write_spins(self, plane: int, spins: np.ndarray) -> None:
        a = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
        if a.size != self.L * self.L:
            raise ValueError("spins must have L*L entries")
        self._check(lib().shk_write_spins(self.handle, int(plane), a.ctypes.data))

    def plane(self, plane: int) -> torch.Tensor:
        """The raw device plane (uint8 view in the handle's layout)."""
        n = plane_bytes(self.L, self.layout)
        off = 0 if plane == 0 else n
        return self.buffer[off:off + n]

    def upload_plane(self, plane: int, host: torch.Tensor | np.ndarray) -> None:
        ptr, n = (host.data_ptr(), host.numel() * host.element_size()) if isinstance(host, torch.Tensor) \
            else (host.ctypes.data, host.nbytes)
        self._check(lib().shk_upload_plane(self.handle, int(plane), ptr, n))

    def download_plane(self, plane: int, host: torch.Tensor | np.ndarray) -> None:
        ptr, n = (host.data_ptr(), host.numel() * host.element_size()) if isinstance(host, torch.Tensor) \
            else (host.ctypes.data, host.nbytes)
        self._check(lib().shk_download_plane(self.handle, int(plane), ptr, n))
