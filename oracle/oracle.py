"""ctypes wrapper around the plain C oracle (``shaken_oracle.c``).

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Every function here
only marshals numpy arrays into the C routines; the arithmetic of the method
lives in ``shaken_oracle.c`` (dynamics, Philox, thresholds) and in
``exact.py`` (exact laws by enumeration).
"""
from __future__ import annotations

import ctypes
import functools

import numpy as np

from . import build as _build

_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p

INIT_ALL_UP, INIT_ALL_DOWN, INIT_RANDOM = 0, 1, 2
N_OBS = 5  # M_sigma, M_tau, S_q, S_J, C_nn


@functools.lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    path = _build.build()
    so = ctypes.CDLL(path)
    so.orc_philox4x32_10.argtypes = [_ptr, _ptr, _ptr]
    so.orc_philox4x32_10.restype = None
    so.orc_block_uniforms.argtypes = [_u64, _u32, _u32, _u32, _u32, _ptr]
    so.orc_block_uniforms.restype = None
    so.orc_thresholds.argtypes = [_dbl, _dbl, _ptr]
    so.orc_thresholds.restype = _int
    so.orc_init.argtypes = [_ptr, _int, _int, _u64, _u32, _u32]
    so.orc_init.restype = None
    so.orc_halfstep_rows.argtypes = [_int, _ptr, _ptr, _int, _ptr, _u64, _u32, _u32, _int, _int]
    so.orc_halfstep_rows.restype = None
    so.orc_observables.argtypes = [_ptr, _ptr, _int, _ptr]
    so.orc_observables.restype = None
    so.orc_run.argtypes = [_ptr, _ptr, _int, _dbl, _dbl, _u64, _u32, _u64, _u64, _ptr]
    so.orc_run.restype = _int
    so.orc_diag_correlations.argtypes = [_ptr, _int, _ptr, _int, _ptr]
    so.orc_diag_correlations.restype = None
    so.orc_checkerboard_thresholds.argtypes = [_dbl, _ptr]
    so.orc_checkerboard_thresholds.restype = _int
    so.orc_checkerboard_halfstep.argtypes = [_ptr, _int, _ptr, _u64, _u32, _u32, _int]
    so.orc_checkerboard_halfstep.restype = None
    so.orc_checkerboard_run.argtypes = [_ptr, _int, _dbl, _u64, _u32, _u64, _u64, _ptr]
    so.orc_checkerboard_run.restype = _int
    so.orc_cftp.argtypes = [_int, _int, _dbl, _dbl, _u64, _u32, _int, _ptr]
    so.orc_cftp.restype = _int
    so.orc_cftp_many.argtypes = [_int, _int, _dbl, _dbl, _u64, _u32, _i64, _int, _ptr, _ptr]
    so.orc_cftp_many.restype = _int
    so.orc_many_chains.argtypes = [_int, _dbl, _dbl, _u64, _u32, _i64, _ptr, _u64, _ptr, _ptr]
    so.orc_many_chains.restype = _int
    return so


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block for a 4-word counter and a 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def block_uniforms(seed: int, c0: int, w: int, lattice_id: int, domain: int) -> np.ndarray:
    """The 32 site uniforms r(32w + p), p = 0..31, of one block."""
    out = np.zeros(32, dtype=np.uint32)
    lib().orc_block_uniforms(seed, c0, w, lattice_id, domain, _p(out))
    return out


def thresholds(q: float, J: float) -> np.ndarray:
    out = np.zeros(6, dtype=np.uint32)
    rc = lib().orc_thresholds(q, J, _p(out))
    if rc != 0:
        raise ValueError("q and J must be finite")
    return out


def init_plane(L: int, kind: int, init_seed: int = 0, lattice_id: int = 0,
               plane_index: int = 0) -> np.ndarray:
    out = np.zeros(L * L, dtype=np.int8)
    lib().orc_init(_p(out), L, kind, init_seed, lattice_id, plane_index)
    return out


def halfstep(half: int, src: np.ndarray, L: int, T: np.ndarray, seed: int,
             lattice_id: int, hs: int, row0: int = 0, row1: int | None = None,
             dst: np.ndarray | None = None) -> np.ndarray:
    """Half-step A (half=0, sigma -> tau) or B (half=1, tau -> sigma) on rows
    [row0, row1) of the output; rows outside keep the contents of ``dst``."""
    src = np.ascontiguousarray(src, dtype=np.int8).reshape(-1)
    if dst is None:
        dst = np.zeros(L * L, dtype=np.int8)
    T = np.ascontiguousarray(T, dtype=np.uint32)
    lib().orc_halfstep_rows(half, _p(src), _p(dst), L, _p(T), seed, lattice_id, hs,
                            row0, L if row1 is None else row1)
    return dst


def observables(sigma: np.ndarray, tau: np.ndarray, L: int) -> np.ndarray:
    out = np.zeros(N_OBS, dtype=np.int64)
    s = np.ascontiguousarray(sigma, dtype=np.int8).reshape(-1)
    t = np.ascontiguousarray(tau, dtype=np.int8).reshape(-1)
    lib().orc_observables(_p(s), _p(t), L, _p(out))
    return out


def run(sigma: np.ndarray, tau: np.ndarray, L: int, q: float, J: float, seed: int,
        lattice_id: int, t0: int, n: int, want_obs: bool = True):
    """n full steps in place on (sigma, tau); returns the (n, 5) int64 sums."""
    assert sigma.dtype == np.int8 and tau.dtype == np.int8
    obs = np.zeros((max(n, 1), N_OBS), dtype=np.int64) if want_obs else None
    rc = lib().orc_run(_p(sigma), _p(tau), L, q, J, seed, lattice_id, t0, n,
                       _p(obs) if want_obs else None)
    if rc != 0:
        raise ValueError("invalid oracle run arguments")
    return obs[:n] if want_obs else None


def many_chains(L: int, q: float, J: float, seed: int, id0: int, M: int,
                init_sigma: np.ndarray, n: int, want_tau: bool = False):
    """Final states of M independent chains (lattice ids id0..id0+M-1) as
    integer codes, bit u set iff the spin at u is +1."""
    init = np.ascontiguousarray(init_sigma, dtype=np.int8).reshape(-1)
    cs = np.zeros(M, dtype=np.uint64)
    ct = np.zeros(M, dtype=np.uint64) if want_tau else None
    rc = lib().orc_many_chains(L, q, J, seed, id0, M, _p(init), n, _p(cs),
                               _p(ct) if want_tau else None)
    if rc != 0:
        raise ValueError("invalid arguments")
    return (cs, ct) if want_tau else cs


def diag_correlations(sigma: np.ndarray, L: int, lags) -> np.ndarray:
    """SW-NE sums then NW-SE sums (see orc_diag_correlations)."""
    s = np.ascontiguousarray(sigma, dtype=np.int8).reshape(-1)
    lg = np.ascontiguousarray(lags, dtype=np.int32)
    out = np.zeros(2 * lg.size, dtype=np.int64)
    lib().orc_diag_correlations(_p(s), L, _p(lg), int(lg.size), _p(out))
    return out


def checkerboard_thresholds(J: float) -> np.ndarray:
    out = np.zeros(5, dtype=np.uint32)
    if lib().orc_checkerboard_thresholds(J, _p(out)) != 0:
        raise ValueError("J must be finite")
    return out


def checkerboard_halfstep(s: np.ndarray, L: int, T5, seed: int, lattice_id: int, hs: int, parity: int) -> np.ndarray:
    """In place: redraw the sites with (i + j) % 2 == parity."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    T = np.ascontiguousarray(T5, dtype=np.uint32)
    lib().orc_checkerboard_halfstep(_p(s), L, _p(T), seed, lattice_id, hs, parity)
    return s


def checkerboard_run(s: np.ndarray, L: int, J: float, seed: int, lattice_id: int, t0: int, n: int):
    """n full checkerboard steps in place; returns (n, 2) rows of (M, C_nn)."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    obs = np.zeros((max(n, 1), 2), dtype=np.int64)
    if lib().orc_checkerboard_run(_p(s), L, J, seed, lattice_id, t0, n, _p(obs)) != 0:
        raise ValueError("invalid checkerboard arguments (L must be even)")
    return obs[:n]


SHAKEN, CHECKERBOARD = 0, 1


def cftp(dyn: int, L: int, q: float, J: float, seed: int, lattice_id: int, k_max: int = 20):
    """One coupling-from-the-past sample (see orc_cftp): (k, state) with
    state None when no attempt up to k_max coalesced."""
    s = np.zeros(L * L, dtype=np.int8)
    k = lib().orc_cftp(dyn, L, q, J, seed, lattice_id, k_max, _p(s))
    if k == -2:
        raise ValueError("invalid cftp arguments")
    return k, (s if k >= 0 else None)


def cftp_many(dyn: int, L: int, q: float, J: float, seed: int, id0: int, M: int, k_max: int = 20):
    """M samples of a torus with L*L <= 64 as state codes, and their k."""
    codes = np.zeros(M, dtype=np.uint64)
    ks = np.zeros(M, dtype=np.int32)
    if lib().orc_cftp_many(dyn, L, q, J, seed, id0, M, k_max, _p(codes), _p(ks)) != 0:
        raise ValueError("invalid cftp arguments")
    return codes, ks
