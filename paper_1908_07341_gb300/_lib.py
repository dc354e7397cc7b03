"""ctypes loader for libshaken.so.

Argument marshalling only: every step of the hot path runs in the CUDA
kernels behind the C ABI declared in include/shaken.h.  There is no CPU
fallback -- importing the binding without the built library raises.
"""
from __future__ import annotations

import atexit
import ctypes
import functools
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# SHK_LIBRARY selects another build of the same library, e.g. the bounds-checked
# libshaken_debug.so (build.py --debug-bounds).
LIB_PATH = os.environ.get("SHK_LIBRARY") or os.path.join(_PKG, "libshaken.so")

# status codes and enums (mirrors of include/shaken.h)
OK, EINVAL, ENOMEM, ECUDA, ESTATE, EBUSY, ETIMEOUT, ECANCELLED = 0, -1, -2, -3, -4, -5, -6, -7
BITPACK, INT8 = 1, 2
INIT_ALL_UP, INIT_ALL_DOWN, INIT_RANDOM = 0, 1, 2
HALF_A, HALF_B = 0, 1
NOBS = 5
NSTATS = 11
DYN_SHAKEN, DYN_CHECKERBOARD = 0, 1
CFTP_MAX_K = 20
MAX_L = 262144
MAX_STEP = 0x80000000

_c = ctypes
_vp, _i, _u32, _u64, _i64, _d, _sz = (_c.c_void_p, _c.c_int, _c.c_uint32, _c.c_uint64,
                                      _c.c_int64, _c.c_double, _c.c_size_t)

# name -> (restype, argtypes); every symbol include/shaken.h declares.
SIGNATURES = {
    "shk_strerror": (_c.c_char_p, [_i]),
    "shk_last_error": (_c.c_char_p, [_vp]),
    "shk_version": (_i, []),
    "shk_thresholds": (_i, [_d, _d, _vp]),
    "shk_plane_bytes": (_sz, [_i, _i]),
    "shk_halfstep": (_i, [_i, _i, _vp, _vp, _i, _vp, _u64, _u32, _u32, _vp, _vp]),
    "shk_sweep_variant_count": (_i, [_i]),
    "shk_sweep_variant_name": (_c.c_char_p, [_i, _i]),
    "shk_get_sweep_variant": (_i, [_i]),
    "shk_set_sweep_variant": (_i, [_i, _i]),
    "shk_diag_correlations": (_i, [_vp, _i, _vp, _i, _vp, _vp]),
    "shk_coalescence_scratch_bytes": (_sz, [_i]),
    "shk_coalescence_times": (_i, [_i, _i, _vp, _vp, _vp, _vp, _vp, _u64, _vp, _sz, _vp, _vp]),
    "shk_cftp_scratch_bytes": (_sz, [_i]),
    "shk_philox_peak": (_i, [_i, _u32, _vp, _vp]),
    "shk_debug_bounds": (_i, [_vp]),
    "shk_sweep_status": (_i, [_vp]),
    "shk_bulk_wait_timeout_test": (_i, [_u32, _vp, _vp]),
    "shk_set_specialize": (_i, [_i]),
    "shk_get_specialize": (_i, []),
    "shk_specialize_prepare": (_i, [_i, _i, _d, _d, _i]),
    "shk_specialize_shutdown": (_i, []),
    "shk_specialize_status": (_i, [_vp, _vp, _vp, _vp, _vp, _sz]),
    "shk_cftp": (_i, [_i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, _sz, _vp, _sz, _vp, _vp]),
    "shk_checkerboard_thresholds": (_i, [_d, _vp]),
    "shk_checkerboard_run": (_i, [_vp, _i, _d, _u64, _u32, _u64, _u64, _vp, _vp]),
    "shk_init_plane": (_i, [_i, _vp, _i, _i, _u64, _u32, _u32, _vp]),
    "shk_lattice_bytes": (_sz, [_i, _i]),
    "shk_lattice_create": (_i, [_i, _i, _vp, _sz, _vp, _vp]),
    "shk_lattice_destroy": (None, [_vp]),
    "shk_lattice_init": (_i, [_vp, _i, _u64]),
    "shk_set_params": (_i, [_vp, _d, _d]),
    "shk_set_seed": (_i, [_vp, _u64, _u32]),
    "shk_set_step": (_i, [_vp, _u64]),
    "shk_get_step": (_i, [_vp, _vp]),
    "shk_run": (_i, [_vp, _u64, _vp]),
    "shk_read_observables": (_i, [_vp, _vp]),
    "shk_read_spins": (_i, [_vp, _i, _vp]),
    "shk_write_spins": (_i, [_vp, _i, _vp]),
    "shk_upload_plane": (_i, [_vp, _i, _vp, _sz]),
    "shk_download_plane": (_i, [_vp, _i, _vp, _sz]),
    "shk_plane_ptr": (_vp, [_vp, _i]),
    "shk_batch_bytes": (_sz, [_i, _vp]),
    "shk_batch_create": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "shk_batch_destroy": (None, [_vp]),
    "shk_batch_last_error": (_c.c_char_p, [_vp]),
    "shk_batch_configure": (_i, [_vp, _i, _i, _i]),
    "shk_batch_init": (_i, [_vp, _i, _u64]),
    "shk_batch_run": (_i, [_vp, _u64, _u64]),
    "shk_batch_get_step": (_i, [_vp, _vp]),
    "shk_batch_read_stats": (_i, [_vp, _vp]),
    "shk_batch_read_observables": (_i, [_vp, _vp]),
    "shk_batch_read_spins": (_i, [_vp, _i, _i, _vp]),
    "shk_server_bytes": (_sz, [_i, _sz]),
    "shk_server_create": (_i, [_i, _sz, _vp, _sz, _vp, _vp]),
    "shk_server_destroy": (None, [_vp]),
    "shk_server_last_error": (_c.c_char_p, [_vp]),
    "shk_server_configure": (_i, [_vp, _i, _i, _i, _i, _sz]),
    "shk_server_submit": (_i, [_vp, _vp, _vp]),
    "shk_server_cancel": (_i, [_vp, _u64]),
    "shk_server_tick": (_i, [_vp, _vp, _vp]),
    "shk_server_poll": (_i, [_vp, _vp, _i, _vp]),
    "shk_server_stats": (_i, [_vp, _vp, _vp]),
    "shk_server_read_job": (_i, [_vp, _u64, _i, _vp, _sz, _vp]),
    "shk_shaken_run_static": (_i, [_i, _vp, _i, _d, _d, _u64, _u32, _u64, _u64, _vp, _vp]),
}


class ShakenError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


@functools.lru_cache(maxsize=1)
def lib() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"` "
            "(the shaken-dynamics hot path has no CPU fallback)")
    so = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(so, name)
        fn.restype = res
        fn.argtypes = args
    # interpreter exit runs this before any C exit handler: a run-time compile
    # still in flight finishes before the process tears anything down
    atexit.register(so.shk_specialize_shutdown)
    return so


def check(status: int, handle=None) -> None:
    if status != OK:
        msg = lib().shk_last_error(handle)
        raise ShakenError(status, (msg or b"").decode(errors="replace")
                          or lib().shk_strerror(status).decode())
