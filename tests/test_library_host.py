"""CPU checks of the C-ABI library: it loads, exports every symbol the header
declares, computes the same threshold table as the oracle (independently
written), and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1908_07341_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def so():
    from paper_1908_07341_gb300 import build
    build.build()
    return _lib.lib()


def _declared_functions():
    with open(os.path.join(ROOT, "include", "shaken.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(shk_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(so):
    names = _declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(so, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"
    assert set(_lib.SIGNATURES) <= set(names)


def test_header_constants_match_binding():
    with open(os.path.join(ROOT, "include", "shaken.h")) as f:
        text = f.read()
    consts = dict(re.findall(r"#define\s+(SHK_[A-Z0-9_]+)\s+\(?(-?[0-9x]+)", text))
    for name, val in (("SHK_OK", _lib.OK), ("SHK_EINVAL", _lib.EINVAL), ("SHK_ESTATE", _lib.ESTATE),
                      ("SHK_BITPACK", _lib.BITPACK), ("SHK_INT8", _lib.INT8),
                      ("SHK_INIT_RANDOM", _lib.INIT_RANDOM), ("SHK_NOBS", _lib.NOBS),
                      ("SHK_MAX_L", _lib.MAX_L)):
        assert int(consts[name], 0) == val, name


@pytest.mark.parametrize("q,J", [(1.0, 0.25), (0.5, 0.5), (1.0, 0.35), (0.6585, 0.6585),
                                 (3.0, 0.44), (0.0, 0.0), (-2.0, 0.7), (30.0, 30.0), (1e-12, 0.0)])
def test_thresholds_equal_the_oracle(so, orc, q, J):
    out = np.zeros(6, dtype=np.uint32)
    assert so.shk_thresholds(q, J, out.ctypes.data) == _lib.OK
    assert np.array_equal(out, orc.thresholds(q, J))


def test_thresholds_equal_the_oracle_on_a_grid(so, orc):
    rng = np.random.default_rng(0)
    out = np.zeros(6, dtype=np.uint32)
    for q, J in rng.uniform(-4, 4, size=(2000, 2)):
        so.shk_thresholds(q, J, out.ctypes.data)
        assert np.array_equal(out, orc.thresholds(q, J))


def test_bad_arguments_are_rejected_without_a_gpu(so):
    out = np.zeros(6, dtype=np.uint32)
    assert so.shk_thresholds(float("nan"), 0.1, out.ctypes.data) == _lib.EINVAL
    assert b"finite" in so.shk_last_error(None)
    assert so.shk_plane_bytes(33, _lib.BITPACK) == 0
    assert so.shk_plane_bytes(1, _lib.INT8) == 0
    assert so.shk_plane_bytes(_lib.MAX_L * 2, _lib.INT8) == 0
    assert so.shk_plane_bytes(64, 7) == 0
    assert so.shk_plane_bytes(64, _lib.BITPACK) == 512
    assert so.shk_lattice_bytes(16384, _lib.BITPACK) == 2 * 16384 * 16384 // 8 + 512   # planes, ring, barrier
    h = ctypes.c_void_p()
    assert so.shk_lattice_create(33, _lib.BITPACK, 256, 1 << 20, None, ctypes.byref(h)) == _lib.EINVAL
    assert so.shk_lattice_create(64, _lib.BITPACK, 0, 1 << 20, None, ctypes.byref(h)) == _lib.EINVAL
    assert so.shk_lattice_create(64, _lib.BITPACK, 100, 1 << 20, None, ctypes.byref(h)) == _lib.EINVAL
    assert so.shk_lattice_create(64, _lib.BITPACK, 256, 16, None, ctypes.byref(h)) == _lib.ENOMEM
    assert b"needed" in so.shk_last_error(None)
    bad_T = np.full(6, 7, dtype=np.uint32)
    assert so.shk_halfstep(_lib.BITPACK, 0, 256, 512, 64, bad_T.ctypes.data, 1, 0, 0, None,
                           None) == _lib.EINVAL
    assert so.shk_halfstep(_lib.BITPACK, 2, 256, 512, 64, out.ctypes.data, 1, 0, 0, None,
                           None) == _lib.EINVAL
    assert so.shk_run(None, 5, None) == _lib.EINVAL
    assert so.shk_strerror(_lib.EBUSY) == b"busy"


def test_misaligned_planes_are_rejected_without_a_gpu(so):
    # the kernels move planes in 16-byte vectors: a misaligned pointer is an
    # argument error, reported before anything is launched
    T = np.zeros(6, dtype=np.uint32)
    assert so.shk_thresholds(0.5, 0.5, T.ctypes.data) == _lib.OK
    for layout in (_lib.BITPACK, _lib.INT8):
        assert so.shk_halfstep(layout, 0, 256 + 4, 1 << 20, 64, T.ctypes.data, 1, 0, 0, None, None) == _lib.EINVAL
        assert b"aligned" in so.shk_last_error(None)
        assert so.shk_halfstep(layout, 1, 256, (1 << 20) + 8, 64, T.ctypes.data, 1, 0, 0, None, None) == _lib.EINVAL
        assert so.shk_init_plane(layout, 256 + 1, 64, _lib.INIT_RANDOM, 1, 0, 0, None) == _lib.EINVAL
    lags = np.array([1], dtype=np.int32)
    assert so.shk_diag_correlations(256 + 4, 64, lags.ctypes.data, 1, 512, None) == _lib.EINVAL
    assert so.shk_checkerboard_run(ctypes.c_void_p(256 + 12), 64, 0.4, 1, 0, 0, 1, None, None) == _lib.EINVAL


def test_allocation_free_run_rejects_misaligned_pointers_without_a_gpu(so):
    # The allocation-free entry point runs the same vector-load sweeps: a sigma
    # plane off a 16-byte boundary (or a result buffer off an 8-byte one) is
    # refused before any CUDA call.  The pointers below are never dereferenced.
    for layout, L in ((_lib.BITPACK, 96), (_lib.BITPACK, 4096), (_lib.INT8, 257)):
        for off in (1, 4, 8, 12):
            rc = so.shk_shaken_run_static(layout, 0x10000 + off, L, 0.5, 0.5, 1, 0, 0, 3, None, None)
            assert rc == _lib.EINVAL, (layout, L, off)
            assert b"16-byte aligned" in so.shk_last_error(None)
        rc = so.shk_shaken_run_static(layout, 0x10000, L, 0.5, 0.5, 1, 0, 0, 3, 0x20004, None)
        assert rc == _lib.EINVAL
        assert b"8-byte aligned" in so.shk_last_error(None)
    assert so.shk_shaken_run_static(_lib.BITPACK, None, 96, 0.5, 0.5, 1, 0, 0, 3, None, None) == _lib.EINVAL


def test_handle_state_checks_without_a_gpu(so):
    # A handle over a fake (never dereferenced) aligned address: configuration
    # calls are host-only, and running before set_params is refused.
    h = ctypes.c_void_p()
    need = so.shk_lattice_bytes(64, _lib.BITPACK)
    assert so.shk_lattice_create(64, _lib.BITPACK, 1 << 20, need, None, ctypes.byref(h)) == _lib.OK
    try:
        assert so.shk_run(h, 3, None) == _lib.ESTATE
        assert b"set_params" in so.shk_last_error(h)
        assert so.shk_set_params(h, float("inf"), 0.2) == _lib.EINVAL
        assert so.shk_set_step(h, _lib.MAX_STEP) == _lib.EINVAL
        assert so.shk_set_step(h, 41) == _lib.OK
        t = ctypes.c_uint64()
        assert so.shk_get_step(h, ctypes.byref(t)) == _lib.OK and t.value == 41
        out = np.zeros(5, dtype=np.int64)
        assert so.shk_read_observables(h, out.ctypes.data) == _lib.ESTATE
        assert so.shk_plane_ptr(h, 1) == (1 << 20) + 512
    finally:
        so.shk_lattice_destroy(h)


def test_batch_arguments_are_checked_without_a_gpu(so):
    L = np.array([64, 2048, 32], dtype=np.int32)
    need = so.shk_batch_bytes(3, L.ctypes.data)
    assert need > 3 * (2048 * 2048 // 8)
    bad = np.array([64, 33], dtype=np.int32)
    assert so.shk_batch_bytes(2, bad.ctypes.data) == 0
    q = np.ones(3)
    J = np.ones(3)
    seed = np.zeros(3, dtype=np.uint64)
    ids = np.zeros(3, dtype=np.uint32)
    h = ctypes.c_void_p()
    assert so.shk_batch_create(3, L.ctypes.data, q.ctypes.data, J.ctypes.data, seed.ctypes.data,
                               ids.ctypes.data, 256, 1024, None, ctypes.byref(h)) == _lib.ENOMEM
    assert so.shk_batch_create(2, bad.ctypes.data, q.ctypes.data, J.ctypes.data, seed.ctypes.data,
                               ids.ctypes.data, 256, 1 << 30, None, ctypes.byref(h)) == _lib.EINVAL
    assert b"L=33" in so.shk_last_error(None)


def test_bulk_wait_timeout_test_argument_checks_without_a_gpu(so):
    flag = np.zeros(1, dtype=np.int32)
    assert so.shk_bulk_wait_timeout_test(0, flag.ctypes.data, None) == _lib.EINVAL
    assert so.shk_bulk_wait_timeout_test((1 << 30) + 1, flag.ctypes.data, None) == _lib.EINVAL
    assert so.shk_bulk_wait_timeout_test(1000, None, None) == _lib.EINVAL


def test_server_read_job_argument_checks_without_a_gpu(so):
    buf = np.zeros(64, dtype=np.int8)
    steps = ctypes.c_uint64()
    assert so.shk_server_read_job(None, 1, 0, buf.ctypes.data, buf.size, ctypes.byref(steps)) == _lib.EINVAL


def test_checkerboard_argument_checks_without_gpu():
    so = _lib.lib()
    dummy = ctypes.c_void_p(16)
    assert so.shk_checkerboard_run(dummy, 48, 0.4, 1, 0, 0, 1, None, None) == _lib.EINVAL
    assert so.shk_checkerboard_run(None, 64, 0.4, 1, 0, 0, 1, None, None) == _lib.EINVAL
    assert so.shk_checkerboard_run(dummy, 64, 0.4, 1, 0, 2 ** 31, 1, None, None) == _lib.EINVAL
    assert so.shk_checkerboard_run(dummy, 64, float("nan"), 1, 0, 0, 1, None, None) == _lib.EINVAL
    out = (ctypes.c_uint32 * 5)()
    assert so.shk_checkerboard_thresholds(float("inf"), out) == _lib.EINVAL
    assert so.shk_checkerboard_thresholds(0.0, out) == _lib.OK and list(out) == [2 ** 31] * 5


def test_philox_peak_argument_checks_without_gpu():
    so = _lib.lib()
    assert so.shk_philox_peak(0, 4, ctypes.c_void_p(16), None) == _lib.EINVAL
    assert so.shk_philox_peak(4, 0, ctypes.c_void_p(16), None) == _lib.EINVAL
    assert so.shk_philox_peak(4, 4, None, None) == _lib.EINVAL


def test_debug_bounds_is_refused_by_the_normal_build():
    so = _lib.lib()
    site = np.ones(1, dtype=np.uint32)
    assert so.shk_debug_bounds(site.ctypes.data) == _lib.ESTATE and site[0] == 0


def test_bounds_checked_build_exports_the_same_symbols():
    from paper_1908_07341_gb300 import build
    path = build.build(debug_bounds=True)
    dbg = ctypes.CDLL(path)
    for name in _lib.SIGNATURES:
        assert hasattr(dbg, name), name


def test_coalescence_and_cftp_argument_checks_without_gpu():
    so = _lib.lib()
    dummy = ctypes.c_void_p(256)
    L = np.array([32, 48], dtype=np.int32)
    q = np.array([1.0, 1.0])
    J = np.array([0.3, 0.3])
    seed = np.array([1, 1], dtype=np.uint64)
    ids = np.array([0, 1], dtype=np.uint32)
    T = np.zeros(2, dtype=np.uint64)
    ks = np.zeros(2, dtype=np.int32)
    nb = so.shk_coalescence_scratch_bytes(2)
    args = (L.ctypes.data, q.ctypes.data, J.ctypes.data, seed.ctypes.data, ids.ctypes.data)
    # L = 48 is not a multiple of 32; unknown dynamics; steps out of range
    assert so.shk_coalescence_times(0, 2, *args, 100, dummy, nb, T.ctypes.data, None) == _lib.EINVAL
    assert so.shk_coalescence_times(7, 1, *args, 100, dummy, nb, T.ctypes.data, None) == _lib.EINVAL
    assert so.shk_coalescence_times(0, 1, *args, 0, dummy, nb, T.ctypes.data, None) == _lib.EINVAL
    assert so.shk_coalescence_times(0, 1, *args, 100, dummy, 8, T.ctypes.data, None) == _lib.ENOMEM
    nc = so.shk_cftp_scratch_bytes(2)
    assert so.shk_cftp(0, 1, *args, 21, dummy, 128, dummy, nc, ks.ctypes.data, None) == _lib.EINVAL  # k_max
    assert so.shk_cftp(0, 2, *args, 10, dummy, 288, dummy, nc, ks.ctypes.data, None) == _lib.EINVAL  # L = 48
    assert so.shk_cftp(0, 1, *args, 10, dummy, 100, dummy, nc, ks.ctypes.data, None) == _lib.EINVAL  # stride < L^2/8
    assert so.shk_cftp(0, 1, *args, 10, dummy, 128, dummy, 4, ks.ctypes.data, None) == _lib.ENOMEM
    # the checkerboard dynamics needs no q
    assert so.shk_cftp(1, 1, L.ctypes.data, None, J.ctypes.data, seed.ctypes.data, ids.ctypes.data, 21,
                       dummy, 128, dummy, nc, ks.ctypes.data, None) == _lib.EINVAL       # still k_max
    assert so.shk_cftp(0, 1, L.ctypes.data, None, J.ctypes.data, seed.ctypes.data, ids.ctypes.data, 10,
                       dummy, 128, dummy, nc, ks.ctypes.data, None) == _lib.EINVAL       # shaken needs q


def test_step_counters_do_not_wrap():
    so = _lib.lib()
    huge = 2 ** 64 - 5
    assert so.shk_checkerboard_run(ctypes.c_void_p(256), 64, 0.4, 1, 0, 3, huge, None, None) == _lib.EINVAL
    assert so.shk_checkerboard_run(ctypes.c_void_p(256), 64, 0.4, 1, 0, huge, 3, None, None) == _lib.EINVAL
