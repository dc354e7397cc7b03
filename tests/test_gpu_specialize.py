"""The run-time specialised sweeps (thresholds compiled in as constants) draw
the same spins and sums as the generic kernels and the oracle, for every
sweep variant, both layouts, and threshold tables at the edges of the
range; and they are the kernels that actually ran."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_1908_07341_gb300 as shk
from paper_1908_07341_gb300 import _lib, tune

from gpu_util import from_device_plane, to_device_plane
from inputs import random_spins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield
    _lib.lib().shk_set_specialize(1)


def _status():
    c, f, qd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    log = ctypes.create_string_buffer(4096)
    assert _lib.lib().shk_specialize_status(ctypes.byref(c), ctypes.byref(f), ctypes.byref(qd), None, log, 4096) == _lib.OK
    return c.value, f.value, log.value.decode(errors="replace")


def _run(L, layout, q, J, n, specialize):
    # blocking mode: the specialised kernel is compiled before the first launch
    _lib.lib().shk_set_specialize(2 if specialize else 0)
    try:
        lat = shk.Lattice(L, layout).set_seed(21, 3).set_params(q, J).init("random", init_seed=4)
        obs = lat.run(n, obs=True).cpu().numpy()
        out = (lat.read_spins(0), lat.read_spins(1), obs)
        lat.close()
    finally:
        _lib.lib().shk_set_specialize(1)
    return out


# (q, J): generic, zero field everywhere (all thresholds 2^31), saturated
# thresholds, antiferromagnetic coupling, negative q
POINTS = [(0.7, 0.45), (0.0, 0.0), (25.0, 25.0), (0.3, -0.8), (-0.6, 0.5)]


@pytest.mark.parametrize("layout", ["bitpack", "int8"])
def test_every_variant_specialised_equals_generic(layout):
    L, n = 4096, 3      # large enough that no variant falls back to another
    before = tune.get_variant(layout)
    try:
        for v in range(len(tune.variant_names(layout))):
            tune.set_variant(layout, v)
            for q, J in POINTS[:3]:
                a = _run(L, layout, q, J, n, True)
                b = _run(L, layout, q, J, n, False)
                for x, y in zip(a, b):
                    assert np.array_equal(x, y), (tune.variant_names(layout)[v], q, J)
    finally:
        tune.set_variant(layout, before)
    c, f, log = _status()
    assert f == 0, log
    assert c >= 3


@pytest.mark.parametrize("layout,L", [("bitpack", 96), ("bitpack", 2048), ("int8", 288), ("int8", 1024)])
@pytest.mark.parametrize("q,J", POINTS)
def test_specialised_halfstep_matches_oracle(orc, layout, L, q, J):
    T = orc.thresholds(q, J)
    src = random_spins(L, seed=L + 7)
    _lib.lib().shk_set_specialize(2)
    for half in (0, 1):
        d_src = to_device_plane(src, L, layout)
        d_dst = to_device_plane(np.ones(L * L, np.int8), L, layout)
        shk.halfstep(layout, half, d_src, d_dst, L, T, 5, 2, 2 * 11 + half, None)
        want = orc.halfstep(half, src, L, T, 5, 2, 2 * 11 + half)
        assert np.array_equal(from_device_plane(d_dst, L, layout), want), (half, q, J)
    c, f, log = _status()
    assert f == 0, log


def test_specialised_kernels_are_cached_per_threshold_table():
    c0, _, _ = _status()
    _run(1024, "bitpack", 1.3, 0.21, 2, True)
    c1, _, _ = _status()
    _run(1024, "bitpack", 1.3, 0.21, 2, True)      # same table: no new compile
    c2, _, _ = _status()
    _run(1024, "bitpack", 1.3, 0.22, 2, True)      # new table: one more
    c3, f, log = _status()
    assert f == 0, log
    assert c1 == c0 + 1 and c2 == c1 and c3 == c2 + 1


def test_background_mode_switches_kernels_mid_run(orc):
    """Default mode: the first launches run generic while the compile is
    queued, later ones specialised; the trajectory is the oracle's throughout."""
    import time
    L, n, q, J = 288, 6, 0.8, 0.377
    _lib.lib().shk_set_specialize(1)
    lat = shk.Lattice(L, "bitpack").set_seed(2, 6).set_params(q, J).init("random", init_seed=3)
    rows = [lat.run(n, obs=True).cpu().numpy()]
    for _ in range(200):                   # the compile takes about a second
        c, f, qd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.lib().shk_specialize_status(ctypes.byref(c), ctypes.byref(f), ctypes.byref(qd), None, None, 0)
        if qd.value == 0:
            break
        time.sleep(0.05)
    rows.append(lat.run(n, obs=True).cpu().numpy())
    got = np.concatenate(rows)
    s = orc.init_plane(L, orc.INIT_RANDOM, 3, 6, 0)
    t = orc.init_plane(L, orc.INIT_RANDOM, 3, 6, 1)
    ref = orc.run(s, t, L, q, J, 2, 6, 0, 2 * n)
    assert np.array_equal(got, ref)
    assert np.array_equal(lat.read_spins(0).reshape(-1), s)
    lat.close()


def test_disabled_compiles_nothing():
    c0, f0, _ = _status()
    _run(1024, "bitpack", 0.9, 0.123, 2, False)
    c1, f1, _ = _status()
    assert (c1, f1) == (c0, f0)


_EXIT_CHILD = r"""
import sys
import paper_1908_07341_gb300 as shk
shk.specialize(1)
lat = shk.Lattice(1024, "bitpack").set_seed(1, 0).set_params(0.8, 0.31).init("random", init_seed=1)
lat.run(2)                      # the process's first compile, on this thread
for k in range(3):              # more tables: compiled in the background
    lat.set_params(0.8, 0.32 + 0.01 * k)
    lat.run(2)
lat.read_observables()
print("exiting", shk.specialize_status()["queued"], flush=True)
"""


def test_exit_with_compiles_in_flight_is_clean():
    """A process that exits right after queuing background compiles waits for
    the one in flight and exits normally."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _EXIT_CHILD], capture_output=True, text=True, timeout=300,
                           cwd=root)
        assert r.returncode == 0, (r.returncode, r.stdout[-500:], r.stderr[-2000:])
        assert "exiting" in r.stdout


@pytest.mark.parametrize("J", [0.44, 0.0, -0.3, 3.0])
def test_specialised_checkerboard_matches_generic_and_oracle(orc, J):
    """The checkerboard kernel compiled with the thresholds of J draws the
    oracle's spins and sums, as the generic one does."""
    from paper_1908_07341_gb300.lattice import checkerboard_run, pack_bits, unpack_bits
    L, n = 96, 3
    spins = random_spins(L, seed=13)
    out = []
    for mode in (2, 0):
        _lib.lib().shk_set_specialize(mode)
        try:
            plane = shk.alloc_plane(L, "bitpack")
            plane.zero_()
            raw = pack_bits(spins).view(np.uint8)
            plane[: raw.size].copy_(torch.from_numpy(raw.copy()))
            rows = checkerboard_run(plane, L, J, 4, 2, 5, n).cpu().numpy()
            out.append((unpack_bits(plane.cpu().numpy()[: L * L // 8], L).reshape(-1), rows))
        finally:
            _lib.lib().shk_set_specialize(1)
    ref = spins.copy()
    ref_rows = orc.checkerboard_run(ref, L, J, 4, 2, 5, n)
    for got, rows in out:
        assert np.array_equal(got, ref) and np.array_equal(rows, ref_rows)
    c, f, log = _status()
    assert f == 0, log
