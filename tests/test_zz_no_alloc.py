"""GPU test of the allocation-free entry point shk_shaken_run_static.

That entry point is for callers that cannot allocate device memory, for
example a plug-in whose host application owns all device memory through its
own pool, or a latency-critical loop that cannot accept cudaMalloc's implicit
synchronisation.  It keeps the transient tau plane and the observable
accumulators in a static array inside the library.  Here it is called through
the C ABI twice in a row on the same sigma plane, and each call's spins and
sums must equal those of the ordinary lattice-handle path (shk_run) over the
same steps.  Spins and sums are integers, so the comparison is exact.  This
file is collected last.
"""
import numpy as np
import pytest
import torch

import paper_1908_07341_gb300 as shk
from paper_1908_07341_gb300 import _lib
from tests.gpu_util import from_device_plane, to_device_plane

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _run_static(layout, plane, L, q, J, seed, lat_id, t0, n, last):
    so = _lib.lib()
    rc = so.shk_shaken_run_static(_lib.BITPACK if layout == "bitpack" else _lib.INT8,
                                  plane.data_ptr(), L, q, J, seed, lat_id, t0, n,
                                  last.data_ptr() if last is not None else None,
                                  torch.cuda.current_stream().cuda_stream)
    return rc


@pytest.mark.parametrize("layout,L", [("bitpack", 1024), ("bitpack", 8192), ("bitpack", 64),
                                      ("int8", 257), ("int8", 2896)])
def test_static_scratch_run_equals_handle_run(layout, L):
    q, J, seed, lat_id = 0.8, 0.55, 4242, 3
    ref = shk.Lattice(L, layout).set_seed(seed, lat_id).set_params(q, J).init("random", init_seed=6)
    sigma0 = ref.read_spins(0).reshape(-1).copy()
    plane = to_device_plane(sigma0, L, layout)
    last = torch.zeros(shk.NOBS, dtype=torch.int64, device="cuda")
    t0 = 0
    for n in (9, 4):                                 # two calls in a row
        want_obs = ref.run(n, obs=True)[-1].cpu().numpy()
        want_sigma = ref.read_spins(0).reshape(-1)
        last.fill_(-12345)
        assert _run_static(layout, plane, L, q, J, seed, lat_id, t0, n, last) == _lib.OK
        torch.cuda.synchronize()
        t0 += n
        assert np.array_equal(from_device_plane(plane, L, layout), want_sigma), (layout, L, t0)
        assert np.array_equal(last.cpu().numpy(), want_obs), (layout, L, t0)


def test_static_scratch_rejects_sizes_beyond_its_limit():
    plane = torch.zeros(256, dtype=torch.uint8, device="cuda")   # never touched
    so = _lib.lib()
    for layout, L in ((_lib.BITPACK, 8224), (_lib.INT8, 2897)):
        rc = so.shk_shaken_run_static(layout, plane.data_ptr(), L, 0.5, 0.5, 1, 0, 0, 3, None, None)
        assert rc == _lib.EINVAL
        assert b"too large for the static scratch" in so.shk_last_error(None)
    rc = so.shk_shaken_run_static(_lib.BITPACK, plane.data_ptr(), 64, float("nan"), 0.5, 1, 0, 0, 3,
                                  None, None)
    assert rc == _lib.EINVAL


def test_static_scratch_without_result_buffer():
    L, layout = 96, "bitpack"
    ref = shk.Lattice(L, layout).set_seed(7, 0).set_params(1.0, 0.3).init("random", init_seed=2)
    plane = to_device_plane(ref.read_spins(0).reshape(-1), L, layout)
    ref.run(5)
    assert _run_static(layout, plane, L, 1.0, 0.3, 7, 0, 0, 5, None) == _lib.OK
    torch.cuda.synchronize()
    assert np.array_equal(from_device_plane(plane, L, layout), ref.read_spins(0).reshape(-1))


def test_static_scratch_queues_no_compile_even_in_blocking_mode():
    # Compiling a specialised sweep, or loading one as a module, allocates, so
    # the allocation-free entry point must do neither, whatever the
    # specialisation mode.  With blocking compiles requested, a call with a
    # threshold table the process has never seen still queues no compile, and
    # its spins equal those of a handle run with specialisation off.
    L, layout, q, J, seed = 4096, "bitpack", 0.9137, 0.4071, 77
    ref = shk.Lattice(L, layout).set_seed(seed, 0).set_params(q, J).init("random", init_seed=4)
    sigma0 = ref.read_spins(0).reshape(-1).copy()
    mode = shk.specialize()
    try:
        shk.specialize(shk.lattice.SPECIALIZE_OFF)
        want = ref.run(3, obs=True)[-1].cpu().numpy()
        want_sigma = ref.read_spins(0).reshape(-1)
        shk.specialize(shk.lattice.SPECIALIZE_BLOCKING)
        before = shk.specialize_status()
        plane = to_device_plane(sigma0, L, layout)
        last = torch.zeros(shk.NOBS, dtype=torch.int64, device="cuda")
        assert _run_static(layout, plane, L, q, J, seed, 0, 0, 3, last) == _lib.OK
        torch.cuda.synchronize()
        after = shk.specialize_status()
        assert (after["compiled"], after["queued"], after["failed"]) == \
            (before["compiled"], before["queued"], before["failed"])
        assert np.array_equal(from_device_plane(plane, L, layout), want_sigma)
        assert np.array_equal(last.cpu().numpy(), want)
    finally:
        shk.specialize(mode)

