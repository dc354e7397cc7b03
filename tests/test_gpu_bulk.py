"""The int8 sweeps that move rows with bulk asynchronous copies: spins and
sums equal to the oracle's, no fault reported after normal runs, and the
failure path of their bounded waits (a wait that cannot complete gives up,
sets the fault word and the host reports it), exercised without a fault."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1908_07341_gb300 as shk
from paper_1908_07341_gb300 import _lib, tune

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("name", ["strip-bulk4-256x3"])
@pytest.mark.parametrize("L", [1024, 3072])
def test_bulk_strip_walk_matches_the_oracle(orc, name, L):
    names = tune.variant_names("int8")
    before = tune.get_variant("int8")
    tune.set_variant("int8", names.index(name))
    try:
        lat = shk.Lattice(L, "int8").set_seed(17, 2).set_params(0.9, 0.45).init("random", init_seed=5)
        obs = lat.run(3, obs=True).cpu().numpy()
        s = orc.init_plane(L, orc.INIT_RANDOM, 5, 2, 0)
        t = orc.init_plane(L, orc.INIT_RANDOM, 5, 2, 1)
        ref = orc.run(s, t, L, 0.9, 0.45, 17, 2, 0, 3)
        assert np.array_equal(obs, ref)
        assert np.array_equal(lat.read_spins(0).reshape(-1), s)
        assert np.array_equal(lat.read_spins(1).reshape(-1), t)
        assert _lib.lib().shk_sweep_status(None) == _lib.OK
    finally:
        tune.set_variant("int8", before)


def test_bounded_bulk_wait_gives_up_and_is_reported():
    so = _lib.lib()
    flag = ctypes.c_int(-1)
    stream = torch.cuda.current_stream().cuda_stream
    # about a millisecond at the GB300's clock: the probe's barrier never completes
    assert so.shk_bulk_wait_timeout_test(2_000_000, ctypes.byref(flag), stream) == _lib.OK
    assert flag.value == 1
    # the word was cleared by the test call: the next status check is clean,
    # and the context still runs work
    assert so.shk_sweep_status(stream) == _lib.OK
    lat = shk.Lattice(64, "int8").set_seed(1, 0).set_params(1.0, 0.25).init("up")
    lat.run(2)
    assert lat.read_spins(0).shape == (64, 64)
