"""The one-launch path of shk_run (all steps of a mid-size bit-packed lattice
in one cooperative launch, a bounded grid barrier between half-steps) gives
the same spins and per-step sums as the per-launch path and the oracle, and
its barrier gives up with a reported timeout instead of hanging."""
import numpy as np
import pytest
import torch

import paper_1908_07341_gb300 as shk
from paper_1908_07341_gb300 import _lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield
    _lib.lib().shk_set_one_launch(0)


def _run(L, one_launch, n, t_split, obs):
    _lib.lib().shk_set_one_launch(1 if one_launch else 0)
    lat = shk.Lattice(L, "bitpack").set_seed(9, 4).set_params(0.7, 0.45).init("random", init_seed=5)
    rows = []
    for m in (t_split, n - t_split):        # two calls: the second resumes mid-run
        r = lat.run(m, obs=obs)
        if obs:
            rows.append(r.cpu().numpy())
    last = lat.read_observables()
    out = (lat.read_spins(0), lat.read_spins(1), np.concatenate(rows) if obs else None, last)
    lat.close()
    return out


@pytest.mark.parametrize("L", [288, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("obs", [True, False])
def test_one_launch_equals_per_launch(L, obs):
    n = 24 if L <= 1024 else 8
    a = _run(L, True, n, 5, obs)
    b = _run(L, False, n, 5, obs)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[3], b[3])
    if obs:
        assert np.array_equal(a[2], b[2])


def test_one_launch_matches_oracle(orc):
    L, n = 288, 6
    _lib.lib().shk_set_one_launch(1)
    try:
        _check_oracle(orc, L, n)
    finally:
        _lib.lib().shk_set_one_launch(0)


def _check_oracle(orc, L, n):
    lat = shk.Lattice(L, "bitpack").set_seed(3, 1).set_params(1.1, 0.35).init("random", init_seed=8)
    got = lat.run(n, obs=True).cpu().numpy()
    s = orc.init_plane(L, orc.INIT_RANDOM, 8, 1, 0)
    t = orc.init_plane(L, orc.INIT_RANDOM, 8, 1, 1)
    ref = orc.run(s, t, L, 1.1, 0.35, 3, 1, 0, n)
    assert np.array_equal(got, ref)
    assert np.array_equal(lat.read_spins(0).reshape(-1), s) and np.array_equal(lat.read_spins(1).reshape(-1), t)
    lat.close()


def test_grid_barrier_gives_up_and_reports():
    words = torch.zeros(4, dtype=torch.int32, device="cuda")
    flag = np.zeros(1, dtype=np.int32)
    so = _lib.lib()
    assert so.shk_barrier_timeout_test(2000, words.data_ptr(), flag.ctypes.data, None) == _lib.OK
    assert int(flag[0]) == 1
    # the context is still usable afterwards
    lat = shk.Lattice(512, "bitpack").set_seed(1, 0).set_params(1.0, 0.3).init("random", init_seed=1)
    lat.run(3)
    assert lat.read_observables().shape == (5,)
    lat.close()
