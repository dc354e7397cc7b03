"""GPU parity of the Section 3 kernels: diagonal correlation sums and
coalescence times, against the oracle."""
import numpy as np
import pytest
import torch

import paper_1908_07341_gb300 as shk
from paper_1908_07341_gb300.lattice import coalescence_times, diag_correlations
from tests.gpu_util import to_device_plane
from tests.inputs import random_spins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("L", [32, 64, 96, 1024])
def test_diag_correlations_match_oracle(orc, L):
    lags = [0, 1, 2, 4, 8, 16, 31, L - 1] if L > 32 else [0, 1, 2, 4, 8, 16, 31]
    s = random_spins(L, seed=L + 3, p_up=0.6)
    got = diag_correlations(to_device_plane(s, L, "bitpack"), L, lags).cpu().numpy()
    assert np.array_equal(got, orc.diag_correlations(s, L, lags))


def _oracle_T(orc, L, q, J, seed, lat_id, max_steps):
    top_s, top_t = np.ones(L * L, np.int8), np.ones(L * L, np.int8)
    bot_s, bot_t = -np.ones(L * L, np.int8), -np.ones(L * L, np.int8)
    for t in range(max_steps):
        orc.run(top_s, top_t, L, q, J, seed, lat_id, t, 1, want_obs=False)
        orc.run(bot_s, bot_t, L, q, J, seed, lat_id, t, 1, want_obs=False)
        if np.array_equal(top_s, bot_s):
            return t + 1
    return max_steps + 1


def test_coalescence_times_match_oracle(orc):
    """T = min{n : sigma_top(n) = sigma_bottom(n)} of Section 3.2 for coupled
    chains from all + and all -, computed step by step by the oracle."""
    pairs = [(32, 0.5, 0.3, 7, 0), (32, 1.0, 0.4, 7, 1), (64, 0.6585, 0.55, 9, 2), (32, 3.0, 0.3, 1, 3),
             (32, 0.2, 0.9, 2, 4), (96, 0.8, 0.35, 5, 5)]
    max_steps = 1500
    L, q, J, seed, ids = (np.array(x) for x in zip(*pairs))
    got = coalescence_times(L, q, J, seed.astype(np.uint64), ids.astype(np.uint32), max_steps)
    for k, (l_, q_, j_, s_, i_) in enumerate(pairs):
        assert int(got[k]) == _oracle_T(orc, l_, q_, j_, s_, i_, max_steps), pairs[k]
    assert np.any(got <= max_steps)


def test_coalescence_not_reached_is_reported():
    # deep in the ordered phase on a 64x64 torus the chains do not meet quickly
    got = coalescence_times([64], [2.0], [1.5], [3], [0], 20)
    assert int(got[0]) == 21


# ---- checkerboard heat bath of the square-lattice Ising model (Section 3.2)

from paper_1908_07341_gb300.lattice import checkerboard_run  # noqa: E402
from tests.gpu_util import from_device_plane  # noqa: E402


@pytest.mark.parametrize("L,J,n", [(32, 0.44, 3), (64, 0.3, 40), (96, -0.5, 7), (64, 0.0, 5), (32, 9.0, 4),
                                   (1024, 0.4406868, 3)])
def test_checkerboard_run_matches_oracle(orc, L, J, n):
    s = random_spins(L, seed=L + 11, p_up=0.55)
    plane = to_device_plane(s, L, "bitpack")
    got_obs = checkerboard_run(plane, L, J, seed=13, lattice_id=2, t0=5, n_steps=n).cpu().numpy()
    ref = s.copy()
    ref_obs = orc.checkerboard_run(ref, L, J, 13, 2, 5, n)
    assert np.array_equal(from_device_plane(plane, L, "bitpack"), ref)
    assert np.array_equal(got_obs, ref_obs)


def test_checkerboard_16384_full_plane_against_oracle(orc):
    """The benchmark's checkerboard workload (16384^2, J = 0.44, seed 3, random
    start) in the benchmark's launch configuration (specialised kernels):
    after 6 GPU steps, step t = 6 is recomputed by the oracle from the GPU's
    state over the whole plane and both (M, C_nn) sums compared; then the
    benchmark's diagonal sums (lags 1..16) of that plane."""
    L, J, seed = 16384, 0.44, 3
    shk.specialize(2)
    try:
        plane = shk.alloc_plane(L, "bitpack")
        shk.init_plane("bitpack", plane, L, "random", init_seed=3)
        checkerboard_run(plane, L, J, seed, 0, 0, 6, obs=False)
        ref = from_device_plane(plane, L, "bitpack")
        rows = checkerboard_run(plane, L, J, seed, 0, 6, 1).cpu().numpy()
        ref_rows = orc.checkerboard_run(ref, L, J, seed, 0, 6, 1)
        assert np.array_equal(rows, ref_rows)
        assert np.array_equal(from_device_plane(plane, L, "bitpack"), ref)
        assert shk.specialize_status()["failed"] == 0
        # the benchmark's diagonal sums on the same plane
        lags = [1, 2, 4, 8, 16]
        assert np.array_equal(diag_correlations(plane, L, lags).cpu().numpy(), orc.diag_correlations(ref, L, lags))
    finally:
        shk.specialize(1)


def test_checkerboard_resume_and_lattice_ids(orc):
    L = 64
    s = random_spins(L, seed=5, p_up=0.5)
    a, b = to_device_plane(s, L, "bitpack"), to_device_plane(s, L, "bitpack")
    checkerboard_run(a, L, 0.5, 21, 0, 0, 12, obs=False)
    checkerboard_run(b, L, 0.5, 21, 0, 0, 5, obs=False)
    checkerboard_run(b, L, 0.5, 21, 0, 5, 7, obs=False)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    c = to_device_plane(s, L, "bitpack")
    checkerboard_run(c, L, 0.5, 21, 1, 0, 12, obs=False)
    assert not torch.equal(a, c)
    ref = s.copy()
    orc.checkerboard_run(ref, L, 0.5, 21, 1, 0, 12)
    assert np.array_equal(from_device_plane(c, L, "bitpack"), ref)


# ---- coupling from the past and checkerboard coalescence

from paper_1908_07341_gb300.lattice import cftp  # noqa: E402
import paper_1908_07341_gb300 as _pkg  # noqa: E402,F401


def _oracle_T_checkerboard(orc, L, J, seed, lat_id, max_steps):
    top, bot = np.ones(L * L, np.int8), -np.ones(L * L, np.int8)
    for t in range(max_steps):
        orc.checkerboard_run(top, L, J, seed, lat_id, t, 1)
        orc.checkerboard_run(bot, L, J, seed, lat_id, t, 1)
        if np.array_equal(top, bot):
            return t + 1
    return max_steps + 1


def test_checkerboard_coalescence_times_match_oracle(orc):
    pairs = [(32, 0.3, 4, 0), (32, 0.4, 4, 1), (64, 0.35, 2, 2), (32, 0.1, 9, 3)]
    L, J, seed, ids = (np.array(x) for x in zip(*pairs))
    got = coalescence_times(L, 0.0, J, seed.astype(np.uint64), ids.astype(np.uint32), 1000,
                            dynamics="checkerboard")
    for k, (l_, j_, s_, i_) in enumerate(pairs):
        assert int(got[k]) == _oracle_T_checkerboard(orc, l_, j_, s_, i_, 1000), pairs[k]


def _unpack(samples, L):
    from paper_1908_07341_gb300 import unpack_bits
    return unpack_bits(samples[: L * L // 8], L).reshape(-1)


@pytest.mark.parametrize("dyn", ["shaken", "checkerboard"])
def test_cftp_matches_oracle(orc, dyn):
    """k and the time-0 sample of every pair equal the oracle's coupling from
    the past; pairs of different L share one launch."""
    if dyn == "shaken":
        pairs = [(32, 0.8, 0.35, 5, 3), (32, 1.0, 0.3, 6, 0), (64, 0.6585, 0.5, 2, 7), (32, 0.3, 0.2, 1, 1)]
    else:
        pairs = [(32, 0.0, 0.3, 5, 3), (32, 0.0, 0.35, 6, 0), (64, 0.0, 0.25, 2, 7)]
    L, q, J, seed, ids = (np.array(x) for x in zip(*pairs))
    ks, samples = cftp(L, q, J, seed.astype(np.uint64), ids.astype(np.uint32), k_max=14, dynamics=dyn)
    host = samples.cpu().numpy()
    code = orc.SHAKEN if dyn == "shaken" else orc.CHECKERBOARD
    for i, (l_, q_, j_, s_, id_) in enumerate(pairs):
        k_ref, s_ref = orc.cftp(code, int(l_), float(q_), float(j_), int(s_), int(id_), k_max=14)
        assert int(ks[i]) == k_ref, pairs[i]
        assert k_ref >= 0
        assert np.array_equal(_unpack(host[i], int(l_)), s_ref), pairs[i]


def test_cftp_reports_no_coalescence():
    ks, samples = cftp([64], [2.0], [1.5], [3], [0], k_max=3)
    assert int(ks[0]) == -1
    assert int(samples.to(torch.int64).sum()) == 0


def test_philox_peak_kernel_computes_the_generator(orc):
    """The measurement kernel runs the half-steps' Philox4x32-10: its XOR fold
    over (block, thread, call) equals the oracle's fold of the same counters
    (i, w, 0, 0) under the key 0x0123456789ABCDEF."""
    from paper_1908_07341_gb300 import _lib
    blocks, iters = 2, 3
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.check(_lib.lib().shk_philox_peak(blocks, iters, out.data_ptr(), None))
    torch.cuda.synchronize()
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    ref = 0
    for w in range(blocks * 256):
        for i in range(iters):
            r = orc.philox4x32_10([i, w, 0, 0], key)
            ref ^= int(r[0]) ^ int(r[1]) ^ int(r[2]) ^ int(r[3])
    assert int(out.item()) & 0xFFFFFFFF == ref
