"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer spins and integer observable sums must agree exactly (bit for bit);
the floating-point values derived from them (magnetisation, pair energy) are
then equal too, which the tests check to 1e-12 relative.  Sizes span several
thread blocks and ragged tails; full-size configurations are checked on
sampled rows that the oracle recomputes from the GPU's own state, which the
counter-based random numbers make exact.
"""
import numpy as np
import pytest
import torch

import paper_1908_07341_gb300 as shk
from tests.gpu_util import from_device_plane, to_device_plane
from tests.inputs import random_spins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    build.build()
    shk.lib()
    torch.cuda.set_device(0)


def _orc_obs_halfstep(orc, half, src, dst, L):
    """Expected fused reductions of one half-step (see shk_halfstep)."""
    out = np.zeros(5, dtype=np.int64)
    if half == 0:
        o = orc.observables(src, dst, L)      # sigma = src, tau = dst
        out[1], out[4] = o[1], o[4]
    else:
        o = orc.observables(dst, src, L)      # sigma = dst, tau = src
        out[0], out[2], out[3] = o[0], o[2], o[3]
    return out


HALFSTEP_CASES = (
    [("int8", L) for L in (2, 3, 5, 31, 32, 33, 64, 96, 100, 257, 288)]
    + [("bitpack", L) for L in (32, 64, 96, 128, 288, 1024)]
)


@pytest.mark.parametrize("layout,L", HALFSTEP_CASES)
@pytest.mark.parametrize("half", [0, 1])
def test_halfstep_matches_oracle(orc, layout, L, half):
    q, J, seed, lat_id = 0.9, 0.45, 0xDEADBEEFCAFE, 7
    T = orc.thresholds(q, J)
    src = random_spins(L, seed=L * 10 + half)
    for hs in (2 * 3 + half, 2 * 1000 + half):
        d_src = to_device_plane(src, L, layout)
        d_dst = to_device_plane(np.ones(L * L, np.int8), L, layout)
        acc = torch.zeros(5, dtype=torch.int64, device="cuda")
        shk.halfstep(layout, half, d_src, d_dst, L, T, seed, lat_id, hs, acc)
        got = from_device_plane(d_dst, L, layout)
        want = orc.halfstep(half, src, L, T, seed, lat_id, hs)
        assert np.array_equal(got, want)
        assert np.array_equal(acc.cpu().numpy(), _orc_obs_halfstep(orc, half, src, want, L))


@pytest.mark.parametrize("layout,L", [("int8", 3), ("int8", 100), ("int8", 257), ("int8", 64),
                                      ("bitpack", 64), ("bitpack", 1024)])
@pytest.mark.parametrize("kind", ["up", "down", "random"])
def test_init_matches_oracle(orc, layout, L, kind):
    plane = shk.alloc_plane(L, layout)
    shk.init_plane(layout, plane, L, kind, init_seed=12345, lattice_id=3, plane_index=1)
    code = {"up": orc.INIT_ALL_UP, "down": orc.INIT_ALL_DOWN, "random": orc.INIT_RANDOM}[kind]
    want = orc.init_plane(L, code, 12345, 3, 1)
    assert np.array_equal(from_device_plane(plane, L, layout), want)


def test_strict_comparison_ties_on_the_gpu(orc):
    """A site uniform equal to its threshold is not below it (Algorithm 3's
    strict rand() < p).  Complement-symmetric tables are set to a site's own
    uniform (and one above it), for + and for - sites, and the GPU must agree
    with the oracle; the tie drives the lazy comparison through all 32 planes."""
    L, seed, lat_id, hs = 64, 99, 3, 6
    for base_spin in (1, -1):
        src = np.full(L * L, base_spin, dtype=np.int8)
        r = orc.block_uniforms(seed, hs, 1, lat_id, 0)
        for p in (0, 13, 31):
            for delta in (0, 1):
                U = int(r[p]) + delta if base_spin > 0 else (2 ** 32 - int(r[p])) + delta
                U = min(max(U, 1), 2 ** 32 - 1)
                T = np.array([2 ** 32 - U] * 3 + [U] * 3, dtype=np.uint32)
                for layout in ("bitpack", "int8"):
                    d_src = to_device_plane(src, L, layout)
                    d_dst = to_device_plane(src, L, layout)
                    shk.halfstep(layout, 0, d_src, d_dst, L, T, seed, lat_id, hs)
                    want = orc.halfstep(0, src, L, T, seed, lat_id, hs)
                    got = from_device_plane(d_dst, L, layout)
                    assert np.array_equal(got, want)


def _run_oracle(orc, L, q, J, seed, init_kind, init_seed, steps, lat_id=0):
    s = orc.init_plane(L, init_kind, init_seed, lat_id, 0)
    t = orc.init_plane(L, init_kind, init_seed, lat_id, 1)
    obs = orc.run(s, t, L, q, J, seed, lat_id, 0, steps)
    return s, t, obs


def test_config_64_int8_1000_steps(orc):
    """64x64 int8, all-up, q=1.0, J=0.25, seed 1, 1000 steps: every step's
    int64 observables and the spins at checkpoints equal the oracle."""
    L, q, J, seed = 64, 1.0, 0.25, 1
    lat = shk.Lattice(L, "int8").set_seed(seed, 0).set_params(q, J).init("up", init_seed=seed)
    s = orc.init_plane(L, orc.INIT_ALL_UP, seed, 0, 0)
    t = orc.init_plane(L, orc.INIT_ALL_UP, seed, 0, 1)
    done = 0
    for chunk in (1, 2, 7, 90, 900):
        got_obs = lat.run(chunk, obs=True).cpu().numpy()
        want_obs = orc.run(s, t, L, q, J, seed, 0, done, chunk)
        done += chunk
        assert np.array_equal(got_obs, want_obs), done
        assert np.array_equal(lat.read_spins(0).reshape(-1), s), done
        assert np.array_equal(lat.read_spins(1).reshape(-1), t), done
    assert done == 1000
    # FP64 values derived from the exact sums
    m_gpu = got_obs[:, 0] / (L * L)
    H_gpu = -(J * got_obs[:, 3] + q * got_obs[:, 2])
    m_ref = want_obs[:, 0] / (L * L)
    H_ref = -(J * want_obs[:, 3] + q * want_obs[:, 2])
    assert np.allclose(m_gpu, m_ref, rtol=1e-12, atol=0) and np.allclose(H_gpu, H_ref, rtol=1e-12, atol=0)


def test_config_1024_bitpack(orc):
    """1024x1024 bit-packed, random start (p=1/2, init seed 2), q=J=0.5, seed 2:
    the first 20 steps in full, then one-step spot checks at t = 1000, 5000 and
    10000 from the GPU's own state at t-1, plus the observables of those steps."""
    L, q, J, seed = 1024, 0.5, 0.5, 2
    lat = shk.Lattice(L, "bitpack").set_seed(seed, 0).set_params(q, J).init("random", init_seed=2)
    got = lat.run(20, obs=True).cpu().numpy()
    s, t, want = _run_oracle(orc, L, q, J, seed, orc.INIT_RANDOM, 2, 20)
    assert np.array_equal(got, want)
    assert np.array_equal(lat.read_spins(0).reshape(-1), s)
    assert np.array_equal(lat.read_spins(1).reshape(-1), t)
    for target in (1000, 5000, 10000):
        lat.run(target - 1 - lat.step)
        s = lat.read_spins(0).reshape(-1).copy()
        t = lat.read_spins(1).reshape(-1).copy()
        got = lat.run(1, obs=True).cpu().numpy()
        want = orc.run(s, t, L, q, J, seed, 0, target - 1, 1)
        assert np.array_equal(got, want), target
        assert np.array_equal(lat.read_spins(0).reshape(-1), s), target
        assert np.array_equal(lat.read_spins(1).reshape(-1), t), target


@pytest.mark.parametrize("layout", ["bitpack", "int8"])
@pytest.mark.parametrize("specialize", [2, 0])
def test_config_16384_sampled(orc, layout, specialize):
    """16384x16384 (2.7e8 sites per sublattice), random start, q=1.0, J=0.35,
    seed 3, in the launch configuration of the benchmark (the default sweep
    variant, compiled with the thresholds as constants; and, for comparison,
    the generic kernel): step t = 2 is checked on sampled row bands, including
    both wrap-around rows, and step t = 1999 (the 2000th) on the whole sigma
    and tau planes, each recomputed by the oracle from the GPU's state at t-1;
    the step's five sums are checked against the oracle on the whole plane."""
    from paper_1908_07341_gb300 import tune
    L, q, J, seed = 16384, 1.0, 0.35, 3
    T = orc.thresholds(q, J)
    before = tune.get_variant(layout)
    tune.set_variant(layout, 0)
    shk.specialize(specialize)
    try:
        _check_16384(orc, layout, L, q, J, seed, T)
        if specialize:
            st = shk.specialize_status()
            assert st["failed"] == 0 and st["compiled"] >= 1, st
    finally:
        shk.specialize(1)
        tune.set_variant(layout, before)


def _check_16384(orc, layout, L, q, J, seed, T):
    lat = shk.Lattice(L, layout).set_seed(seed, 0).set_params(q, J).init("random", init_seed=3)
    for target in (2, 1999):
        # the whole torus at the last step of the 2000-step run
        bands = [(0, 3), (5000, 5003), (16381, 16384)] if target < 1999 else [(0, L)]
        lat.run(target - lat.step, obs=True)
        s_prev = lat.read_spins(0).reshape(-1).copy()
        obs = lat.run(1, obs=True).cpu().numpy()[0]
        s_new = lat.read_spins(0).reshape(-1)
        t_new = lat.read_spins(1).reshape(-1)
        for r0, r1 in bands:
            t_ref = orc.halfstep(0, s_prev, L, T, seed, 0, 2 * target, r0, r1)
            assert np.array_equal(t_ref[r0 * L:r1 * L], t_new[r0 * L:r1 * L]), (target, r0)
            s_ref = orc.halfstep(1, t_new, L, T, seed, 0, 2 * target + 1, r0, r1)
            assert np.array_equal(s_ref[r0 * L:r1 * L], s_new[r0 * L:r1 * L]), (target, r0)
        assert np.array_equal(obs, orc.observables(s_new, t_new, L)), target


def _plane_rows(plane, layout, L, rows):
    """int8 +/-1 copies of some rows of a device plane (only those rows leave the device)."""
    idx = torch.tensor(rows, dtype=torch.long, device=plane.device)
    if layout == "bitpack":
        words = plane[: L * L // 8].view(torch.int32).view(L, L // 32).index_select(0, idx).cpu().numpy()
        bits = (words.view(np.uint32)[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1
        vals = (2 * bits.astype(np.int8) - 1).reshape(len(rows), L)
    else:
        vals = plane[: L * L].view(torch.int8).view(L, L).index_select(0, idx).cpu().numpy()
    return {r: vals[k] for k, r in enumerate(rows)}


@pytest.mark.parametrize("layout,L", [("bitpack", 65536), ("int8", 32768)])
def test_largest_planes_sampled(orc, layout, L):
    """Planes far beyond the benchmark's 16384^2: 2^32 sites per sublattice
    bit-packed (block indices up to 2^27) and 2^30 int8, in the default launch
    shape.  After one step from a random start, the oracle recomputes step 1
    (Eqs. leftTrans / rightTrans) from the GPU's own state on row bands that
    include both wrap-around rows and the middle of the torus.  Only the
    needed rows are copied to the host; the oracle gets them in a full-size
    array that is otherwise never touched."""
    q, J, seed, lid = 0.9, 0.4, 11, 5
    T = orc.thresholds(q, J)
    lat = shk.Lattice(L, layout).set_seed(seed, lid).set_params(q, J).init("random", init_seed=3)
    lat.run(1)
    bands = [(0, 2), (L // 2 - 1, L // 2 + 1), (L - 2, L)]
    around = sorted({r % L for r0, r1 in bands for r in range(r0 - 1, r1 + 1)})
    sigma0 = _plane_rows(lat.plane(0), layout, L, around)
    lat.run(1)
    tau1 = _plane_rows(lat.plane(1), layout, L, around)
    sigma1 = _plane_rows(lat.plane(0), layout, L, around)
    src = np.zeros(L * L, dtype=np.int8)
    dst = np.zeros(L * L, dtype=np.int8)
    for r, v in sigma0.items():
        src[r * L:(r + 1) * L] = v
    for r0, r1 in bands:
        orc.halfstep(0, src, L, T, seed, lid, 2, r0, r1, dst=dst)
        for r in range(r0, r1):
            assert np.array_equal(dst[r * L:(r + 1) * L], tau1[r]), ("tau", r)
    for r, v in tau1.items():
        src[r * L:(r + 1) * L] = v
    for r0, r1 in bands:
        orc.halfstep(1, src, L, T, seed, lid, 3, r0, r1, dst=dst)
        for r in range(r0, r1):
            assert np.array_equal(dst[r * L:(r + 1) * L], sigma1[r]), ("sigma", r)
    lat.close()


@pytest.mark.parametrize("L", [64, 96, 288, 1024])
def test_layouts_give_identical_trajectories(L):
    """The random numbers depend on the site index only, so the bit-packed and
    int8 layouts follow the same trajectory."""
    res = []
    for layout in ("bitpack", "int8"):
        lat = shk.Lattice(L, layout).set_seed(77, 5).set_params(0.8, 0.6).init("random", init_seed=9)
        obs = lat.run(25, obs=True).cpu().numpy()
        res.append((obs, lat.read_spins(0), lat.read_spins(1)))
    for a, b in zip(*res):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("layout,L", [("int8", 5), ("int8", 257), ("bitpack", 64), ("bitpack", 288)])
def test_checkpoint_resume(layout, L):
    """State after step t-1 plus (q, J, seed, lattice id, t) fixes the future:
    12 steps in one call equal 7 + 5 steps, and equal a restart from spins
    written back through the host at step 7."""
    def fresh():
        return shk.Lattice(L, layout).set_seed(2024, 1).set_params(0.7, 0.55).init("random", init_seed=4)
    a = fresh()
    full = a.run(12, obs=True).cpu().numpy()
    b = fresh()
    first = b.run(7, obs=True).cpu().numpy()
    s7, t7 = b.read_spins(0), b.read_spins(1)
    second = b.run(5, obs=True).cpu().numpy()
    assert np.array_equal(full, np.concatenate([first, second]))
    c = fresh()
    c.write_spins(0, s7)
    c.write_spins(1, t7)
    c.step = 7
    assert c.step == 7
    third = c.run(5, obs=True).cpu().numpy()
    assert np.array_equal(third, second)
    assert np.array_equal(c.read_spins(0), a.read_spins(0))


@pytest.mark.parametrize("layout,L", [("int8", 64), ("bitpack", 1024), ("int8", 257)])
def test_observable_ring_keeps_last_step(layout, L):
    a = shk.Lattice(L, layout).set_seed(5, 0).set_params(1.1, 0.3).init("random", init_seed=1)
    rows = a.run(9, obs=True).cpu().numpy()
    assert np.array_equal(a.read_observables(), rows[-1])
    b = shk.Lattice(L, layout).set_seed(5, 0).set_params(1.1, 0.3).init("random", init_seed=1)
    b.run(4)
    b.run(5)
    assert np.array_equal(b.read_observables(), rows[-1])


def test_monotone_coupling_at_scale():
    """Section 3.2: top (all +) and bottom (all -) chains with the same random
    numbers stay ordered site by site at every step (bottom & ~top == 0 on the
    bit-packed words) on a 1024x1024 torus."""
    L = 1024
    top = shk.Lattice(L, "bitpack").set_seed(11, 0).set_params(0.6585, 0.6585).init("up")
    bot = shk.Lattice(L, "bitpack").set_seed(11, 0).set_params(0.6585, 0.6585).init("down")
    for _ in range(60):
        top.run(1)
        bot.run(1)
        for p in (0, 1):
            bad = torch.bitwise_and(bot.plane(p), torch.bitwise_not(top.plane(p)))
            assert int(bad.count_nonzero()) == 0


def test_run_argument_errors():
    lat = shk.Lattice(64, "bitpack")
    with pytest.raises(shk.ShakenError) as e:
        lat.run(3)
    assert e.value.status == -4
    lat.set_params(1.0, 0.2).set_seed(1, 0).init("up")
    assert lat.run(0) is None
    lat.step = 2 ** 31 - 2
    with pytest.raises(shk.ShakenError):
        lat.run(5)
    with pytest.raises(shk.ShakenError):
        lat.read_observables()


@pytest.mark.parametrize("layout,L", [("bitpack", 96), ("bitpack", 128), ("bitpack", 192), ("bitpack", 1024),
                                      ("bitpack", 2048), ("bitpack", 4096), ("int8", 64),
                                      ("int8", 288), ("int8", 1024)])
def test_every_sweep_variant_draws_the_same_spins(orc, layout, L):
    """The launch-shape variants the autotuner chooses from differ only in
    speed: each one reproduces the oracle's half-step exactly."""
    from paper_1908_07341_gb300 import tune
    q, J, seed, lat_id = 0.7, 0.6, 99, 4
    T = orc.thresholds(q, J)
    src = random_spins(L, seed=L + 1)
    before = tune.get_variant(layout)
    try:
        for v in range(len(tune.variant_names(layout))):
            tune.set_variant(layout, v)
            for half in (0, 1):
                d_src = to_device_plane(src, L, layout)
                d_dst = to_device_plane(np.ones(L * L, np.int8), L, layout)
                acc = torch.zeros(5, dtype=torch.int64, device="cuda")
                shk.halfstep(layout, half, d_src, d_dst, L, T, seed, lat_id, 2 * 5 + half, acc)
                want = orc.halfstep(half, src, L, T, seed, lat_id, 2 * 5 + half)
                assert np.array_equal(from_device_plane(d_dst, L, layout), want), (v, half)
                assert np.array_equal(acc.cpu().numpy(), _orc_obs_halfstep(orc, half, src, want, L))
    finally:
        tune.set_variant(layout, before)
