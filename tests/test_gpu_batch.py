"""Batched lattices (one persistent kernel, graph-replayed) against single-
lattice runs: every lattice of a batch must follow exactly the trajectory
shk_run gives it, and the batch statistics must equal the sums of the single
runs' per-step observables (all integers, compared exactly).  The single-
lattice path is itself checked against the oracle in test_gpu_parity."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import paper_1908_07341_gb300 as shk
from paper_1908_07341_gb300.batch import Batch, derived, stats_from_observables
from paper_1908_07341_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _single(L, q, J, seed, lat_id, init_seed, n):
    lat = shk.Lattice(int(L), "bitpack").set_seed(int(seed), int(lat_id)).set_params(float(q), float(J))
    lat.init("random", init_seed=init_seed)
    obs = lat.run(n, obs=True).cpu().numpy()
    return obs, lat.read_spins(0), lat.read_spins(1)


MIXED = dict(L=[32, 64, 96, 128, 160, 256, 32, 64],
             q=[1.0, 0.5, 0.6585, 3.0, 0.05, 0.8, 2.0, 0.3],
             J=[0.25, 0.5, 0.6585, 0.44, 1.7, 0.6, 0.1, 1.2],
             seed=[1, 2, 3, 4, 5, 6, 7, 2 ** 40 + 9],
             lattice_id=[0, 1, 2, 3, 4, 5, 6, 7])


@pytest.mark.parametrize("k,block,tile_sites", [(1, 256, 1 << 18), (3, 128, 1024), (8, 256, 4096),
                                                (8, 512, 1 << 18), (4, 256, 2048)])
def test_batch_equals_single_lattice_runs(k, block, tile_sites):
    n, burn = 24, 10
    b = Batch(**MIXED).configure(k, block, tile_sites).init("random", init_seed=11)
    b.run(n, burn_in=burn)
    assert b.step == n
    stats, last = b.read_stats(), b.read_observables()
    for i in range(b.n):
        obs, s, t = _single(MIXED["L"][i], MIXED["q"][i], MIXED["J"][i], MIXED["seed"][i],
                            MIXED["lattice_id"][i], 11, n)
        assert np.array_equal(b.read_spins(i, 0), s), i
        assert np.array_equal(b.read_spins(i, 1), t), i
        assert np.array_equal(last[i], obs[-1]), i
        assert np.array_equal(stats[i], stats_from_observables(obs[burn:])), i


def test_batch_large_tiles_and_resume():
    """L = 1024 and 2048 cut into several tiles; 16 + 16 steps equal 32."""
    cfg = dict(L=[2048, 1024, 512], q=[1.0, 0.7, 0.5], J=[0.35, 0.6, 0.9], seed=[3, 3, 3],
               lattice_id=[10, 11, 12])
    b = Batch(**cfg).configure(8, 256, 1 << 17).init("random", init_seed=3)
    b.run(16, burn_in=0)
    b.run(16, burn_in=0)
    stats, last = b.read_stats(), b.read_observables()
    for i in range(3):
        obs, s, t = _single(cfg["L"][i], cfg["q"][i], cfg["J"][i], 3, cfg["lattice_id"][i], 3, 32)
        assert np.array_equal(b.read_spins(i, 0), s), i
        assert np.array_equal(b.read_spins(i, 1), t), i
        assert np.array_equal(last[i], obs[-1])
        assert np.array_equal(stats[i], stats_from_observables(obs))


def test_phase_diagram_subset_matches_single_runs():
    """A 64-lattice slice of the phase-diagram workload (uneven L, its own
    (q, J) cell each) with burn-in, checked lattice by lattice."""
    w = workloads.phase_diagram_batch()
    idx = np.arange(0, 1024, 16)
    cfg = {key: w[key][idx] for key in ("L", "q", "J", "seed", "lattice_id")}
    n, burn = 40, 20
    b = Batch(**cfg).configure(8, 256, 1 << 18).init("random", init_seed=w["init_seed"])
    b.run(n, burn_in=burn)
    stats = b.read_stats()
    for i in range(0, len(idx), 4):
        obs, s, _ = _single(cfg["L"][i], cfg["q"][i], cfg["J"][i], cfg["seed"][i], cfg["lattice_id"][i],
                            w["init_seed"], n)
        assert np.array_equal(stats[i], stats_from_observables(obs[burn:])), i
        assert np.array_equal(b.read_spins(i, 0), s), i
    d = derived(stats, cfg["L"], cfg["q"], cfg["J"])
    assert np.all(np.abs(d["m"]) <= 1) and np.all(d["chi"] >= 0)


def test_batch_argument_errors():
    b = Batch(L=[64, 32], q=[1.0, 1.0], J=[0.3, 0.3], seed=[1, 1], lattice_id=[0, 1])
    with pytest.raises(shk.ShakenError):
        b.configure(0, 256, 1 << 18)
    with pytest.raises(shk.ShakenError):
        b.configure(8, 100, 1 << 18)
    b.configure(8, 256, 1 << 18).init("up")
    with pytest.raises(shk.ShakenError):
        b.run(12)          # not a multiple of steps_per_launch
    with pytest.raises(ValueError):
        Batch(L=[33], q=[1.0], J=[0.3], seed=[1], lattice_id=[0])


def test_full_phase_diagram_batch_spot_checks(orc):
    """The whole 1024-lattice phase-diagram batch in a launch shape of the
    kind the benchmark uses (8 steps per launch, 256 threads, 2^18-site
    tiles): after 96 steps, the oracle takes the GPU's sigma of sampled
    lattices (the largest and smallest included) and runs steps 96..103
    itself; sigma and tau after the GPU's next launch must agree bit for bit."""
    w = workloads.phase_diagram_batch()
    b = Batch(w["L"], w["q"], w["J"], w["seed"], w["lattice_id"]).configure(8, 256, 1 << 18)
    b.init("random", init_seed=w["init_seed"])
    b.run(96)
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.choice(len(w["L"]), size=10, replace=False).tolist()
                        + [int(np.argmax(w["L"])), int(np.argmin(w["L"]))]))
    before = {i: b.read_spins(i, 0).reshape(-1).astype(np.int8) for i in sample}
    b.run(8)
    for i in sample:
        L = int(w["L"][i])
        sigma = before[i].copy()
        tau = np.zeros(L * L, np.int8)
        orc.run(sigma, tau, L, float(w["q"][i]), float(w["J"][i]), int(w["seed"][i]), int(w["lattice_id"][i]),
                96, 8, want_obs=False)
        assert np.array_equal(b.read_spins(i, 0).reshape(-1), sigma), i
        assert np.array_equal(b.read_spins(i, 1).reshape(-1), tau), i


@pytest.mark.parametrize("k,block,tile_sites", [(4, 512, 1 << 18), (2, 256, 1 << 17)])
def test_phase_diagram_batch_against_the_oracle(orc, k, block, tile_sites):
    """The batched configuration at its full size, in the launch shape the
    benchmark's autotuner picks (4 steps per launch, 512 threads, 2^18-site
    tiles) and in a second one with smaller tiles and more halo rows (2
    steps, 256 threads, 2^17 sites): all 1024 lattices of the phase diagram
    (L log-uniform in {32, ..., 2048}, one (q, J) cell each) run 56 steps
    with a 16-step burn-in.
    - Every lattice with L <= 256 is recomputed by the oracle from its random
      start: final sigma and tau, the five sums of the last step, and the
      eleven exact statistics of the 40 measured steps (Eq. fact applied to
      each lattice on its own, as in the task-parallel runs of the paper).
    - 48 larger lattices (16 each of L = 512, 1024, 2048, whose tiles carry
      recomputed halo rows) are spot-checked over one launch: the oracle takes
      the GPU's sigma after step 56 and runs the next launch's k steps; sigma,
      tau and the last step's sums must agree after the GPU's next launch.
    The oracle runs on every host core (its C calls release the interpreter
    lock); it shares no code with the GPU path."""
    w = workloads.phase_diagram_batch()
    n, burn = 56, 16
    b = Batch(w["L"], w["q"], w["J"], w["seed"], w["lattice_id"]).configure(k, block, tile_sites)
    b.init("random", init_seed=w["init_seed"])
    b.run(n, burn_in=burn)
    stats, last = b.read_stats(), b.read_observables()
    small = [i for i in range(len(w["L"])) if w["L"][i] <= 256]
    assert len(small) > 500

    def cfg(i):
        return (int(w["L"][i]), float(w["q"][i]), float(w["J"][i]), int(w["seed"][i]), int(w["lattice_id"][i]))

    def full(i):
        L, q, J, seed, lid = cfg(i)
        s = orc.init_plane(L, orc.INIT_RANDOM, w["init_seed"], lid, 0)
        t = orc.init_plane(L, orc.INIT_RANDOM, w["init_seed"], lid, 1)
        return i, s, t, orc.run(s, t, L, q, J, seed, lid, 0, n)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        for i, s, t, obs in ex.map(full, small):
            assert np.array_equal(b.read_spins(i, 0).reshape(-1), s), i
            assert np.array_equal(b.read_spins(i, 1).reshape(-1), t), i
            assert np.array_equal(last[i], obs[-1]), i
            assert np.array_equal(stats[i], stats_from_observables(obs[burn:])), i

    rng = np.random.default_rng(56)
    large = []
    for L in (512, 1024, 2048):
        idx = np.flatnonzero(w["L"] == L)
        large += rng.choice(idx, size=min(16, idx.size), replace=False).tolist()
    assert len(large) >= 32
    before = {i: b.read_spins(i, 0).reshape(-1).copy() for i in large}
    b.run(k)
    last = b.read_observables()

    def spot(i):
        L, q, J, seed, lid = cfg(i)
        s = before[i].copy()
        t = np.zeros(L * L, np.int8)
        return i, s, t, orc.run(s, t, L, q, J, seed, lid, n, k)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        for i, s, t, obs in ex.map(spot, large):
            assert np.array_equal(b.read_spins(i, 0).reshape(-1), s), i
            assert np.array_equal(b.read_spins(i, 1).reshape(-1), t), i
            assert np.array_equal(last[i], obs[-1]), i

