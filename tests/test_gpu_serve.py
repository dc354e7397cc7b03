"""Serving with continuous batching: jobs admitted at different ticks share
launches, yet each job's result (exact statistics, last observables, hash of
the final sigma) is the same alone, in the mix, and as a single-lattice run."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import paper_1908_07341_gb300 as shk
from paper_1908_07341_gb300.batch import stats_from_observables
from paper_1908_07341_gb300.serve import Server, fnv1a64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    build.build()
    torch.cuda.set_device(0)


# the serving benchmark's launch shape (bench.py, bench_serving)
BENCH_SHAPE = dict(steps_per_launch=2, launches_per_tick=16, block_threads=256, tile_sites=1 << 17)

JOBS = [dict(L=64, q=1.0, J=0.25, seed=1, lattice_id=0, n_steps=37, burn_in=10),
        dict(L=128, q=0.5, J=0.5, seed=2, lattice_id=1, n_steps=16, burn_in=0),
        dict(L=32, q=3.0, J=0.44, seed=3, lattice_id=2, n_steps=5, burn_in=2),
        dict(L=256, q=0.6585, J=0.6585, seed=4, lattice_id=3, n_steps=50, burn_in=25),
        dict(L=96, q=0.05, J=1.7, seed=5, lattice_id=4, n_steps=23, burn_in=0, init="up"),
        dict(L=512, q=1.2, J=0.3, seed=6, lattice_id=5, n_steps=19, burn_in=9),
        dict(L=160, q=0.8, J=0.6, seed=2 ** 40 + 7, lattice_id=6, n_steps=64, burn_in=63),
        dict(L=64, q=2.0, J=0.1, seed=8, lattice_id=7, n_steps=1, burn_in=0, init="down")]


def _single(job):
    lat = shk.Lattice(job["L"], "bitpack").set_seed(job["seed"], job["lattice_id"])
    lat.set_params(job["q"], job["J"]).init(job.get("init", "random"), init_seed=job.get("init_seed", 0))
    obs = lat.run(job["n_steps"], obs=True).cpu().numpy()
    raw = lat.plane(0)[: job["L"] * job["L"] // 8].cpu().numpy().tobytes()
    return stats_from_observables(obs[job["burn_in"]:]), obs[-1], fnv1a64(raw)


def _run_all(server, jobs, arrive_at_tick):
    ids, results, tick = {}, {}, 0
    while len(results) < len(jobs):
        for i, j in enumerate(jobs):
            if arrive_at_tick[i] == tick:
                ids[server.submit(**j)] = i
        server.tick()
        for r in server.poll():
            results[ids[r["job_id"]]] = r
        tick += 1
        assert tick < 10_000
    return [results[i] for i in range(len(jobs))]


@pytest.mark.parametrize("k,launches", [(1, 1), (2, 4), (3, 5), (8, 2)])
def test_each_job_same_alone_and_in_the_mix(k, launches):
    mixed = Server(max_slots=16, arena_bytes=64 << 20).configure(steps_per_launch=k, launches_per_tick=launches)
    res_mix = _run_all(mixed, JOBS, [0, 0, 1, 1, 2, 3, 3, 5])
    for i, j in enumerate(JOBS):
        alone = Server(max_slots=2, arena_bytes=8 << 20).configure(steps_per_launch=k, launches_per_tick=launches)
        (r_alone,) = _run_all(alone, [j], [0])
        want_stats, want_last, want_hash = _single(j)
        for r in (res_mix[i], r_alone):
            assert r["status"] == 0 and r["steps_done"] == j["n_steps"]
            assert np.array_equal(r["stats"], want_stats), i
            assert np.array_equal(r["last_obs"], want_last), i
            assert r["sigma_hash"] == want_hash, i


def test_admission_waits_for_memory_and_results_do_not_change():
    # a 110 kB budget: the 512^2 job (three 32 kB planes and its scratch) must
    # wait until the jobs admitted before it have finished
    srv = Server(max_slots=16, arena_bytes=64 << 20, hbm_budget=110_000).configure(steps_per_launch=2,
                                                                                  launches_per_tick=4)
    ids = [srv.submit(**j) for j in JOBS]
    saw_waiting = False
    results = {}
    for _ in range(10_000):
        active, pending = srv.tick()
        saw_waiting |= pending > 0 and active > 0
        assert srv.stats()["used_bytes"] <= 110_000
        for r in srv.poll():
            results[r["job_id"]] = r
        if len(results) == len(JOBS):
            break
    assert saw_waiting
    for jid, j in zip(ids, JOBS):
        want_stats, want_last, want_hash = _single(j)
        assert np.array_equal(results[jid]["stats"], want_stats)
        assert results[jid]["sigma_hash"] == want_hash


def test_queue_limit_cancel_and_validation():
    srv = Server(max_slots=1, arena_bytes=8 << 20).configure(steps_per_launch=2, launches_per_tick=2,
                                                             max_pending=2)
    a = srv.submit(**JOBS[3])
    b = srv.submit(**JOBS[0])
    with pytest.raises(shk.ShakenError) as e:
        srv.submit(**JOBS[1])
    assert e.value.status == -5                       # SHK_EBUSY, never blocks
    srv.tick()                                        # a admitted, b waits
    srv.cancel(b)                                     # cancel a queued job
    srv.tick()
    srv.cancel(a)                                     # cancel a running job
    got = {r["job_id"]: r for r in srv.poll()}
    assert got[a]["status"] == -7 and got[b]["status"] == -7
    assert 0 < got[a]["steps_done"] < JOBS[3]["n_steps"]
    with pytest.raises(shk.ShakenError):
        srv.submit(L=33, q=1.0, J=0.3, seed=1, lattice_id=0, n_steps=5)
    with pytest.raises(shk.ShakenError):
        srv.submit(L=64, q=float("nan"), J=0.3, seed=1, lattice_id=0, n_steps=5)
    with pytest.raises(shk.ShakenError):
        srv.cancel(12345)
    assert srv.tick() == (0, 0)


def test_deadlines_expire_queued_and_running_jobs():
    """One slot, 4 steps per tick.  Job a (deadline 3 ticks) is still running
    at the end of tick 3 and is retired with SHK_ETIMEOUT after 12 steps, its
    statistics and sigma hash those of the first 12 steps of a single-lattice
    run; job b (deadline 2) expires in the queue without running; job c (no
    deadline) then runs to completion unaffected."""
    srv = Server(max_slots=1, arena_bytes=8 << 20).configure(steps_per_launch=2, launches_per_tick=2)
    ja = dict(L=64, q=1.0, J=0.3, seed=1, lattice_id=0, n_steps=40, burn_in=4, init_seed=7)
    jb = dict(L=64, q=0.5, J=0.4, seed=2, lattice_id=1, n_steps=8, burn_in=0, init_seed=7)
    jc = dict(L=32, q=2.0, J=0.44, seed=3, lattice_id=2, n_steps=8, burn_in=0, init_seed=7)
    a = srv.submit(**ja, deadline_ticks=3)
    b = srv.submit(**jb, deadline_ticks=2)
    c = srv.submit(**jc)
    got = {}
    for _ in range(20):
        srv.tick()
        got.update({r["job_id"]: r for r in srv.poll()})
        if len(got) == 3:
            break
    assert got[a]["status"] == -6 and got[a]["steps_done"] == 12 and got[a]["done_tick"] == 3
    stats, last, h = _single(dict(ja, n_steps=12))
    assert np.array_equal(got[a]["stats"], stats) and np.array_equal(got[a]["last_obs"], last)
    assert got[a]["sigma_hash"] == h
    assert got[b]["status"] == -6 and got[b]["steps_done"] == 0 and got[b]["done_tick"] == 2
    assert got[c]["status"] == 0 and got[c]["steps_done"] == 8 and got[c]["admit_tick"] == 3
    stats, last, h = _single(jc)
    assert np.array_equal(got[c]["stats"], stats) and got[c]["sigma_hash"] == h


def test_result_log_lines(tmp_path):
    import json
    log = tmp_path / "results.jsonl"
    srv = Server(max_slots=2, arena_bytes=8 << 20, result_log=str(log)).configure(steps_per_launch=2,
                                                                                 launches_per_tick=2)
    ids = [srv.submit(**JOBS[2]), srv.submit(**JOBS[7])]
    got = []
    for _ in range(10):
        srv.tick()
        got += srv.poll()
        if len(got) == 2:
            break
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert sorted(r["job_id"] for r in lines) == sorted(ids)
    for r in lines:
        want = next(g for g in got if g["job_id"] == r["job_id"])
        assert r["stats"] == want["stats"].tolist() and r["sigma_hash"] == want["sigma_hash"]


def test_serving_stream_jobs_spot_checked_against_the_oracle(orc):
    """Jobs of the serving workload itself (the first 300 jobs of the Poisson
    stream, L log-uniform in [64, 4096], steps log-uniform in [10^3, 10^5]) in
    the benchmark's launch shape (2 steps per launch, 16 launches per tick,
    256 threads, 2^17-site tiles), all in one mix; the smallest ones (the
    oracle finishes them in seconds) are recomputed by the oracle: exact
    statistics after burn-in, last-step sums and the hash of the final sigma."""
    from paper_1908_07341_gb300 import workloads
    from paper_1908_07341_gb300.lattice import pack_bits
    w = workloads.serving_stream(n_jobs=300)
    jobs = w["jobs"]
    cost = [j["L"] ** 2 * j["n_steps"] for j in jobs]
    check = sorted(range(len(jobs)), key=lambda i: cost[i])[:4]
    mix = sorted(set(check) | set(range(0, 300, 30)))        # the checked jobs among larger ones
    srv = Server(max_slots=64, arena_bytes=1 << 30).configure(**BENCH_SHAPE)
    ids = {srv.submit(**jobs[i]): i for i in mix}
    got = {}
    for _ in range(100_000):
        srv.tick()
        got.update({ids[r["job_id"]]: r for r in srv.poll()})
        if len(got) == len(mix):
            break
    assert len(got) == len(mix)
    for i in check:
        j = jobs[i]
        L = j["L"]
        s = orc.init_plane(L, orc.INIT_RANDOM, j["init_seed"], j["lattice_id"], 0)
        t = orc.init_plane(L, orc.INIT_RANDOM, j["init_seed"], j["lattice_id"], 1)
        obs = orc.run(s, t, L, j["q"], j["J"], j["seed"], j["lattice_id"], 0, j["n_steps"])
        assert got[i]["status"] == 0 and got[i]["steps_done"] == j["n_steps"]
        assert np.array_equal(got[i]["stats"], stats_from_observables(obs[j["burn_in"]:])), i
        assert np.array_equal(got[i]["last_obs"], obs[-1]), i
        assert got[i]["sigma_hash"] == fnv1a64(pack_bits(s).view(np.uint8).tobytes()), i


def test_serving_stream_mixed_jobs_against_the_oracle(orc):
    """40 jobs of the serving workload (the first 400 jobs of the Poisson
    stream: L log-uniform in [64, 4096], q, J uniform, steps log-uniform in
    [10^3, 10^5], seed 5, lattice id = job index) in one mix, in the
    benchmark's launch shape (2 steps per launch, 16 launches per tick, 256
    threads, 2^17-site tiles):
    - 32 jobs spread over the whole range of L (the largest included) are
      spot-checked in flight after a tick of that shape: the test reads each
      job's sigma and step count between ticks (shk_server_read_job), the
      server runs one tick of a single launch (2 steps, every job in the mix
      advancing), sigma and tau are read again, and the oracle runs the same
      two steps from the GPU's sigma; the checked jobs are then cancelled;
    - the 8 cheapest jobs run to completion and are recomputed by the oracle
      from their random starts: the exact statistics after burn-in, the last
      step's sums and the hash of the final sigma."""
    from paper_1908_07341_gb300 import workloads
    from paper_1908_07341_gb300.lattice import pack_bits
    w = workloads.serving_stream(n_jobs=400)
    jobs = w["jobs"]
    cost = np.array([j["L"] ** 2 * j["n_steps"] for j in jobs], dtype=np.float64)
    full = np.argsort(cost)[:8].tolist()
    rest = sorted((i for i in range(len(jobs)) if i not in full), key=lambda i: (jobs[i]["L"], i))
    spot = sorted({rest[int(round(x))] for x in np.linspace(0, len(rest) - 1, 32)})
    assert len(spot) == 32 and max(jobs[i]["L"] for i in spot) == max(j["L"] for j in jobs)
    k = BENCH_SHAPE["steps_per_launch"]
    assert all(jobs[i]["n_steps"] > 32 + k for i in spot)
    srv = Server(max_slots=64, arena_bytes=1 << 30).configure(**BENCH_SHAPE)
    ids = {srv.submit(**jobs[i]): i for i in sorted(set(full) | set(spot))}
    job_id = {i: jid for jid, i in ids.items()}
    got = {}
    srv.tick()                                      # admits all 40; 32 steps of every job
    got.update({ids[r["job_id"]]: r for r in srv.poll()})
    before = {i: srv.read_job(job_id[i], jobs[i]["L"], 0) for i in spot}
    srv.configure(**dict(BENCH_SHAPE, launches_per_tick=1))
    srv.tick()
    got.update({ids[r["job_id"]]: r for r in srv.poll()})
    after = {i: (srv.read_job(job_id[i], jobs[i]["L"], 0), srv.read_job(job_id[i], jobs[i]["L"], 1)[0])
             for i in spot}
    srv.configure(**BENCH_SHAPE)
    for i in spot:
        srv.cancel(job_id[i])

    def spot_check(i):
        j = jobs[i]
        (s0, t0) = before[i]
        s = s0.reshape(-1).copy()
        t = np.zeros_like(s)
        obs = orc.run(s, t, j["L"], j["q"], j["J"], j["seed"], j["lattice_id"], t0, k)
        return i, t0, s, t, obs

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        for i, t0, s, t, obs in ex.map(spot_check, spot):
            (s1, t1), tau1 = after[i]
            assert t0 == 32 and t1 == 32 + k, (i, t0, t1)
            assert np.array_equal(s1.reshape(-1), s), i
            assert np.array_equal(tau1.reshape(-1), t), i
    for _ in range(100_000):
        if all(i in got and got[i]["status"] == 0 for i in full):
            break
        srv.tick()
        got.update({ids[r["job_id"]]: r for r in srv.poll()})
    for i in spot:
        assert got[i]["status"] == -7, i          # SHK_ECANCELLED
    for i in full:
        j = jobs[i]
        L = j["L"]
        s = orc.init_plane(L, orc.INIT_RANDOM, j["init_seed"], j["lattice_id"], 0)
        t = orc.init_plane(L, orc.INIT_RANDOM, j["init_seed"], j["lattice_id"], 1)
        obs = orc.run(s, t, L, j["q"], j["J"], j["seed"], j["lattice_id"], 0, j["n_steps"])
        assert got[i]["status"] == 0 and got[i]["steps_done"] == j["n_steps"]
        assert np.array_equal(got[i]["stats"], stats_from_observables(obs[j["burn_in"]:])), i
        assert np.array_equal(got[i]["last_obs"], obs[-1]), i
        assert got[i]["sigma_hash"] == fnv1a64(pack_bits(s).view(np.uint8).tobytes()), i
    srv.close()


def test_read_job_refuses_unknown_jobs_and_short_buffers():
    srv = Server(max_slots=2, arena_bytes=8 << 20).configure(steps_per_launch=2, launches_per_tick=1)
    jid = srv.submit(**JOBS[0])
    with pytest.raises(shk.ShakenError):
        srv.read_job(jid, 64)                   # queued, not running yet
    srv.tick()
    s, steps = srv.read_job(jid, 64)
    assert steps == 2 and s.shape == (64, 64)
    from paper_1908_07341_gb300 import _lib
    import ctypes
    small = np.zeros(64 * 64 - 1, dtype=np.int8)
    n = ctypes.c_uint64()
    assert _lib.lib().shk_server_read_job(srv._h, jid, 0, small.ctypes.data, small.size,
                                          ctypes.byref(n)) == _lib.ENOMEM
    assert _lib.lib().shk_server_read_job(srv._h, jid + 99, 0, small.ctypes.data, 1 << 20,
                                          ctypes.byref(n)) == _lib.EINVAL
    srv.close()

