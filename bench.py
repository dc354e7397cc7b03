"""Benchmark of the shaken-dynamics hot path on GB300.

Workload (one GPU): one 16384 x 16384 bit-packed torus pair (2.7e8 sites per
sublattice), random start (init seed 3), q = 1.0, J = 0.35, Philox seed 3,
2000 full steps with the five observable sums of every step.  One benchmark
step is 100 full steps through shk_run (2 * 16384^2 * 100 = 5.4e10 site
updates); the default 20 timed steps cover the 2000 full steps once.

Metric: site updates per second (one site update = one spin redrawn in one
half-step).  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica lattice (lattice id =
rank) with no data exchange; the timed region is bracketed by barriers and the
slowest rank's time is used.  --impl reference times the single-threaded CPU
oracle (the paper gives no runnable code) on a bounded row band of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L = 16384
Q, J = 1.0, 0.35
SEED = 3
INIT_SEED = 3
STEPS_PER_BENCH_STEP = 100
TOTAL_STEPS = 2000
L2_FLUSH_BYTES = 256 << 20
WORKLOAD = ("shaken dynamics, one 16384x16384 bit-packed torus pair, random start, "
            "q=1.0, J=0.35, seed 3, 2000 full steps, per-step M/E/C_nn sums")
METRIC = "site updates/s at L=16384 (bit-packed, 2000 full steps)"
UNIT = "site updates/s"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
KERNEL_LAUNCHES = 2 * STEPS_PER_BENCH_STEP     # the half-step launches of one benchmark step
FALLBACK_HBM_GBS = 6800.0
SM_COUNT = 152
MAX_SM_MHZ = 2070.0


def replica_lattice_id(rank: int) -> int:
    """Replicas only: rank r advances its own lattice with lattice id r (the
    third Philox counter word), so the ranks' random streams never overlap and
    no data crosses between ranks."""
    return int(rank)


def whole_job_rate(local_ms: float, units_per_rank: float, dist=None, device=None) -> tuple[float, float]:
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time (a MAX all-reduce of the per-rank milliseconds).
    Returns (rate per second, max milliseconds)."""
    import torch

    world = 1
    ms = float(local_ms)
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units_per_rank / (ms / 1e3), ms


def _peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", MAX_SM_MHZ)), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, MAX_SM_MHZ, "fallback"


def _expected_algorithmic_ops_per_block():
    """Integer ops one 32-site block needs under the lazy most-significant-bit-
    first comparison, assuming per-block early exit: P = number of random
    planes until all 32 sites are decided (each plane settles a site with
    probability 1/2, so P(P <= b) = (1 - 2^-b)^32, P <= 32), ceil(P/4) Philox
    calls of 40 ops (10 rounds x (2 wide multiplies + 2 three-input xors)) and
    6 bitwise ops per plane."""
    e_planes = 0.0
    e_calls = 0.0
    prev = 0.0
    for b in range(1, 33):
        cdf = (1.0 - 2.0 ** -b) ** 32 if b < 32 else 1.0
        pb = cdf - prev
        prev = cdf
        e_planes += b * pb
        e_calls += ((b + 3) // 4) * pb
    return 40.0 * e_calls + 6.0 * e_planes, e_planes, e_calls


def measure_philox_peak(dev, stream, iters: int = 16384, reps: int = 5) -> float:
    """Philox4x32-10 calls per second of the library's own generator with no
    memory traffic (shk_philox_peak: 8 CTAs of 256 threads per SM, independent
    calls per thread), best of `reps` launches timed with events on `stream`."""
    import torch

    from paper_1908_07341_gb300 import _lib
    so = _lib.lib()
    out = torch.zeros(1, dtype=torch.int32, device=dev)
    blocks = torch.cuda.get_device_properties(dev).multi_processor_count * 8
    _lib.check(so.shk_philox_peak(blocks, iters, out.data_ptr(), stream.cuda_stream))
    best = float("inf")
    for _ in range(reps):
        s_ev = torch.cuda.Event(enable_timing=True)
        e_ev = torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        _lib.check(so.shk_philox_peak(blocks, iters, out.data_ptr(), stream.cuda_stream))
        e_ev.record(stream)
        torch.cuda.synchronize()
        best = min(best, s_ev.elapsed_time(e_ev))
    return blocks * 256.0 * iters / (best / 1e3)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ["timestamp", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"shk_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, window=None):
        """Stops sampling; keeps the samples whose timestamp falls inside
        window = (t0, t1) in time.time() seconds (all samples if none do)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < len(self.FIELDS):
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(parts[1]), float(parts[2]),
                                 [n for n, v in zip(names, parts[5:9]) if v.lower() == "active"]))
                except ValueError:
                    continue
        os.unlink(self.path)
        inside = [r for r in rows if window and window[0] - 0.05 <= r[0] <= window[1] + 0.05]
        use = inside or rows
        reasons = sorted({n for r in use for n in r[3]})
        return {"sm_mhz": statistics.median(r[1] for r in use) if use else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "samples": len(use), "in_timed_window": bool(inside), "reasons": reasons}


# ----------------------------------------------------------------- oracle timing

def _oracle_band_worker(shm_names, side, r0, r1, q, jj, seed, warmup, steps, barrier, results):
    """One host core of the oracle timing: half-steps A and B on rows [r0, r1)
    of the shared sigma / tau planes, with a barrier after each half-step (B
    reads the tau rows its neighbours wrote)."""
    import numpy as np
    from multiprocessing import shared_memory

    from oracle import oracle as orc

    shm = [shared_memory.SharedMemory(name=n) for n in shm_names]
    sigma = np.ndarray((side * side,), dtype=np.int8, buffer=shm[0].buf)
    tau = np.ndarray((side * side,), dtype=np.int8, buffer=shm[1].buf)
    T = orc.thresholds(q, jj)
    barrier.wait()
    t0 = 0.0
    for t in range(warmup + steps):
        if t == warmup:
            barrier.wait()
            t0 = time.perf_counter()
        orc.halfstep(0, sigma, side, T, seed, 0, 2 * t, r0, r1, dst=tau)
        barrier.wait()
        orc.halfstep(1, tau, side, T, seed, 0, 2 * t + 1, r0, r1, dst=sigma)
        barrier.wait()
    results.put(time.perf_counter() - t0)
    del sigma, tau
    for m in shm:
        m.close()


def _oracle_rate_all_cores(steps: int, warmup: int = 0):
    """Site updates/s of the CPU oracle on every host core: the 16384^2 torus
    split into row bands, one process per core (spawned), all bands advanced
    by `steps` full steps after `warmup` untimed ones.  Returns (rate,
    seconds, units, cores)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    import numpy as np
    from oracle import oracle as orc

    orc.lib()                                   # build once, before the workers load it
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    n = L * L
    shm = [shared_memory.SharedMemory(create=True, size=n) for _ in range(2)]
    try:
        sigma = np.ndarray((n,), dtype=np.int8, buffer=shm[0].buf)
        rng = np.random.default_rng(SEED)
        for r0 in range(0, L, 1024):                # random start, filled in slices
            sl = slice(r0 * L, (r0 + 1024) * L)
            sigma[sl] = rng.integers(0, 2, size=1024 * L, dtype=np.int8) * 2 - 1
        del sigma
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(cores, timeout=600)   # a worker that dies breaks it for the others
        results = ctx.Queue()
        bands = [(L * k // cores, L * (k + 1) // cores) for k in range(cores)]
        procs = [ctx.Process(target=_oracle_band_worker,
                             args=([m.name for m in shm], L, r0, r1, Q, J, SEED, warmup, steps, barrier, results))
                 for r0, r1 in bands]
        for p in procs:
            p.start()
        import queue
        times = []
        while len(times) < cores:
            try:
                times.append(results.get(timeout=5))
            except queue.Empty:
                if not any(p.is_alive() for p in procs) and results.empty():
                    raise RuntimeError("an oracle worker process failed")
        for p in procs:
            p.join()
        dt = max(times)
        units = steps * 2 * L * L
        return units / dt, dt, units, cores
    finally:
        for m in shm:
            m.close()
            m.unlink()


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return 0
    value, dt, units, cores = _oracle_rate_all_cores(args.steps, args.warmup)
    sample = (f"{args.steps} full steps (half-steps A and B) of the whole 16384x16384 torus after "
              f"{args.warmup} untimed ones, row bands on {cores} host cores (one spawned process each)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "L": L, "layout": "int8 (oracle)", "cores": cores},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm

def run_ours(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch

    from paper_1908_07341_gb300 import build as libbuild

    libbuild.build()
    import paper_1908_07341_gb300 as shk

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    # the sweeps run in their specialised form (thresholds compiled in); the
    # one-time compile happens at the first warm-up launch, before any timing
    shk.specialize(shk.lattice.SPECIALIZE_BLOCKING)
    compile_s = {}
    window = [0.0, 0.0]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def bench_layout(layout: str, steps: int, warmup: int, with_e2e: bool):
        from paper_1908_07341_gb300 import tune
        tune.autotune(layout, L)                 # launch shape for this size (untimed)
        lat = shk.Lattice(L, layout, device=dev, stream=stream)
        lat.set_seed(SEED, replica_lattice_id(rank)).set_params(Q, J).init("random", init_seed=INIT_SEED)
        obs = torch.empty((STEPS_PER_BENCH_STEP, shk.NOBS), dtype=torch.int64, device=dev)
        t_c = time.perf_counter()
        lat.run(1)                                # compiles the specialised sweeps (untimed)
        torch.cuda.synchronize()
        compile_s[layout] = time.perf_counter() - t_c
        for _ in range(warmup):
            lat.run(STEPS_PER_BENCH_STEP, obs)
        # the timed steps start the configured run from its initial state:
        # 20 benchmark steps are exactly the 2000 full steps of the workload
        lat.init("random", init_seed=INIT_SEED)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        barrier()
        window[0] = time.time()
        for k in range(steps):
            flush.fill_(k & 0xFF)               # evict L2 between timed steps (not timed)
            starts[k].record(stream)
            lat.run(STEPS_PER_BENCH_STEP, obs)
            ends[k].record(stream)
        barrier()
        window[1] = time.time()
        ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
        e2e = None
        if with_e2e:
            # End to end through the public API with host buffers: upload sigma
            # from pinned host memory, run, read the step's observables back.
            raw = L * L // 8 if layout == "bitpack" else L * L
            host_sigma = torch.empty(raw, dtype=torch.uint8, pin_memory=True)
            lat.download_plane(0, host_sigma)
            host_obs = torch.empty((STEPS_PER_BENCH_STEP, shk.NOBS), dtype=torch.int64, pin_memory=True)
            torch.cuda.synchronize()
            barrier()
            e_start = torch.cuda.Event(enable_timing=True)
            e_end = torch.cuda.Event(enable_timing=True)
            n_e2e = max(1, steps // 2)
            t_host0 = time.perf_counter()
            e_start.record(stream)
            for _ in range(n_e2e):
                lat.upload_plane(0, host_sigma)
                lat.run(STEPS_PER_BENCH_STEP, obs)
                host_obs.copy_(obs, non_blocking=True)
                stream.synchronize()
            e_end.record(stream)
            barrier()
            e_ms = e_start.elapsed_time(e_end)
            host_ms = 1e3 * (time.perf_counter() - t_host0)
            e2e = {"ms": max(e_ms, host_ms), "steps": n_e2e, "h2d": raw, "d2h": int(obs.numel() * 8)}
        # dominant kernel: the two half-step sweeps as they run inside shk_run,
        # back to back on the launching stream (same planes, grid and launch
        # overlap), one event pair around KERNEL_LAUNCHES launches after a
        # warm-up; the mean launch time is their elapsed time / KERNEL_LAUNCHES
        T = shk.thresholds(Q, J)
        src, dst = lat.plane(0), lat.plane(1)
        acc = torch.zeros(shk.NOBS, dtype=torch.int64, device=dev)

        def launches(n, hs0):
            for rep in range(n):
                half = rep & 1
                a, b = (src, dst) if half == 0 else (dst, src)
                shk.halfstep(layout, half, a, b, L, T, SEED, rank, hs0 + rep, acc, stream)

        launches(4, 2 * 4000)
        torch.cuda.synchronize()
        flush.fill_(1)
        s_ev = torch.cuda.Event(enable_timing=True)
        e_ev = torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        launches(KERNEL_LAUNCHES, 2 * 4002)
        e_ev.record(stream)
        torch.cuda.synchronize()
        kern = s_ev.elapsed_time(e_ev) / KERNEL_LAUNCHES
        lat.close()
        return ms, e2e, kern

    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)                          # nvidia-smi start-up
    t_wall0 = time.perf_counter()
    ms, e2e, kern_ms = bench_layout("bitpack", args.steps, args.warmup, with_e2e=True)
    wall = time.perf_counter() - t_wall0
    from paper_1908_07341_gb300 import tune as _tune
    variant_bp = _tune.variant_names("bitpack")[_tune.get_variant("bitpack")]
    clocks = sampler.stop(tuple(window)) if sampler else None

    units_per_step = 2 * L * L * STEPS_PER_BENCH_STEP
    value, ms = whole_job_rate(ms, units_per_step * args.steps, dist, dev)
    e2e_value, _ = whole_job_rate(e2e["ms"], units_per_step * e2e["steps"], dist, dev)

    # secondary line: the int8 layout on the same workload (fewer steps)
    ms8, _, kern8_ms = bench_layout("int8", max(2, args.steps // 5), 1, with_e2e=False)
    variant_i8 = _tune.variant_names("int8")[_tune.get_variant("int8")]
    value8, _ = whole_job_rate(ms8, units_per_step * max(2, args.steps // 5), dist, dev)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    hbm_gbs, sm_max, peak_kind = _peaks()
    ops_block, e_planes, e_calls = _expected_algorithmic_ops_per_block()
    philox_cps = measure_philox_peak(dev, stream)
    sites_per_launch = L * L
    blocks_per_launch = sites_per_launch / 32
    kern_s = kern_ms / 1e3
    # Binding unit: the integer multiply pipe.  A Philox4x32-10 call is 20
    # wide (32 x 32 -> 64-bit) products; a 32-site block needs E[calls]
    # calls under the lazy comparison (e_calls ~ 2.0), so the algorithmic
    # products per launch are 20 * e_calls * blocks.  Peak from unit counts
    # and clock: 152 SMs x 4 partitions x 8 wide products per clock (16 lanes,
    # two passes each) x max SM clock; the measured Philox peak (products/s of
    # shk_philox_peak) is reported beside it.
    prod_per_launch = 20.0 * e_calls * blocks_per_launch
    prod_achieved = prod_per_launch / kern_s / 1e12
    prod_peak = SM_COUNT * 4 * 8 * sm_max * 1e6 / 1e12
    prod_measured = philox_cps * 20.0 / 1e12
    alu_ops = ops_block * blocks_per_launch
    alu_peak = SM_COUNT * 128 * sm_max * 1e6 / 1e12          # Tops/s, issue slots at max clock
    alu_achieved = alu_ops / kern_s / 1e12
    hbm_bytes_bp = 2 * sites_per_launch / 8                  # read 1 bit + write 1 bit per site
    hbm_bytes_i8 = 2 * sites_per_launch                      # read 1 byte + write 1 byte per site
    traffic = _load_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "L": L, "layout": "bitpack", "q": Q, "J": J, "seed": SEED,
                   "full_steps_per_bench_step": STEPS_PER_BENCH_STEP,
                   "site_updates_per_bench_step": units_per_step,
                   "l2": "flushed between timed steps (256 MiB write); both planes (64 MiB) fit in L2 "
                         "during a step", "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e["h2d"],
                "d2h_bytes_per_step": e2e["d2h"]},
        "gpu_launches": args.steps * (2 * STEPS_PER_BENCH_STEP + 1),
        "roofline": {
            "bound": "alu", "achieved": prod_achieved, "peak": prod_peak,
            "unit": "T wide integer products/s", "frac": prod_achieved / prod_peak,
            "traffic": traffic.get(f"bitpack:{variant_bp}"),
            "kernel": f"bit-packed half-step A/B, launch shape {variant_bp}", "kernel_ms": kern_ms,
            "kernel_ms_basis": f"one event pair around {KERNEL_LAUNCHES} back-to-back launches (overlapped "
                               f"as in shk_run) / {KERNEL_LAUNCHES}",
            "peak_basis": f"{SM_COUNT} SMs x 4 partitions x 8 wide products per clock x {sm_max:.0f} MHz "
                          "(derived); the binding pipe of Philox4x32-10",
            "algorithmic_products_per_launch": prod_per_launch,
            "algorithmic_basis": "20 wide products per Philox call x expected calls per 32-site block "
                                 f"({e_calls:.4f}) x {blocks_per_launch:.0f} blocks",
            "measured_peak": prod_measured, "frac_of_measured": prod_achieved / prod_measured,
            "philox": {"calls_per_s": philox_cps, "expected_calls_per_32_sites": e_calls,
                       "ceiling": philox_cps * 32.0 / e_calls,
                       "achieved": sites_per_launch / kern_s, "unit": "site updates/s",
                       "frac": sites_per_launch / kern_s / (philox_cps * 32.0 / e_calls),
                       "basis": "measured shk_philox_peak x 32 sites / expected Philox calls per block"},
            "issue": {"achieved": alu_achieved, "peak": alu_peak, "unit": "Tops/s", "frac": alu_achieved / alu_peak,
                      "algorithmic_ops_per_32_sites": ops_block,
                      "peak_basis": f"{SM_COUNT} SMs x 128 issue lanes x {sm_max:.0f} MHz (derived)"},
            "hbm": {"achieved": hbm_bytes_bp / kern_s / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                    "frac": hbm_bytes_bp / kern_s / 1e9 / hbm_gbs, "peak_kind": peak_kind},
            "check": {"kernel_ms_x_launches": kern_ms * KERNEL_LAUNCHES, "ms_per_step": ms / args.steps},
        },
        "int8": {"value": value8, "unit": UNIT, "steps": max(2, args.steps // 5),
                 "roofline": {"bound": "hbm", "achieved": hbm_bytes_i8 / (kern8_ms / 1e3) / 1e9,
                              "peak": hbm_gbs, "unit": "GB/s",
                              "frac": hbm_bytes_i8 / (kern8_ms / 1e3) / 1e9 / hbm_gbs,
                              "traffic": traffic.get(f"int8:{variant_i8}"), "kernel_ms": kern8_ms,
                              "kernel_ms_basis": f"one event pair around {KERNEL_LAUNCHES} back-to-back "
                                                 "launches / their number",
                              "kernel": f"int8 half-step A/B, launch shape {variant_i8}",
                              "peak_kind": peak_kind}},
        "clocks": clocks,
        "wall_s_bitpack": wall,
        "specialized": {"status": {k: v for k, v in shk.specialize_status().items() if k != "log"},
                        "first_launch_s": compile_s,
                        "note": "sweeps compiled at run time with the (q, J) thresholds as constants, "
                                "once per (launch shape, thresholds): the autotuner's and the first "
                                "launch's compiles (compile_s, host seconds) come before the warm-up "
                                "steps"},
    }
    def spec_status():
        return {k: v for k, v in shk.specialize_status().items() if k != "log"}

    if not args.no_batched:
        line["batched"] = bench_batched(dev, stream)
        line["specialized"]["after_batched"] = spec_status()
    if not args.no_section3:
        line["section3"] = bench_section3(dev, stream)
        line["l_sweep"] = bench_l_sweep(dev, stream)
        line["specialized"]["after_section3"] = spec_status()
    if not args.no_serving:      # last: the longest leg, which heats the GPU most
        line["serving"] = bench_serving(dev, stream, n_jobs=args.serving_jobs, sub_jobs=args.serving_sub_jobs)
    if world == 1 and not args.no_cpu_baseline:
        rate, secs, units, cores = _oracle_rate_all_cores(steps=4, warmup=1)
        line["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"4 full steps of the whole 16384x16384 torus after 1 untimed step ({units} site "
                      f"updates, {secs:.1f} s), row bands on {cores} host cores, one spawned oracle "
                      f"process each"}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def bench_batched(dev, stream, plain_steps: int = 100):
    """The phase-diagram batch (1024 lattices, uneven L, one (q, J) cell each,
    10^4 steps, burn-in 5000) in the persistent graph-replayed kernel, and the
    same lattices advanced by plain per-lattice shk_run calls on one stream for
    plain_steps steps.  Returns a dict for the JSON line."""
    import numpy as np
    import torch

    import paper_1908_07341_gb300 as shk
    from paper_1908_07341_gb300 import tune, workloads
    from paper_1908_07341_gb300.batch import Batch

    w = workloads.phase_diagram_batch()
    L = w["L"]
    units_per_step = float((2 * L.astype(np.float64) ** 2).sum())
    b = Batch(w["L"], w["q"], w["J"], w["seed"], w["lattice_id"], device=dev, stream=stream)
    tuned = tune.autotune_batch(b, init_kind="random", init_seed=w["init_seed"])
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    b.run(w["steps"], burn_in=w["burn_in"])
    e.record(stream)
    torch.cuda.synchronize()
    batched_ms = s.elapsed_time(e)
    stats = b.read_stats()
    assert int(stats[:, 10].min()) == w["steps"] - w["burn_in"]
    b.close()
    # plain per-lattice launches of the same lattices on one stream, in the
    # library's default specialisation mode (compiles in the background, at
    # most two queued): with one (q, J) table per lattice, blocking compiles
    # would take minutes and fill the compile cache, so most of these
    # lattices run the generic sweeps, as they would for a user
    mode_before = shk.specialize()
    shk.specialize(shk.lattice.SPECIALIZE_BACKGROUND)
    lats = []
    for i in range(len(L)):
        lat = shk.Lattice(int(L[i]), "bitpack", device=dev, stream=stream)
        lat.set_seed(int(w["seed"][i]), int(w["lattice_id"][i])).set_params(float(w["q"][i]), float(w["J"][i]))
        lat.init("random", init_seed=w["init_seed"])
        lats.append(lat)
    for lat in lats:
        lat.run(2)
    torch.cuda.synchronize()
    s.record(stream)
    for lat in lats:
        lat.run(plain_steps)
    e.record(stream)
    torch.cuda.synchronize()
    plain_ms = s.elapsed_time(e)
    for lat in lats:
        lat.close()
    shk.wait_specialized()
    shk.specialize(mode_before)
    batched_rate = units_per_step * w["steps"] / (batched_ms / 1e3)
    plain_rate = units_per_step * plain_steps / (plain_ms / 1e3)
    return {"workload": "1024 lattices, L log-uniform in {32..2048} (seeded), 32x32 (q,J) grid "
                        "q in [0.05,3], J in [0.05,1.5], random starts, 10^4 steps, burn-in 5000",
            "value": batched_rate, "unit": UNIT, "ms": batched_ms, "steps": w["steps"],
            "site_updates": units_per_step * w["steps"],
            "plain_value": plain_rate, "plain_steps_timed": plain_steps, "plain_ms": plain_ms,
            "speedup_vs_plain": batched_rate / plain_rate, "tuned": list(tuned["best"]),
            "launches": w["steps"] // tuned["best"][0]}


def bench_section3(dev, stream) -> dict:
    """Throughput of the Section 3 kernels, each on a synthetic workload of
    the paper's shape, timed with events on `stream` after a warm-up:
    the checkerboard heat bath on the 16384^2 torus, coalescence times and
    coupling from the past on 32x32 pairs near the critical curve (the
    paper's box), and the diagonal sums of a 16384^2 plane."""
    import numpy as np
    import torch

    import paper_1908_07341_gb300 as shk
    from paper_1908_07341_gb300.experiments import critical_J
    from paper_1908_07341_gb300.lattice import (cftp, checkerboard_run, coalescence_times, diag_correlations)

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        s_ev = torch.cuda.Event(enable_timing=True)
        e_ev = torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        for _ in range(reps):
            out = fn()
        e_ev.record(stream)
        torch.cuda.synchronize()
        return s_ev.elapsed_time(e_ev) / reps, out

    out = {}
    Lc = 16384
    plane = shk.alloc_plane(Lc, "bitpack", device=dev)
    shk.init_plane("bitpack", plane, Lc, "random", init_seed=INIT_SEED, stream=stream)
    n_cb = 20
    ms, _ = timed(lambda: checkerboard_run(plane, Lc, 0.44, SEED, 0, 0, n_cb, obs=True, stream=stream))
    out["checkerboard"] = {"workload": f"{Lc}x{Lc} square-lattice heat bath, J=0.44, {n_cb} steps with (M, C_nn)",
                           "value": Lc * Lc * n_cb / (ms / 1e3), "unit": UNIT, "ms": ms,
                           "gpu_launches": 3 * n_cb}
    lags = [1, 2, 4, 8, 16]
    ms, _ = timed(lambda: diag_correlations(plane, Lc, lags, stream=stream), reps=10)
    out["diag_correlations"] = {"workload": f"{Lc}x{Lc} plane, lags {lags}", "ms": ms,
                                "value": (Lc * Lc / 8) / (ms / 1e3) / 1e9, "unit": "GB/s of plane read"}
    del plane
    n_pairs, L = 1024, 32
    q = np.repeat(np.array([0.5, 1.0, 1.5, 2.0]), n_pairs // 4)
    J = critical_J(q) - 0.05
    ids = np.arange(n_pairs, dtype=np.uint32)
    max_steps = 1 << 16
    ms, T = timed(lambda: coalescence_times(np.full(n_pairs, L), q, J, np.uint64(SEED), ids, max_steps,
                                            device=dev, stream=stream))
    steps = np.minimum(T.astype(np.float64), max_steps).sum()
    out["coalescence"] = {"workload": f"{n_pairs} pairs of {L}x{L} tori at J = J_c(q) - 0.05, q in "
                                      "{0.5, 1, 1.5, 2}", "ms": ms, "pair_steps": steps,
                          "value": steps * 4 * L * L / (ms / 1e3), "unit": UNIT + " (both chains)"}
    Jg = critical_J(q) - 0.1
    ms, (ks, _) = timed(lambda: cftp(np.full(n_pairs, L), q, Jg, np.uint64(SEED), ids, k_max=18,
                                      device=dev, stream=stream))
    steps = float(np.sum(2.0 ** (ks[ks >= 0].astype(np.float64) + 1) - 1))
    out["cftp"] = {"workload": f"{n_pairs} perfect samples of {L}x{L} tori at J = J_c(q) - 0.1",
                   "ms": ms, "samples_per_s": float((ks >= 0).sum()) / (ms / 1e3),
                   "value": steps * 4 * L * L / (ms / 1e3), "unit": UNIT + " (both chains, all attempts)"}
    return out


def bench_l_sweep(dev, stream) -> dict:
    """The paper's own benchmark shape (Section 4, time per update against L):
    J = 0.44, q = 0.66, one bit-packed lattice of side L = 32 .. 16384 (powers
    of two), random start; time per full step through shk_run, timed with
    events on `stream` over enough steps to last a few milliseconds."""
    import torch

    import paper_1908_07341_gb300 as shk

    rows = []
    for e in range(5, 15):
        side = 1 << e
        n = int(max(20, min(4000, (1 << 29) // (side * side))))
        lat = shk.Lattice(side, "bitpack", device=dev, stream=stream).set_seed(SEED, 0).set_params(0.66, 0.44)
        lat.init("random", init_seed=INIT_SEED)
        lat.run(min(n, 50))
        s_ev = torch.cuda.Event(enable_timing=True)
        e_ev = torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        lat.run(n)
        e_ev.record(stream)
        torch.cuda.synchronize()
        ms = s_ev.elapsed_time(e_ev)
        row = {"L": side, "steps": n, "us_per_step": 1e3 * ms / n,
               "site_updates_per_s": 2.0 * side * side * n / (ms / 1e3)}
        lat.close()
        if side <= 4096:
            # the same lattice as a batch of one: k steps per launch of the
            # persistent kernel, one graph node replayed
            from paper_1908_07341_gb300.batch import Batch
            k = 8 if side <= 512 else 2        # deeper temporal blocking only while halos are cheap
            nb = max(k, (n // k) * k)
            b = Batch([side], [0.66], [0.44], [SEED], [0], device=dev, stream=stream)
            b.configure(k, 256, 1 << 17).init("random", INIT_SEED)
            b.run(k)
            s_ev.record(stream)
            b.run(nb)
            e_ev.record(stream)
            torch.cuda.synchronize()
            ms_b = s_ev.elapsed_time(e_ev)
            row["batch_of_one_us_per_step"] = 1e3 * ms_b / nb
            b.close()
        rows.append(row)
    return {"workload": "one L x L bit-packed torus, J=0.44, q=0.66, random start, full steps through shk_run "
                        "(sums of the last step kept on the device)", "rows": rows}


def bench_serving(dev, stream, n_jobs: int = 10_000, sub_jobs: int = 1000, steps_per_launch: int = 2,
                  launches_per_tick: int = 16, block_threads: int = 256, tile_sites: int = 1 << 17):
    """Continuous batching on the serving stream: its first n_jobs jobs (the
    whole configured stream by default: 10^4 jobs, Poisson arrivals at a mean
    of 200/s, L log-uniform in [64, 4096], steps log-uniform in [10^3, 10^5],
    admission cap 96 GB) replayed in real time, then two replays of sub_jobs
    jobs each at about 50% and 80% of the capacity the first replay measured,
    so that their p99 is a percentile of a steady state rather than the depth
    of a backlog.  Latency = end of the tick that finished a job - its
    arrival."""
    import numpy as np

    from paper_1908_07341_gb300 import workloads
    from paper_1908_07341_gb300.serve import Server, replay_stream

    def one(n, rate, seed=5):
        w = workloads.serving_stream(n_jobs=n, rate_per_s=rate, seed=seed)
        srv = Server(max_slots=1024, arena_bytes=8 << 30, hbm_budget=96 << 30, device=dev, stream=stream)
        srv.configure(steps_per_launch=steps_per_launch, launches_per_tick=launches_per_tick,
                      block_threads=block_threads, tile_sites=tile_sites)
        r = replay_stream(srv, w["jobs"], w["arrivals"])
        srv.close()
        assert all(x["status"] == 0 for x in r["results"])
        lat = np.array([x["latency_s"] for x in r["results"]])
        return {"jobs": n, "arrival_rate_per_s": rate, "site_updates": w["site_updates"],
                "wall_s": r["wall_s"], "throughput": w["site_updates"] / r["wall_s"],
                "jobs_per_s": n / r["wall_s"], "p50_latency_s": r["p50_s"], "p90_latency_s":
                float(np.percentile(lat, 90)), "p99_latency_s": r["p99_s"], "mean_latency_s": r["mean_s"],
                "max_latency_s": float(lat.max()), "last_arrival_s": float(np.max(w["arrivals"]))}

    sat = one(n_jobs, 200.0)
    mean_work = sat["site_updates"] / n_jobs
    capacity_jobs_per_s = sat["throughput"] / mean_work
    sub = [dict(one(sub_jobs, round(f * capacity_jobs_per_s, 2), seed=6 + i), utilisation=f)
           for i, f in enumerate((0.5, 0.8))]
    return {"workload": f"first {n_jobs} jobs of the serving stream (Poisson 200/s, L log-uniform [64,4096], "
                        "q~U[0.05,3], J~U[0.05,1.5], steps log-uniform [1e3,1e5], seed 5, admission cap 96 GB)",
            "jobs": n_jobs, "unit": UNIT, "value": sat["throughput"], "p50_latency_s": sat["p50_latency_s"],
            "p99_latency_s": sat["p99_latency_s"], "saturated": sat, "sub_saturation": sub,
            "steps_per_launch": steps_per_launch, "launches_per_tick": launches_per_tick,
            "block_threads": block_threads, "tile_sites": tile_sites,
            "capacity_jobs_per_s": capacity_jobs_per_s,
            "note": f"the stream offers about {200.0 / capacity_jobs_per_s:.1f}x the capacity, so the saturated "
                    "latencies measure the backlog; the sub-saturation replays (other seeds of the same job "
                    "distribution) give the latency of a steady state"}


def run_kernel_case(spec: str) -> int:
    """--kernel-case LAYOUT:L:LAUNCHES[:VARIANT[:generic]] -- a random-start
    lattice and LAUNCHES alternating half-step launches through shk_halfstep
    (the benchmark's kernel and grid), nothing else: the command profiled in
    profiles/.  Without VARIANT the launch shape is autotuned first (which
    launches every variant); with it that variant is set directly.  The sweeps
    run specialised (thresholds compiled in, as in the benchmark) unless the
    last field is "generic"."""
    import torch

    from paper_1908_07341_gb300 import build as libbuild

    libbuild.build()
    import paper_1908_07341_gb300 as shk

    parts = spec.split(":")
    layout, side, launches = parts[0], int(parts[1]), int(parts[2])
    if layout == "checkerboard":             # LAUNCHES / 2 full checkerboard steps at J = 0.44
        from paper_1908_07341_gb300.lattice import checkerboard_run
        plane = shk.alloc_plane(side, "bitpack")
        shk.init_plane("bitpack", plane, side, "random", init_seed=INIT_SEED)
        rows = checkerboard_run(plane, side, 0.44, SEED, 0, 0, max(1, launches // 2))
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": spec, "last": rows[-1].cpu().tolist()}))
        return 0
    if layout == "cftp":                     # LAUNCHES pairs of side x side, one k_cftp launch
        import numpy as np

        from paper_1908_07341_gb300.experiments import critical_J
        from paper_1908_07341_gb300.lattice import cftp
        q = np.full(launches, 1.0)
        ks, _ = cftp(np.full(launches, side), q, critical_J(q) - 0.1, np.uint64(SEED),
                     np.arange(launches, dtype=np.uint32), k_max=16)
        print(json.dumps({"kernel_case": spec, "mean_k": float(ks.mean()), "min_k": int(ks.min())}))
        return 0
    from paper_1908_07341_gb300 import tune
    generic = len(parts) > 4 and parts[4] == "generic"
    shk.specialize(shk.lattice.SPECIALIZE_OFF if generic else shk.lattice.SPECIALIZE_BLOCKING)
    if len(parts) > 3:
        tune.set_variant(layout, int(parts[3]))
    else:
        tune.autotune(layout, side)              # the launch shape the benchmark uses
    lat = shk.Lattice(side, layout).set_seed(SEED, 0).set_params(Q, J).init("random", init_seed=INIT_SEED)
    T = shk.thresholds(Q, J)
    acc = torch.zeros(shk.NOBS, dtype=torch.int64, device="cuda")
    a, b = lat.plane(0), lat.plane(1)
    for k in range(launches):
        half = k & 1
        shk.halfstep(layout, half, a if half == 0 else b, b if half == 0 else a, side, T, SEED, 0, k, acc)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": spec, "sums": acc.cpu().tolist()}))
    return 0


def run_batch_case(spec: str) -> int:
    """--batch-case N[:K:BLOCK:TILE] -- the first N lattices of the
    phase-diagram workload, autotuned (or configured with K steps per launch,
    BLOCK threads and TILE sites when given), then 8 launches: the command
    profiled for k_batch."""
    import torch

    from paper_1908_07341_gb300 import build as libbuild

    libbuild.build()
    from paper_1908_07341_gb300 import tune, workloads
    from paper_1908_07341_gb300.batch import Batch

    parts = [int(x) for x in str(spec).split(":")]
    n_lattices = parts[0]
    w = workloads.phase_diagram_batch()
    sel = {k: w[k][:n_lattices] for k in ("L", "q", "J", "seed", "lattice_id")}
    b = Batch(**sel)
    if len(parts) == 4:
        best = tuple(parts[1:])
        b.configure(*best).init("random", w["init_seed"])
    else:
        best = tune.autotune_batch(b, init_kind="random", init_seed=w["init_seed"])["best"]
    b.run(8 * best[0])
    torch.cuda.synchronize()
    print(json.dumps({"batch_case": n_lattices, "tuned": list(best), "step": b.step}))
    return 0


def _kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("device.cuh", "bounds.cuh", "sweep.cuh", "sweep_kernels.cuh"):   # the sweep kernels' device code
        with open(os.path.join(ROOT, "paper_1908_07341_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def _load_traffic():
    """DRAM bytes per launch from the committed ncu summaries (profiles/
    traffic.txt), kept only when they were taken on the current kernel sources."""
    out = {}
    try:
        current = _kernel_source_hash()
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 3 and not line.startswith("#") and parts[2] == current:
                    out[parts[0]] = int(parts[1])
    except Exception:
        return {}
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched phase-diagram line")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving line")
    ap.add_argument("--no-section3", action="store_true", help="skip the Section 3 kernels")
    ap.add_argument("--serving-jobs", type=int, default=10_000,
                    help="jobs of the serving stream to replay (default: the full stream of 10^4)")
    ap.add_argument("--serving-sub-jobs", type=int, default=1000,
                    help="jobs of each sub-saturation replay (50%% and 80%% of the measured capacity)")
    ap.add_argument("--batch-case", default=None,
                    help="N[:K:BLOCK:TILE] -- only run the first N phase-diagram lattices (for profiling)")
    ap.add_argument("--kernel-case", default=None,
                    help="LAYOUT:L:LAUNCHES[:VARIANT] -- only run half-step launches (for profiling)")
    args = ap.parse_args()
    if args.kernel_case:
        return run_kernel_case(args.kernel_case)
    if args.batch_case:
        return run_batch_case(args.batch_case)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
