"""Host-side logic of bench.py's multi-rank (replicas-only) mode, run as two
gloo ranks on the CPU: the slowest rank's time sets the whole-job rate and
every rank gets its own lattice id."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [100.0, 250.0][rank]          # rank 1 is the slow one
        rate, ms = bench.whole_job_rate(local_ms, 1e9, dist, "cpu")
        out[rank] = (rate, ms, bench.replica_lattice_id(rank))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_uses_the_slowest_rank():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        rate, ms, lat_id = out[r]
        assert ms == 250.0
        assert rate == pytest.approx(2 * 1e9 / 0.25)
        assert lat_id == r


def test_single_process_rate():
    import bench
    rate, ms = bench.whole_job_rate(200.0, 5e8)
    assert ms == 200.0 and rate == pytest.approx(2.5e9)
