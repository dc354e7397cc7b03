"""Child process of test_gpu_debug_bounds: with SHK_LIBRARY pointing at the
bounds-checked build, runs small cases of every kernel family, checks them
against the oracle (or against the single-lattice path, itself checked), and
prints the library's bounds record as JSON.  Nothing here is a deliberate
out-of-range access: the point is that legitimate runs record none."""
import json
import sys

import numpy as np
import torch


def main() -> int:
    import paper_1908_07341_gb300 as shk
    from paper_1908_07341_gb300 import _lib
    from paper_1908_07341_gb300.batch import Batch, stats_from_observables
    from paper_1908_07341_gb300.lattice import (cftp, checkerboard_run, coalescence_times, diag_correlations,
                                               pack_bits, unpack_bits)
    from paper_1908_07341_gb300.serve import Server
    from oracle import oracle as orc

    assert _lib.LIB_PATH.endswith("libshaken_debug.so"), _lib.LIB_PATH
    so = _lib.lib()
    site = np.zeros(1, dtype=np.uint32)
    assert so.shk_debug_bounds(site.ctypes.data) == _lib.OK   # clears any earlier record
    checked = []

    # handle runs: one-CTA path (int8 ragged, bit-packed) and the grid sweeps
    for L, layout, steps in ((5, "int8", 3), (33, "int8", 3), (64, "int8", 4), (96, "bitpack", 3),
                             (288, "bitpack", 2), (1024, "bitpack", 2), (1024, "int8", 2), (2048, "bitpack", 2)):
        lat = shk.Lattice(L, layout).set_seed(5, 1).set_params(0.8, 0.4).init("random", init_seed=3)
        obs = lat.run(steps, obs=True).cpu().numpy()
        s = orc.init_plane(L, orc.INIT_RANDOM, 3, 1, 0)
        t = orc.init_plane(L, orc.INIT_RANDOM, 3, 1, 1)
        ref = orc.run(s, t, L, 0.8, 0.4, 5, 1, 0, steps)
        assert np.array_equal(obs, ref), (L, layout)
        assert np.array_equal(lat.read_spins(0).reshape(-1), s), (L, layout)
        lat.close()
        checked.append(f"run {layout} L={L}")
    # the allocation-free entry point: tau plane and sums in the library's
    # static scratch array, compared with a handle run over the same steps
    for L, layout in ((96, "bitpack"), (257, "int8")):
        lat = shk.Lattice(L, layout).set_seed(5, 2).set_params(0.7, 0.45).init("random", init_seed=8)
        from tests.gpu_util import from_device_plane, to_device_plane
        plane = to_device_plane(lat.read_spins(0).reshape(-1).copy(), L, layout)
        last = torch.zeros(shk.NOBS, dtype=torch.int64, device="cuda")
        want = lat.run(3, obs=True)[-1].cpu().numpy()
        rc = so.shk_shaken_run_static(_lib.BITPACK if layout == "bitpack" else _lib.INT8, plane.data_ptr(), L,
                                      0.7, 0.45, 5, 2, 0, 3, last.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
        assert rc == _lib.OK
        torch.cuda.synchronize()
        assert np.array_equal(from_device_plane(plane, L, layout), lat.read_spins(0).reshape(-1)), (L, layout)
        assert np.array_equal(last.cpu().numpy(), want), (L, layout)
        lat.close()
    checked.append("allocation-free run")
    # every launch shape of the sweeps at a strip-walk size
    from paper_1908_07341_gb300 import tune
    for layout in ("bitpack", "int8"):
        for v in range(len(tune.variant_names(layout))):
            tune.set_variant(layout, v)
            lat = shk.Lattice(1024, layout).set_seed(2, 0).set_params(1.0, 0.35).init("random", init_seed=1)
            lat.run(2)
            lat.close()
        tune.set_variant(layout, 0)
        checked.append(f"variants {layout}")
    # batched sweep (wrapping single tiles and multi-tile lattices) and serving
    cfg = dict(L=[32, 96, 512, 1024], q=[1.0, 0.5, 0.8, 0.6], J=[0.3, 0.6, 0.4, 0.5], seed=[1, 2, 3, 4],
               lattice_id=[0, 1, 2, 3])
    b = Batch(**cfg).configure(4, 256, 1 << 15).init("random", init_seed=9)
    b.run(8)
    st = b.read_stats()
    for i in range(4):
        lat = shk.Lattice(cfg["L"][i], "bitpack").set_seed(cfg["seed"][i], cfg["lattice_id"][i])
        lat.set_params(cfg["q"][i], cfg["J"][i]).init("random", init_seed=9)
        assert np.array_equal(st[i], stats_from_observables(lat.run(8, obs=True).cpu().numpy())), i
        lat.close()
    b.close()
    srv = Server(max_slots=3, arena_bytes=8 << 20).configure(steps_per_launch=2, launches_per_tick=2)
    for i in range(4):
        srv.submit(L=cfg["L"][i], q=cfg["q"][i], J=cfg["J"][i], seed=cfg["seed"][i], lattice_id=i, n_steps=6)
    done = 0
    for _ in range(20):
        srv.tick()
        done += len(srv.poll())
        if done == 4:
            break
    assert done == 4
    srv.close()
    checked.append("batch and serve")
    # Section 3 kernels
    L = 64
    s0 = np.where(np.random.default_rng(4).random(L * L) < 0.5, 1, -1).astype(np.int8)
    plane = shk.alloc_plane(L, "bitpack")
    plane.zero_()
    raw = pack_bits(s0).view(np.uint8)
    plane[: raw.size].copy_(torch.from_numpy(raw.copy()))
    rows = checkerboard_run(plane, L, 0.44, 3, 0, 0, 3).cpu().numpy()
    ref = s0.copy()
    assert np.array_equal(rows, orc.checkerboard_run(ref, L, 0.44, 3, 0, 0, 3))
    assert np.array_equal(unpack_bits(plane.cpu().numpy()[: L * L // 8], L).reshape(-1), ref)
    assert np.array_equal(diag_correlations(plane, L, [1, 5, 63]).cpu().numpy(),
                          orc.diag_correlations(ref, L, [1, 5, 63]))
    coalescence_times([32, 64], [1.0, 1.0], [0.3, 0.3], [1, 1], [0, 1], 300)
    coalescence_times([32, 96], [0.0, 0.0], [0.3, 0.3], [1, 1], [0, 1], 300, dynamics="checkerboard")
    cftp([32, 64], [1.0, 1.0], [0.3, 0.3], [1, 1], [0, 1], k_max=10)
    cftp([32, 96], [0.0, 0.0], [0.3, 0.3], [1, 1], [0, 1], k_max=10, dynamics="checkerboard")
    checked.append("section 3")
    torch.cuda.synchronize()
    status = so.shk_debug_bounds(site.ctypes.data)
    print(json.dumps({"status": int(status), "site": int(site[0]), "checked": checked}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
