"""GPU checks of the Section 3 experiment drivers: properties that hold for
any run (torus identities, monotone trends far outside the noise), on small
sizes."""
import numpy as np
import pytest
import torch

from paper_1908_07341_gb300 import experiments as ex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1908_07341_gb300 import build
    build.build()


def test_correlation_table_properties():
    """On a 32 x 32 torus the displacements (16, 16) and (16, -16) coincide, so
    the two directions agree exactly at lag 16; for small q the SW-NE
    correlation is far below the NW-SE one (Theorem 2.4 of the cited work)."""
    r = ex.diagonal_correlations_table(points=((0.05, 1.7), (2.5, 0.43)), burn_in=2000, n_samples=200, gap=5)
    for row in r["rows"]:
        assert row["sw_ne"][-1] == row["nw_se"][-1]
        assert all(-1.0 <= v <= 1.0 for v in row["sw_ne"] + row["nw_se"])
    small_q = r["rows"][0]
    assert small_q["sw_ne"][0] < small_q["nw_se"][0] - 0.3


def test_coalescence_grows_towards_the_critical_curve():
    r = ex.coalescence_scan([0.6585], J_offsets=(-0.2, -0.1, 0.0), n_samples=32, max_steps=1 << 20)
    T = r["mean_T"][0]
    assert np.all(np.isfinite(T)) and T[0] < T[1] < T[2]
    assert r["not_reached"].sum() == 0


def test_critical_curve_sweep_small_grid():
    r = ex.critical_curve_sweep(L=32, n_grid=4, warmup=2000, measured=2000, steps_per_launch=8)
    assert r["var_m"].shape == (4, 4) and r["peak_J"].shape == (4,)
    assert np.all(r["var_m"] >= 0) and np.all(np.abs(r["mean_m"]) <= 1) and np.all(r["abs_m"] <= 1)
    # from the all -1 start, the deep ordered corner (largest q and J) stays magnetised
    assert r["abs_m"][-1, -1] > 0.9


def test_gibbs_comparison_rows():
    r = ex.gibbs_comparison(J_values=(0.3,), q_values=(3.0,), n_samples=16, k_max=16)
    assert [row["dynamics"] for row in r["rows"]] == ["checkerboard", "shaken"]
    for row in r["rows"]:
        assert row["n"] == 16 and row["sd_m"] >= 0 and row["mean_H"] < 0
