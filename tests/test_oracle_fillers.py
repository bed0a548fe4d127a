"""Pins of the oracle's filler plan (Sec. III-A, eqs. filler-vol and
free-filler-vol): a worked example by hand, the two utilisation extremes, the
volume balance, and the instance volume against the total charge of the
direct density map (an independent routine)."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2403_09070_gb300 import synth
from tests.helpers import problem


def test_hand_example():
    # Region 10 x 10, grid 2x2x2: w_b = h_b = d_b = 5, d_z = 10, V = 1000,
    # instance depth d_z/2 = 5.
    # cell 0 (bottom, z=2): 2 x 1 x 5 = 10; cell 1 (top, z=8): 3.2 x 0.8 x 5 = 12.8;
    # macro (z = d_z/2: top weight 2*5/10 - 1/2 = 1/2): 3.6 x 3.6 x 5 = 64.8.
    # vol_a = 87.6; u+ = 0.7, u- = 0.9: vol_f+ = 500 * 0.3 = 150, vol_f- = 50,
    # vol_fr = 1000 - 200 - 87.6 = 712.4.
    # footprints: top (1.6+3.2)/2 x 0.8 = 2.4 x 0.8, bottom 3 x 1.
    # counts: 150 / 9.6 = 15.6 -> 16; 50 / 15 = 3.3 -> 3; 712.4 / 12.3 = 57.9 -> 58.
    p = problem([(2, 1, 1.6, 0.8), (4, 1, 3.2, 0.8), (4, 4, 3.2, 3.2)], grid=(2, 2, 2), macros=(2,))
    f = Oracle(p).filler_plan(np.array([2.0, 8.0, 5.0]), 0.7, 0.9)
    assert f["vol_a"] == pytest.approx(87.6, rel=1e-14)
    assert f["vol_f_top"] == pytest.approx(150.0, rel=1e-14)
    assert f["vol_f_bot"] == pytest.approx(50.0, rel=1e-14)
    assert f["vol_fr"] == pytest.approx(712.4, rel=1e-14)
    assert (f["w_top"], f["h_top"], f["w_bot"], f["h_bot"]) == pytest.approx((2.4, 0.8, 3.0, 1.0), rel=1e-14)
    assert (f["n_top"], f["n_bot"], f["n_free"]) == (16, 3, 58)


def test_z_fixed_instances_count_in_volume_not_in_footprint():
    sizes = [(2, 1, 1.6, 0.8), (4, 1, 3.2, 0.8), (2, 2, 2, 2)]
    p = problem(sizes, grid=(2, 2, 2), z_fixed=(2,))
    f = Oracle(p).filler_plan(np.array([2.0, 8.0, 2.5]), 0.8, 0.8)
    assert f["vol_a"] == pytest.approx(10 + 12.8 + 2 * 2 * 5, rel=1e-14)
    assert (f["w_top"], f["h_top"], f["w_bot"], f["h_bot"]) == pytest.approx((2.4, 0.8, 3.0, 1.0), rel=1e-14)


@pytest.mark.parametrize("u", [(1.0, 1.0), (0.0, 0.0), (0.6, 1.0)])
def test_utilisation_extremes_and_balance(u):
    p = synth.make_problem("cells_2k")
    o = Oracle(p)
    g = o.geometry()
    V = g["dx"] * g["dy"] * g["dz"]
    f = o.filler_plan(p["z"], *u)
    assert f["vol_f_top"] == pytest.approx(0.5 * V * (1 - u[0]), rel=1e-14, abs=1e-9)
    assert f["vol_f_bot"] == pytest.approx(0.5 * V * (1 - u[1]), rel=1e-14, abs=1e-9)
    if u == (0.0, 0.0):
        assert f["vol_fr"] == 0.0 and f["n_free"] == 0  # no white space left
    else:
        assert f["vol_f_top"] + f["vol_f_bot"] + f["vol_fr"] + f["vol_a"] == pytest.approx(V, rel=1e-12)
    unit_t = f["w_top"] * f["h_top"] * 0.5 * g["dz"]
    unit_b = f["w_bot"] * f["h_bot"] * 0.5 * g["dz"]
    assert abs(f["n_top"] * unit_t - f["vol_f_top"]) <= 0.5 * unit_t
    assert abs(f["n_bot"] * unit_b - f["vol_f_bot"]) <= 0.5 * unit_b
    assert abs(f["n_free"] * 0.5 * (unit_t + unit_b) - f["vol_fr"]) <= 0.25 * (unit_t + unit_b)


def test_instance_volume_equals_total_charge():
    """Every instance well inside the region: the direct density map (eq.
    density-map-accum, stretched footprints weighted by omega) holds exactly
    the instances' volume, which is vol_a."""
    p = synth.make_problem("cells_2k")
    d = p["xh"] - p["xl"]
    x = np.clip(p["x"], p["xl"] + 0.15 * d, p["xh"] - 0.15 * d)
    y = np.clip(p["y"], p["yl"] + 0.15 * d, p["yh"] - 0.15 * d)
    o = Oracle(p)
    g = o.geometry()
    rho = o.density_direct(x, y, p["z"])
    charge = rho.sum() * g["wb"] * g["hb"] * g["db"]
    f = o.filler_plan(p["z"], 0.8, 0.8)
    assert charge == pytest.approx(f["vol_a"], rel=1e-10)
