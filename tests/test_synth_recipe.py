"""The synthetic input recipe (seeded generators shared by the GPU tests, the
bench and the oracle legs; they hold none of the method's arithmetic): the
workloads are reproducible and have the stated structure -- degree mix,
distinct instances per net, macros' pin share and area, per-die sizes,
offsets, positions inside the movable range, and the grid sizes."""
import numpy as np
import pytest

from paper_2403_09070_gb300 import synth


def test_workloads_are_reproducible():
    a = synth.make_problem("cells_2k")
    b = synth.make_problem("cells_2k")
    for k, v in a.items():
        if isinstance(v, np.ndarray):
            np.testing.assert_array_equal(v, b[k], err_msg=k)
        else:
            assert v == b[k], k


@pytest.mark.parametrize("name,grid", [("cells_2k", (64, 64, 2)), ("cells_200k", (256, 256, 4))])
def test_recipe_structure(name, grid):
    p = synth.make_problem(name)
    n, E = p["n_inst"], p["n_net"]
    assert (p["nx"], p["ny"], p["nz"]) == grid
    d = np.diff(p["net_start"])
    assert d.sum() == p["n_pin"] and d.min() >= 2 and d.max() <= 64
    mix = [((d >= lo) & (d <= hi)).mean() for lo, hi in ((2, 2), (3, 4), (5, 16), (17, 64))]
    for got, want in zip(mix, (0.55, 0.25, 0.17, 0.03)):
        assert abs(got - want) < 0.02, (mix, name)
    assert 3.9 < p["n_pin"] / E < 4.4
    # each pin of a net on a distinct instance, all instance indices valid
    pi = np.asarray(p["pin_inst"])
    assert pi.min() >= 0 and pi.max() < n
    for e in range(0, E, max(1, E // 500)):
        s, t = p["net_start"][e], p["net_start"][e + 1]
        assert len(set(pi[s:t].tolist())) == t - s
    mac = np.asarray(p["is_macro"]).astype(bool)
    assert 0.005 < np.isin(pi, np.flatnonzero(mac)).mean() < 0.02  # macros take about 1 % of pins
    die = (p["xh"] - p["xl"]) * (p["yh"] - p["yl"])
    assert (np.asarray(p["w_bot"])[mac] * np.asarray(p["h_bot"])[mac]).sum() == pytest.approx(0.2 * die, rel=0.02)
    # top-die sizes 0.8x, cells 1-8 sites wide and one row high on the bottom die
    np.testing.assert_allclose(p["w_top"], 0.8 * np.asarray(p["w_bot"]))
    np.testing.assert_allclose(p["h_top"], 0.8 * np.asarray(p["h_bot"]))
    wc = np.asarray(p["w_bot"])[~mac]
    assert wc.min() >= 1 and wc.max() <= 8 and np.all(np.asarray(p["h_bot"])[~mac] == 1.0)
    # top offsets 0.8x the bottom ones, bottom offsets inside the bottom footprint
    np.testing.assert_allclose(p["off_tx"], 0.8 * np.asarray(p["off_bx"]))
    np.testing.assert_allclose(p["off_ty"], 0.8 * np.asarray(p["off_by"]))
    assert np.all(np.abs(p["off_bx"]) <= 0.5 * np.asarray(p["w_bot"])[pi] + 1e-12)
    # centres in the region, z in the movable range [d_z/4, 3 d_z/4]
    zlo, zhi = synth.depth_range(p)
    assert np.all((p["z"] >= zlo) & (p["z"] <= zhi))
    assert np.all((p["x"] >= p["xl"]) & (p["x"] <= p["xh"]) & (p["y"] >= p["yl"]) & (p["y"] <= p["yh"]))


def test_batch_sizes_are_log_uniform_and_grids_follow_the_rule():
    probs = synth.make_batch(24, seed=4)
    ns = np.array([p["n_inst"] for p in probs])
    assert len(probs) == 24 and ns.min() >= 5000 and ns.max() <= 300_000 * 1.01
    for p in probs:
        assert p["nx"] == p["ny"] and p["nx"] in (64, 128, 256, 512)
        assert p["nz"] == (2 if p["nx"] <= 128 else 4)
