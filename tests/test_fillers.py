"""Host logic of the dummy fillers (Sec. III-A): the product's filler plan
against the oracle's, and the structure of the inserted instance table."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2403_09070_gb300 import fillers, synth


@pytest.mark.parametrize("u", [(0.8, 0.8), (0.7, 0.9), (1.0, 0.6), (0.0, 0.0)])
@pytest.mark.parametrize("kind", ["uniform", "center"])
def test_plan_matches_oracle(u, kind):
    p = synth.make_problem("cells_2k", positions=kind)
    a = fillers.plan(p, *u)
    b = Oracle(p).filler_plan(p["z"], *u)
    for k in ("vol_a", "vol_f_top", "vol_f_bot", "vol_fr", "w_top", "h_top", "w_bot", "h_bot"):
        assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-9), k
    assert (a["n_top"], a["n_bot"], a["n_free"]) == (b["n_top"], b["n_bot"], b["n_free"])


def test_plan_matches_oracle_200k_sample():
    p = synth.make_problem("cells_200k", n_std=50_000, n_net=52_000)
    a = fillers.plan(p, 0.8, 0.75)
    b = Oracle(p).filler_plan(p["z"], 0.8, 0.75)
    assert (a["n_top"], a["n_bot"], a["n_free"]) == (b["n_top"], b["n_bot"], b["n_free"])
    assert a["vol_a"] == pytest.approx(b["vol_a"], rel=1e-12)


def test_insert_structure():
    p = synth.make_problem("cells_2k", positions="center")
    q = fillers.insert(p, 0.8, 0.8, seed=3)
    f = q["fillers"]
    n0, nt, nb, nf = p["n_inst"], f["n_top"], f["n_bot"], f["n_free"]
    assert f["first"] == n0 and q["n_inst"] == n0 + nt + nb + nf
    assert nt > 0 and nb > 0 and nf > 0
    # netlist untouched: fillers are pinless
    for k in ("net_start", "pin_inst", "off_bx", "off_ty"):
        assert np.array_equal(q[k], p[k])
    assert q["pin_inst"].max() < n0
    zlo, zhi = synth.depth_range(p)
    zf = q["z_fixed"].astype(bool)
    assert not zf[:n0].any() and zf[n0:n0 + nt + nb].all() and not zf[n0 + nt + nb:].any()
    assert np.all(q["z"][n0:n0 + nt] == zhi) and np.all(q["z"][n0 + nt:n0 + nt + nb] == zlo)
    zfree = q["z"][n0 + nt + nb:]
    assert np.all((zfree >= zlo) & (zfree <= zhi))
    assert 0.3 < np.mean(zfree > 0.5 * (zlo + zhi) * 1.0) < 0.7  # about half on each die
    assert not q["is_macro"][n0:].any()
    # one footprint per die: top fillers carry the top footprint in both tables
    assert np.all(q["w_top"][n0:n0 + nt] == f["w_top"]) and np.all(q["w_bot"][n0:n0 + nt] == f["w_top"])
    assert np.all(q["w_bot"][n0 + nt:n0 + nt + nb] == f["w_bot"])
    assert np.all(q["w_top"][n0 + nt + nb:] == f["w_top"]) and np.all(q["h_bot"][n0 + nt + nb:] == f["h_bot"])
    # instances keep their positions; fillers start inside the region
    for k in ("x", "y", "z"):
        assert np.array_equal(q[k][:n0], p[k])
    assert np.all((q["x"] >= p["xl"]) & (q["x"] <= p["xh"]))
    # the inserted volume matches the plan within one filler per set
    dz = 4 * zlo
    ut = f["w_top"] * f["h_top"] * 0.5 * dz
    ub = f["w_bot"] * f["h_bot"] * 0.5 * dz
    assert abs(nt * ut - f["vol_f_top"]) <= 0.5 * ut and abs(nb * ub - f["vol_f_bot"]) <= 0.5 * ub


def test_insert_then_replan_sees_no_white_space():
    """After insertion at u+ = u- = 0.8 the region is full: a second plan over
    the augmented table finds (nearly) no white space left for free fillers."""
    p = synth.make_problem("cells_2k", positions="center")
    q = fillers.insert(p, 0.8, 0.8)
    again = Oracle(q).filler_plan(q["z"], 1.0, 1.0)
    g = Oracle(q).geometry()
    V = g["dx"] * g["dy"] * g["dz"]
    assert again["vol_fr"] < 2e-3 * V
