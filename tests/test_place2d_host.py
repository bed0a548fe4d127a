"""Host set-up of the multi-die 2D placement (Sec. V-B): HBTs at the
centres of their optimal regions (eq. optimal-region) checked against a
brute-force minimisation of the D2D HPWL (eq. exact-wirelength), and the
dies' fillers filling each die's free area."""
import numpy as np
import pytest

from paper_2403_09070_gb300 import place2d, synth


def _d2d_hpwl_net(px, py, top, hx, hy):
    w = 0.0
    for m in (top, ~top):
        xs = np.r_[px[m], hx]
        ys = np.r_[py[m], hy]
        w += xs.max() - xs.min() + ys.max() - ys.min()
    return w


def test_hbt_positions_minimise_d2d_hpwl_brute_force():
    p = synth.make_problem("cells_2k")
    hx, hy, nets = place2d.hbt_positions(p)
    zlo, zhi = synth.depth_range(p)
    top = p["z"] > 0.5 * (zlo + zhi)
    rng = np.random.default_rng(0)
    for k in rng.choice(nets.size, 25, replace=False):
        e = nets[k]
        s0, s1 = p["net_start"][e], p["net_start"][e + 1]
        ins = p["pin_inst"][s0:s1]
        t = top[ins]
        px = p["x"][ins] + np.where(t, p["off_tx"][s0:s1], p["off_bx"][s0:s1])
        py = p["y"][ins] + np.where(t, p["off_ty"][s0:s1], p["off_by"][s0:s1])
        best = _d2d_hpwl_net(px, py, t, hx[k], hy[k])
        gx = np.linspace(px.min() - 5, px.max() + 5, 61)
        gy = np.linspace(py.min() - 5, py.max() + 5, 61)
        brute = min(_d2d_hpwl_net(px, py, t, a, b) for a in gx for b in gy)
        assert best <= brute + 1e-9
        # and equals eq. wl-obj per axis: max{p_e, p_e+ + p_e-}
        wl = 0.0
        for v in (px, py):
            wl += max(v.max() - v.min(), v[t].max() - v[t].min() + v[~t].max() - v[~t].min())
        assert best == pytest.approx(wl, rel=1e-12)
    assert nets.size > 1000


def test_from_3d_structure_and_die_fillers():
    p = synth.make_problem("cells_2k")
    q = place2d.from_3d(p, lam_layer=(1e-3, 2e-3, 3e-3))
    f = q["fillers"]
    nh = int(q["is_hbt"].sum())
    assert q["mode"] == 1 and q["nz"] == 3
    assert nh == f["first"] - p["n_inst"] and q["n_inst"] == f["first"] + f["n_top"] + f["n_bot"]
    assert not q["is_hbt"][f["first"]:].any()
    area = (p["xh"] - p["xl"]) * (p["yh"] - p["yl"])
    wb = (q["xh"] - q["xl"]) / q["nx"]
    dz = 3 * wb
    hbt = q["is_hbt"].astype(bool)
    top = (q["z"] > 0.5 * dz) & ~hbt
    bot = ~top & ~hbt
    for on, w, h, key in ((top, "w_top", "h_top", "top"), (bot, "w_bot", "h_bot", "bot")):
        filled = float(np.sum((q[w] * q[h])[on]))
        unit = f[f"w_{key}"] * f[f"h_{key}"]
        assert abs(filled - area) <= 0.5 * unit + 1e-6 * area, key
    # HBT pins close every crossing net, at the optimal-region centres
    hx, hy, nets = place2d.hbt_positions(p)
    np.testing.assert_array_equal(q["hbt_nets"], nets)
    np.testing.assert_allclose(q["x"][p["n_inst"]:p["n_inst"] + nh], hx)
