"""Pins of the oracle's multi-die 2D evaluation (Sec. V-B, eq. 2d-place):
the D2D HPWL with HBTs at the centres of their optimal regions (eq.
optimal-region) equals the bistratal exact wirelength of eq. wl-obj, WA
spans tend to it as gamma -> 0, central differences of the wirelength,
per-layer total charge, single-mode closed forms of the 2D Poisson solve,
independence of the layers, and linearity in the layer weights."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2403_09070_gb300 import synth
from tests.helpers import problem


def _optimal_region_centres(p, x, y, z):
    """Centres of eq. optimal-region for every crossing net, from the
    bounding boxes of the top and bottom pins (pins at their die's offset)."""
    zlo, zhi = synth.depth_range(p)
    top = z > 0.5 * (zlo + zhi)
    ns, pi = p["net_start"], p["pin_inst"]
    out = []
    for e in range(p["n_net"]):
        s0, s1 = ns[e], ns[e + 1]
        ins = pi[s0:s1]
        t = top[ins]
        if t.all() or not t.any():
            continue
        c = []
        for v, ob, ot in ((x, p["off_bx"], p["off_tx"]), (y, p["off_by"], p["off_ty"])):
            pv = v[ins] + np.where(t, ot[s0:s1], ob[s0:s1])
            lo_p, hi_p = pv[t].min(), pv[t].max()
            lo_m, hi_m = pv[~t].min(), pv[~t].max()
            a, b = max(lo_p, lo_m), min(hi_p, hi_m)
            c.append(0.5 * (min(a, b) + max(a, b)))
        out.append(c)
    out = np.array(out).reshape(-1, 2)
    return out[:, 0], out[:, 1]


def test_hbt_at_optimal_region_gives_the_bistratal_wirelength():
    """Sec. III-A: with each HBT inside its optimal region the D2D HPWL of
    eq. exact-wirelength is minimal and equals eq. wl-obj (the 3D oracle's
    exact D2D HPWL)."""
    p = synth.make_problem("cells_2k")
    hx, hy = _optimal_region_centres(p, p["x"], p["y"], p["z"])
    q = synth.to_problem2d(p, hbt_xy=(hx, hy))
    r2 = Oracle(q).eval2d(q["x"], q["y"], q["z"], grads=False)
    w3 = Oracle(p).wirelength(p["x"], p["y"], p["z"])
    assert r2["hpwl_d2d"] == pytest.approx(w3["hpwl_d2d"], rel=1e-12)
    assert r2["n_cross"] == w3["n_cross"] == len(q["hbt_nets"])
    # moving HBTs away from their optimal regions never lowers it
    rng = np.random.default_rng(3)
    q2 = synth.to_problem2d(p, hbt_xy=(hx + rng.normal(0, 20, hx.size), hy + rng.normal(0, 20, hy.size)))
    r3 = Oracle(q2).eval2d(q2["x"], q2["y"], q2["z"], grads=False)
    assert r3["hpwl_d2d"] > r2["hpwl_d2d"]


def test_wa_tends_to_exact_d2d_hpwl():
    p = synth.make_problem("cells_2k")
    q = synth.to_problem2d(p, seed=1)
    prev = None
    for g in (4.0, 0.5, 0.02):
        q["gamma"] = g
        r = Oracle(q).eval2d(q["x"], q["y"], q["z"], grads=False)
        gap = r["hpwl_d2d"] - r["wl"]
        assert gap >= -1e-9
        if prev is not None:
            assert gap < prev
        prev = gap
    assert prev < 1e-3 * r["hpwl_d2d"]


def test_hand_example_hbt_in_both_partial_nets():
    """One net: a top pin at (0, 0), a bottom pin at (10, 0) and its HBT at
    (4, 0).  Partial nets {top, HBT} and {bottom, HBT}: exact D2D HPWL
    4 + 6 = 10; each is a two-point WA span L tanh(L / 2 gamma) whose
    derivative in the right point is tanh(u) + u sech^2(u), u = L / 2 gamma,
    so the HBT feels d(4)/dx - d(6)/dx."""
    g = 1.5
    p = problem([(1, 1, 1, 1), (1, 1, 1, 1), (1, 1, 1, 1)], nets=[[0, 1, 2]], die=(-20.0, -20.0, 20.0, 20.0),
                grid=(4, 4, 3), gamma=g, lam=0.0)
    p.update(mode=1, is_hbt=np.array([0, 0, 1], np.uint8), lam_layer=(0.0, 0.0, 0.0))
    dz = 3 * 10.0
    z = np.array([0.75 * dz, 0.25 * dz, 0.5 * dz])
    r = Oracle(p).eval2d(np.array([0.0, 10.0, 4.0]), np.zeros(3), z)
    assert r["hpwl_d2d"] == pytest.approx(10.0, rel=1e-14)
    assert r["n_cross"] == 1

    def span(L):
        u = L / (2 * g)
        return L * math.tanh(u), math.tanh(u) + u / math.cosh(u) ** 2

    s4, d4 = span(4.0)
    s6, d6 = span(6.0)
    assert r["wl"] == pytest.approx(s4 + s6, rel=1e-12)
    assert r["gx"][2] == pytest.approx(d4 - d6, rel=1e-10)
    assert r["gx"][0] == pytest.approx(-d4, rel=1e-10)
    assert r["gx"][1] == pytest.approx(d6, rel=1e-10)
    assert np.all(r["gy"] == 0)


def test_wirelength_central_differences():
    p = synth.make_problem("cells_2k", n_std=300, n_net=320)
    q = synth.to_problem2d(p, seed=2)
    q["lam_layer"] = (0.0, 0.0, 0.0)
    o = Oracle(q)
    r = o.eval2d(q["x"], q["y"], q["z"])
    rng = np.random.default_rng(5)
    nh = len(q["hbt_nets"])
    idx = np.r_[rng.choice(p["n_inst"], 12, replace=False), p["n_inst"] + rng.choice(nh, 8, replace=False)]
    h = 1e-4
    for i in idx:
        for a, key in ((0, "gx"), (1, "gy")):
            v = [q["x"].copy(), q["y"].copy()]
            v[a][i] += h
            fp = o.eval2d(v[0], v[1], q["z"], grads=False)["obj"]
            v[a][i] -= 2 * h
            fm = o.eval2d(v[0], v[1], q["z"], grads=False)["obj"]
            assert (fp - fm) / (2 * h) == pytest.approx(r[key][i], rel=1e-5, abs=1e-7), (i, a)


def test_density_charge_per_layer():
    """Instances well inside the region: layer l's map holds exactly the
    area of the instances on that layer (their die's footprint; HBTs on the
    third layer)."""
    p = synth.make_problem("cells_2k")
    d = p["xh"] - p["xl"]
    x = np.clip(p["x"], p["xl"] + 0.15 * d, p["xh"] - 0.15 * d)
    y = np.clip(p["y"], p["yl"] + 0.15 * d, p["yh"] - 0.15 * d)
    q = synth.to_problem2d(p, x, y, p["z"], seed=4)
    q["x"] = np.clip(q["x"], p["xl"] + 0.15 * d, p["xh"] - 0.15 * d)
    q["y"] = np.clip(q["y"], p["yl"] + 0.15 * d, p["yh"] - 0.15 * d)
    o = Oracle(q)
    g = o.geometry()
    rho = o.density_direct(q["x"], q["y"], q["z"])
    hbt = q["is_hbt"].astype(bool)
    top = (q["z"] > 0.5 * 3 * g["db"]) & ~hbt
    area_top = (q["w_top"] * q["h_top"])[top].sum()
    area_bot = (q["w_bot"] * q["h_bot"])[~top & ~hbt].sum()
    area_hbt = (q["w_bot"] * q["h_bot"])[hbt].sum()
    A_b = g["wb"] * g["hb"]
    assert rho[0].sum() * A_b == pytest.approx(area_bot, rel=1e-10)
    assert rho[1].sum() * A_b == pytest.approx(area_top, rel=1e-10)
    assert rho[2].sum() * A_b == pytest.approx(area_hbt, rel=1e-10)
    # the fixed-point replica agrees within its rounding
    qf = o.density_fixed(q["x"], q["y"], q["z"], use_float=False) * 2.0 ** -36
    assert np.abs(qf - rho).max() < 1e-9


@pytest.mark.parametrize("layer,j,k", [(0, 1, 0), (1, 2, 3), (2, 0, 5)])
def test_poisson2d_single_mode_and_layer_independence(layer, j, k):
    """rho = A cos(w_j u) cos(w_k v) on one layer: phi = rho / (w_j^2 + w_k^2)
    there (eq. 2d-place's 2D fields), nothing on the other layers, E_z = 0,
    U = 1/2 A_b sum rho phi = 1/2 A_b A^2 N c / (4 w^2) with the mean of
    cos^2 over the grid (1/2 per nonzero index, 1 for a zero index)."""
    nx, ny = 16, 8
    p = problem([], grid=(nx, ny, 3), die=(0.0, 0.0, 32.0, 16.0))
    p["mode"] = 1
    o = Oracle(p)
    g = o.geometry()
    u = (np.arange(nx) + 0.5) * g["wb"]
    v = (np.arange(ny) + 0.5) * g["hb"]
    wj, wk = j * math.pi / g["dx"], k * math.pi / g["dy"]
    A = 0.7
    rho = np.zeros((3, ny, nx))
    rho[layer] = A * np.outer(np.cos(wk * v), np.cos(wj * u))
    out = o.poisson(rho)
    w2 = wj * wj + wk * wk
    np.testing.assert_allclose(out["phi"][layer], rho[layer] / w2, atol=1e-12)
    for other in range(3):
        if other != layer:
            assert np.abs(out["phi"][other]).max() < 1e-12
    assert np.abs(out["ez"]).max() == 0.0
    ex = A * wj * np.outer(np.cos(wk * v), np.sin(wj * u)) / w2
    np.testing.assert_allclose(out["ex"][layer], ex, atol=1e-12)
    mean = (0.5 if j else 1.0) * (0.5 if k else 1.0)
    U = 0.5 * g["wb"] * g["hb"] * A * A * nx * ny * mean / w2
    assert out["energy_layers"][layer] == pytest.approx(U, rel=1e-12)
    assert sum(out["energy_layers"]) == pytest.approx(U, rel=1e-12)


def test_objective_linear_in_layer_weights():
    p = synth.make_problem("cells_2k")
    q = synth.to_problem2d(p, seed=6)
    base = dict(q, lam_layer=(0.0, 0.0, 0.0))
    r0 = Oracle(base).eval2d(q["x"], q["y"], q["z"], grads=False)
    lam = (1e-3, 3e-3, 7e-3)
    r1 = Oracle(dict(q, lam_layer=lam)).eval2d(q["x"], q["y"], q["z"], grads=False)
    assert r0["obj"] == pytest.approx(r0["wl"], rel=1e-14)
    expect = r0["wl"] + sum(l * r0[k] for l, k in zip(lam, ("e_bot", "e_top", "e_hbt")))
    assert r1["obj"] == pytest.approx(expect, rel=1e-12)
    assert min(r0["e_bot"], r0["e_top"], r0["e_hbt"]) > 0
