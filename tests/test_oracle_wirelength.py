"""Pins of the oracle's bistratal WA wirelength (eqs. wa-model-approx,
exact-wirelength, optimal-region, wl-obj, wl-model) and of the FD depth
gradient (eq. fda-grad, Sec. IV-B) and its normalisation (eq. fda-normalize)."""
import itertools
import math

import numpy as np
import pytest

from helpers import dz_of, problem, read_golden
from oracle import Oracle


def _random_nets(rng, n_inst=12, n_net=10, dmax=7, lattice=None, die=(0, 0, 40, 40), gamma=2.0):
    sizes = [(2.0, 1.0, 1.6, 0.8)] * n_inst
    nets = [list(rng.choice(n_inst, size=int(rng.integers(2, dmax + 1)), replace=False))
            for _ in range(n_net)]
    P = sum(len(n) for n in nets)
    off = np.zeros((P, 4))
    off[:, 0] = rng.uniform(-1.0, 1.0, P)
    off[:, 1] = rng.uniform(-0.5, 0.5, P)
    off[:, 2] = 0.8 * off[:, 0] + rng.uniform(-0.1, 0.1, P)
    off[:, 3] = 0.8 * off[:, 1]
    p = problem(sizes, nets=nets, offsets=off, die=die, grid=(8, 8, 2), gamma=gamma)
    dz = dz_of(p)
    if lattice:
        x = rng.integers(1, lattice, n_inst).astype(float) * (die[2] / lattice)
        y = rng.integers(1, lattice, n_inst).astype(float) * (die[3] / lattice)
        p["off_bx"][:] = 0; p["off_by"][:] = 0; p["off_tx"][:] = 0; p["off_ty"][:] = 0
    else:
        x = rng.uniform(2, die[2] - 2, n_inst)
        y = rng.uniform(2, die[3] - 2, n_inst)
    z = np.where(rng.random(n_inst) < 0.5, 0.3 * dz, 0.7 * dz)
    return p, x, y, z


def _pins(p, x, y, z, e, dz):
    s0, s1 = p["net_start"][e], p["net_start"][e + 1]
    out = []
    for pin in range(s0, s1):
        i = p["pin_inst"][pin]
        top = z[i] > dz / 2
        out.append((i, top, x[i] + (p["off_tx"][pin] if top else p["off_bx"][pin]),
                    y[i] + (p["off_ty"][pin] if top else p["off_by"][pin]),
                    x[i] + (p["off_bx"][pin] if top else p["off_tx"][pin]),
                    y[i] + (p["off_by"][pin] if top else p["off_ty"][pin])))
    return out


def _d2d_hpwl_brute(pins):
    """Eq. exact-wirelength with the HBT t_e placed at the best position,
    found by trying every candidate coordinate per axis (the cost is
    piecewise linear in the HBT coordinate with breaks at pin coordinates)."""
    top = [q for q in pins if q[1]]
    bot = [q for q in pins if not q[1]]
    total = 0.0
    for ax in (2, 3):
        vt = [q[ax] for q in top]
        vb = [q[ax] for q in bot]
        if not vt or not vb:  # C_e = 0: plain HPWL, no HBT
            v = vt + vb
            total += max(v) - min(v)
            continue
        best = math.inf
        for t in vt + vb:
            ct = max(vt + [t]) - min(vt + [t])
            cb = max(vb + [t]) - min(vb + [t])
            best = min(best, ct + cb)
        total += best
    return total


def test_wl_obj_equals_brute_force_hbt_position():
    """Eq. wl-obj (max{p_e, p_e+ + p_e-}) == min over the HBT position of eq.
    exact-wirelength (Sec. III-A, eq. optimal-region)."""
    rng = np.random.default_rng(1)
    for trial in range(5):
        p, x, y, z = _random_nets(rng, n_net=15)
        o = Oracle(p)
        dz = dz_of(p)
        exp = sum(_d2d_hpwl_brute(_pins(p, x, y, z, e, dz)) for e in range(p["n_net"]))
        assert o.wirelength(x, y, z)["hpwl_d2d"] == pytest.approx(exp, rel=1e-13)


def test_wa_to_hpwl_as_gamma_to_zero():
    """WA -> exact extremes as gamma -> 0: W^_Bi -> eq. wl-obj and
    p^_e(z) -> p_e(z)."""
    rng = np.random.default_rng(2)
    p, x, y, z = _random_nets(rng, n_net=20)
    for gam, tol in ((1e-2, 0.2), (1e-4, 2e-3), (1e-6, 2e-5)):
        p["gamma"] = gam
        r = Oracle(p).wirelength(x, y, z)
        assert r["wl_bi"] == pytest.approx(r["hpwl_d2d"], abs=tol * p["n_net"])
    # p^(z): instances at two depths -> each crossing net spans 0.4 d_z
    dz = dz_of(p)
    assert r["wl_z"] == pytest.approx(r["n_cross"] * 0.4 * dz, abs=1e-4)


def test_two_pin_closed_form():
    """Two pins a distance L apart: p^ = L tanh(L/2g); d p^/d x_right =
    tanh(u) + u sech^2(u) with u = L/(2 g)."""
    L, gam = 3.0, 1.7
    p = problem([(1.0, 1.0, 1.0, 1.0)] * 2, nets=[[0, 1]], die=(0, 0, 20, 20), grid=(4, 4, 2), gamma=gam)
    dz = dz_of(p)
    x, y, z = [5.0, 5.0 + L], [4.0, 4.0], [0.3 * dz, 0.3 * dz]
    r = Oracle(p).wirelength(x, y, z)
    u = L / (2 * gam)
    assert r["wl_bi"] == pytest.approx(L * math.tanh(u), rel=1e-14)
    d = math.tanh(u) + u / math.cosh(u) ** 2
    np.testing.assert_allclose(r["gx"], [-d, d], rtol=1e-13)
    np.testing.assert_allclose(r["gy"], [0.0, 0.0], atol=1e-15)


def test_translation_invariance():
    """sum_i dW^/dx_i = 0 and sum_i dW^/dy_i = 0 (WA is shift-equivariant)."""
    from paper_2403_09070_gb300 import synth
    p = synth.make_problem("cells_2k")
    r = Oracle(p).wirelength(p["x"], p["y"], p["z"])
    for g in (r["gx"], r["gy"], r["gwaz"]):
        assert abs(g.sum()) < 1e-10 * np.abs(g).sum()


def test_fd_of_smoothed_wirelength():
    """Central differences of sum W^_Bi in x, y and of sum p^_e(z) in z match
    the analytic gradients (away from branch ties and from z = d_z/2)."""
    rng = np.random.default_rng(3)
    p, x, y, z = _random_nets(rng, n_inst=10, n_net=8, gamma=1.5)
    o = Oracle(p)
    r = o.wirelength(x, y, z)
    h = 1e-6
    for i in range(10):
        for arr, key, g in ((x, "wl_bi", r["gx"]), (y, "wl_bi", r["gy"]), (z, "wl_z", r["gwaz"])):
            a1 = arr.copy(); a1[i] += h
            a0 = arr.copy(); a0[i] -= h
            args = lambda a: [a if arr is x else x, a if arr is y else y, a if arr is z else z]
            fd = (o.wirelength(*args(a1))[key] - o.wirelength(*args(a0))[key]) / (2 * h)
            assert fd == pytest.approx(g[i], abs=1e-6 * max(1.0, abs(g[i])))


def _wbi_def(pins, moved=None):
    """W_Bi of one net from eq. wl-obj, optionally with pin `moved` switched
    to the other die (and to its other-die offset)."""
    tot = 0.0
    for ax, axo in ((2, 4), (3, 5)):
        vt, vb = [], []
        for k, q in enumerate(pins):
            top, v = q[1], q[ax]
            if k == moved:
                top, v = not top, q[axo]
            (vt if top else vb).append(v)
        allv = vt + vb
        pe = max(allv) - min(allv)
        pt = max(vt) - min(vt) if vt else 0.0
        pb = max(vb) - min(vb) if vb else 0.0
        tot += max(pe, pt + pb)
    return tot


@pytest.mark.parametrize("lattice", [None, 4])
def test_fd_depth_gradient_definition(lattice):
    """Eq. fda-grad by its definition (brute force, per instance, summed over
    its nets) == the oracle's vanilla and incremental forms; the two forms are
    equal exactly (ties on a coarse lattice exercise the 2nd extremes)."""
    rng = np.random.default_rng(4 if lattice is None else 5)
    p, x, y, z = _random_nets(rng, n_inst=14, n_net=25, dmax=8, lattice=lattice)
    dz = dz_of(p)
    o = Oracle(p)
    exp = np.zeros(p["n_inst"])
    for e in range(p["n_net"]):
        pins = _pins(p, x, y, z, e, dz)
        W = _wbi_def(pins)
        for k, q in enumerate(pins):
            Wm = _wbi_def(pins, moved=k)
            exp[q[0]] += (4.0 / dz) * ((W - Wm) if q[1] else (Wm - W))
    r0 = o.wirelength(x, y, z, fd_mode=0)
    r1 = o.wirelength(x, y, z, fd_mode=1)
    np.testing.assert_allclose(r0["gfd"], exp, rtol=1e-13, atol=1e-12)
    assert np.array_equal(r0["gfd"], r1["gfd"])


def test_fd_incremental_equals_vanilla_on_workload():
    from paper_2403_09070_gb300 import synth
    p = synth.make_problem("cells_2k")
    o = Oracle(p)
    r0 = o.wirelength(p["x"], p["y"], p["z"], fd_mode=0)
    r1 = o.wirelength(p["x"], p["y"], p["z"], fd_mode=1)
    assert np.array_equal(r0["gfd"], r1["gfd"])


def test_incremental_figure_example():
    """Fig. incre-wl: moving p4 to the bottom die changes W_Bi by -0.5."""
    rows = read_golden("incremental_wl_example.txt")
    pts = [(r[0] == "top", float(r[1]), float(r[2])) for r in rows if r[0] in ("top", "bottom")]
    before = float(next(r for r in rows if r[0] == "before")[1])
    k, dW = next((int(r[1]), float(r[2])) for r in rows if r[0] == "move")
    n = len(pts)
    p = problem([(0.1, 0.1, 0.1, 0.1)] * n, nets=[list(range(n))], die=(-10, -10, 10, 10), grid=(4, 4, 2))
    dz = dz_of(p)
    x = [q[1] for q in pts]
    y = [q[2] for q in pts]
    z = [0.75 * dz if q[0] else 0.25 * dz for q in pts]
    o = Oracle(p)
    for mode in (0, 1):
        r = o.wirelength(x, y, z, fd_mode=mode)
        assert r["hpwl_d2d"] == pytest.approx(before, abs=1e-14)
        # p4 is on top: (4/d_z)(W(top) - W(bottom)) = -(4/d_z) * dW
        assert r["gfd"][k] == pytest.approx(-(4.0 / dz) * dW, abs=1e-13)


def test_normalisation_closed_form():
    """Four pins on the corners of an L x L square, two per die on opposite
    corners: every instance has |FD| = 8L/d_z, every |dW^/dx| = |dW^/dy| =
    tanh(u) + u sech^2(u) (u = L/2g, split branch), so eq. fda-normalize
    gives g = D d_z / (8 L) times the FD gradient."""
    L, gam = 2.0, 0.9
    p = problem([(0.1, 0.1, 0.1, 0.1)] * 4, nets=[[0, 1, 2, 3]], die=(0, 0, 10, 10), grid=(4, 4, 2),
                gamma=gam, lam=0.0)
    dz = dz_of(p)
    x = [3.0, 3.0 + L, 3.0, 3.0 + L]
    y = [3.0, 3.0 + L, 3.0 + L, 3.0]
    z = [0.75 * dz, 0.75 * dz, 0.25 * dz, 0.25 * dz]
    o = Oracle(p)
    w = o.wirelength(x, y, z)
    np.testing.assert_allclose(w["gfd"], [8 * L / dz, 8 * L / dz, -8 * L / dz, -8 * L / dz], rtol=1e-14)
    u = L / (2 * gam)
    D = math.tanh(u) + u / math.cosh(u) ** 2
    np.testing.assert_allclose(np.abs(w["gx"]), D, rtol=1e-13)
    np.testing.assert_allclose(np.abs(w["gy"]), D, rtol=1e-13)
    r = o.eval(x, y, z)
    assert r["Sx"] == pytest.approx(4 * D) and r["Sz"] == pytest.approx(32 * L / dz)
    assert r["g_scale"] == pytest.approx(D * dz / (8 * L), rel=1e-13)
    # lambda = 0: gz = g * FD + alpha * d p^(z)/dz
    np.testing.assert_allclose(r["gz"], r["g_scale"] * w["gfd"] + o.alpha * w["gwaz"], rtol=1e-13)
