"""Pins of the oracle's density map (eq. density-map-accum, Theorem 1, the
fixed-point replica) against the paper's worked example, Theorem 1 itself,
closed forms, invariants and brute force."""
import math

import numpy as np
import pytest

from helpers import dz_of, problem, read_golden
from oracle import Oracle

Q = 2.0 ** -36


def _prefix_case():
    rows = read_golden("prefix_example.txt")
    g = next(r for r in rows if r[0] == "grid")
    nx, ny = int(g[1]), int(g[2])
    x0, y0, w, h = (float(v) for v in next(r for r in rows if r[0] == "macro")[1:])
    A = np.zeros((ny, nx))
    rho = np.zeros((ny, nx))
    for r in rows:
        if r[0] == "A":
            A[int(r[2]), int(r[1])] = float(r[3])
        elif r[0] == "rho":
            rho[int(r[2]), int(r[1])] = float(r[3])
    # 3D case with N_z = 2: the macro's depth d_z/2 is exactly layer 0 at z = d_z/4
    p = problem([(w, h, w, h)], die=(0.0, 0.0, float(nx), float(ny)), grid=(nx, ny, 2), macros=[0])
    x, y, z = [x0 + w / 2], [y0 + h / 2], [dz_of(p) / 4]
    return p, (x, y, z), A, rho


def test_prefix_example_corner_map():
    """Fig. prefix-example: A_v printed values (layer 0) and its z-mirror."""
    p, xyz, A, _ = _prefix_case()
    o = Oracle(p)
    Am = o.macro_corner_map(*xyz)
    np.testing.assert_allclose(Am[0], A, atol=1e-12)
    np.testing.assert_allclose(Am[1], -A, atol=1e-12)


def test_prefix_example_density():
    """Fig. prefix-example: prefix sum of A_v, the direct overlap and the
    fixed-point replica all give the printed density map."""
    p, xyz, _, rho = _prefix_case()
    o = Oracle(p)
    P = Oracle.prefix_sum3(o.macro_corner_map(*xyz))
    np.testing.assert_allclose(P[0], rho, atol=1e-12)
    np.testing.assert_allclose(P[1], 0.0, atol=1e-12)
    D = o.density_direct(*xyz)
    np.testing.assert_allclose(D[0], rho, atol=1e-12)
    np.testing.assert_allclose(D[1], 0.0, atol=1e-12)
    for use_float, tol in ((False, 64 * Q), (True, 1e-6)):
        F = o.density_fixed(*xyz, use_float=use_float) * Q
        np.testing.assert_allclose(F[0], rho, atol=tol)
        np.testing.assert_allclose(F[1], 0.0, atol=tol)


def _random_macros(rng, grid, n, die, outside=False):
    sizes, xs, ys = [], [], []
    for _ in range(n):
        wb, hb = rng.uniform(1.0, 0.5 * die[2]), rng.uniform(1.0, 0.5 * die[3])
        sizes.append((wb, hb, 0.8 * wb, 1.2 * hb))
        lo = -0.3 * wb if outside else 0.5 * wb
        xs.append(rng.uniform(lo, die[2] - lo))
        ys.append(rng.uniform(-0.3 * hb if outside else 0.5 * hb, die[3] - (-0.3 * hb if outside else 0.5 * hb)))
    p = problem(sizes, die=die, grid=grid, macros=range(n))
    dz = dz_of(p)
    zs = rng.uniform(dz / 4, 3 * dz / 4, n)
    return p, (np.array(xs), np.array(ys), zs)


@pytest.mark.parametrize("grid,outside", [((7, 5, 3), False), ((9, 11, 2), True), ((16, 16, 4), True)])
def test_theorem1_random_macros(grid, outside):
    """Theorem 1: prefix sum of the 8-corner map == direct cuboid/bin overlap."""
    rng = np.random.default_rng(7 + grid[0])
    die = (0.0, 0.0, 3.0 * grid[0], 2.0 * grid[1])
    p, xyz = _random_macros(rng, grid, 6, die, outside)
    o = Oracle(p)
    P = Oracle.prefix_sum3(o.macro_corner_map(*xyz))
    D = o.density_direct(*xyz)
    np.testing.assert_allclose(P, D, atol=1e-12)


def test_single_cell_closed_form():
    """A 0.5 x 0.5 cell centred on a bin corner of unit bins: stretched to
    sqrt2 x sqrt2 with omega = (0.5/sqrt2)^2, so each of the 4 bins gets
    omega * (sqrt2/2)^2 = 1/16, on the one layer the cell fills."""
    p = problem([(0.5, 0.5, 0.5, 0.5)], die=(0, 0, 8, 8), grid=(8, 8, 2))
    o = Oracle(p)
    D = o.density_direct([2.0], [3.0], [dz_of(p) / 4])
    exp = np.zeros((2, 8, 8))
    exp[0, 2:4, 1:3] = 1.0 / 16
    np.testing.assert_allclose(D, exp, atol=1e-14)
    a = o.attributes([2.0], [3.0], [dz_of(p) / 4])
    assert a["omega"][0] == pytest.approx(0.125, abs=1e-15)


def test_total_charge_per_die():
    """sum_b rho_b vol(b) over each die's layers = sum of w h d_z/2 of the
    instances on that die (local smoothness preserves charge), for instances
    inside the region with z at d_z/4 or 3 d_z/4."""
    rng = np.random.default_rng(3)
    n, nmac = 300, 3
    die = (0.0, 0.0, 60.0, 40.0)
    sizes = [(float(rng.integers(1, 9)), 1.0, 0.8 * 0, 0) for _ in range(n)]
    sizes = [(w, 1.0, 0.8 * w, 0.8) for (w, _, _, _) in sizes]
    sizes += [(8.0, 6.0, 6.4, 4.8)] * nmac
    p = problem(sizes, die=die, grid=(24, 16, 4), macros=range(n, n + nmac))
    dz = dz_of(p)
    wb = 60.0 / 24
    margin = 8.0 + 2 * wb
    x = rng.uniform(margin, die[2] - margin, n + nmac)
    y = rng.uniform(margin, die[3] - margin, n + nmac)
    top = rng.random(n + nmac) < 0.5
    z = np.where(top, 0.75 * dz, 0.25 * dz)
    o = Oracle(p)
    g = o.geometry()
    volb = g["wb"] * g["hb"] * g["db"]
    w = np.where(top, p["w_top"], p["w_bot"])
    h = np.where(top, p["h_top"], p["h_bot"])
    # the fixed-point map carries rounding residuals of a few 2^-36 per bin
    for rho, tol in ((o.density_direct(x, y, z), 1e-12), (o.density_fixed(x, y, z, False) * Q, 1e-9)):
        bot_charge = rho[:2].sum() * volb
        top_charge = rho[2:].sum() * volb
        assert bot_charge == pytest.approx(float((w * h * dz / 2)[~top].sum()), rel=tol)
        assert top_charge == pytest.approx(float((w * h * dz / 2)[top].sum()), rel=tol)


def test_prefix_sum3_brute_force():
    """Eq. def-prefix-sum-3d by the triple sum, int64 and float64."""
    rng = np.random.default_rng(0)
    a = rng.integers(-50, 50, size=(3, 4, 5)).astype(np.int64)
    b = rng.normal(size=(3, 4, 5))
    for arr in (a, b):
        got = Oracle.prefix_sum3(arr)
        exp = np.zeros_like(arr)
        for k in range(3):
            for j in range(4):
                for i in range(5):
                    exp[k, j, i] = arr[:k + 1, :j + 1, :i + 1].sum()
        if arr.dtype == np.int64:
            assert np.array_equal(got, exp)
        else:
            np.testing.assert_allclose(got, exp, atol=1e-12)


def test_fixed_replica_close_to_direct():
    """The quantised map differs from the exact map by rounding only."""
    from paper_2403_09070_gb300 import synth
    p = synth.make_problem("cells_2k")
    o = Oracle(p)
    D = o.density_direct(p["x"], p["y"], p["z"])
    Fd = o.density_fixed(p["x"], p["y"], p["z"], False) * Q
    Ff = o.density_fixed(p["x"], p["y"], p["z"], True) * Q
    assert np.abs(Fd - D).max() < 1e-8
    assert np.abs(Ff - D).max() < 1e-4 * max(1.0, D.max())
    assert abs(Fd.sum() - D.sum()) < 1e-6


def test_macro_size_and_partition():
    """Eq. macro-size-tech: bottom size at d_z/4, top size at 3 d_z/4, the
    mean at d_z/2; eq. std-size-tech: a cell at exactly d_z/2 is bottom."""
    p = problem([(10.0, 6.0, 8.0, 4.0), (3.0, 1.0, 2.4, 0.8)], die=(0, 0, 40, 40), grid=(8, 8, 2),
                macros=[0])
    o = Oracle(p)
    dz = dz_of(p)
    for zz, wm, hm, wc, dc in ((dz / 4, 10.0, 6.0, 3.0, 0), (3 * dz / 4, 8.0, 4.0, 2.4, 1),
                               (dz / 2, 9.0, 5.0, 3.0, 0)):
        a = o.attributes([20.0, 20.0], [20.0, 20.0], [zz, zz])
        assert a["w"][0] == pytest.approx(wm) and a["h"][0] == pytest.approx(hm)
        assert a["w"][1] == pytest.approx(wc) and a["delta"][1] == dc
