"""GPU parity: the CUDA path (through the C ABI) against the oracle on the same
seeded inputs.  Bars: bit-exact fixed-point density map; FP64 path within
1e-9 relative; FP32 paths within 2e-5 relative on the objective and 1e-4
relative on the gradient L2 norm."""
import numpy as np
import pytest

from gpu_harness import Q, rel_l2, rel_max, run_gpu, run_oracle
from helpers import dz_of, problem
from paper_2403_09070_gb300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


def _check_fp64(prob, x, y, z, maps=True, flags=0, autotune=False):
    g = run_gpu(prob, x, y, z, "fp64", maps=maps, flags=flags, autotune=autotune)
    o, r = run_oracle(prob, x, y, z, g["alpha"], density_mode=1)
    if maps:
        q = o.density_fixed(x, y, z, use_float=False)
        assert np.array_equal(g["q"], q), "fixed-point density map differs"
        pe = o.poisson(q * Q)
        for k in ("ex", "ey", "ez"):
            assert rel_max(g[k], pe[k]) < TOL64, k
        w = o.wirelength(x, y, z)
        for k in ("gx", "gy", "gwaz", "gfd"):
            assert rel_max(g["wl"][k], w[k]) < TOL64, k
    res = g["res"]
    for k, kr in (("obj", "obj"), ("wl_bi", "wl_bi"), ("wl_z", "wl_z"), ("energy", "energy"),
                  ("hpwl_d2d", "hpwl_d2d"), ("g_scale", "g_scale"), ("s_x", "Sx"), ("s_y", "Sy"),
                  ("s_z", "Sz")):
        assert res[k] == pytest.approx(r[kr], rel=TOL64, abs=1e-300), k
    assert res["n_cross"] == r["n_cross"]
    for k in ("gx", "gy", "gz"):
        assert rel_max(g[k], r[k]) < TOL64, k
    return g, r


def _check_fp32(prob, x, y, z, precision="fp32", flags=0, autotune=False):
    x32, y32, z32 = (np.asarray(a, np.float32).astype(np.float64) for a in (x, y, z))
    g = run_gpu(prob, x32, y32, z32, precision, flags=flags, autotune=autotune)
    o, r = run_oracle(prob, x32, y32, z32, g["alpha"], density_mode=0)
    q = o.density_fixed(x32, y32, z32, use_float=True)
    assert np.array_equal(g["q"], q), "fixed-point density map (float contract) differs"
    res = g["res"]
    assert res["obj"] == pytest.approx(r["obj"], rel=2e-5)
    assert res["n_cross"] == r["n_cross"]
    for k in ("gx", "gy", "gz"):
        assert rel_l2(g[k], r[k]) < 1e-4, (k, rel_l2(g[k], r[k]))
    return g, r


@pytest.mark.parametrize("positions,origin", [("uniform", (0.0, 0.0)), ("center", (0.0, 0.0)),
                                              ("uniform", (137.0, -42.5))])
def test_fp64_cells_2k(positions, origin):
    p = synth.make_problem("cells_2k", positions=positions, origin=origin)
    _check_fp64(p, p["x"], p["y"], p["z"])


@pytest.mark.parametrize("positions", ["uniform", "center"])
def test_fp32_cells_2k(positions):
    p = synth.make_problem("cells_2k", positions=positions)
    _check_fp32(p, p["x"], p["y"], p["z"])


def test_fp64_cells_200k():
    p = synth.make_problem("cells_200k")
    _check_fp64(p, p["x"], p["y"], p["z"])


def test_fp32_cells_200k():
    p = synth.make_problem("cells_200k")
    _check_fp32(p, p["x"], p["y"], p["z"])


# ---------------- edge cases ----------------

def _edge(kind):
    rng = np.random.default_rng(hash(kind) % 2 ** 32)
    die = (3.0, -7.0, 3.0 + 74.0, -7.0 + 46.0)
    grid = (37, 23, 3)
    n = 120
    sizes = [(float(rng.integers(1, 9)), 1.0, 0.0, 0.0) for _ in range(n)]
    sizes = [(w, h, 0.8 * w, 0.8 * h) for (w, h, _, _) in sizes]
    macros = []
    nets = [list(rng.choice(n, size=int(rng.integers(2, 9)), replace=False)) for _ in range(150)]
    zf = []
    if kind in ("default", "outside", "zmid", "zfixed", "hifanout"):
        sizes += [(12.0, 9.0, 9.6, 7.2), (6.0, 6.0, 4.8, 4.8)]
        macros = [n, n + 1]
        nets += [[n, 3, 5, 7], [n + 1, n, 11]]
    if kind == "nonets":
        nets = []
    if kind == "hifanout":
        nets += [list(rng.choice(n, size=100, replace=False)),
                 list(range(n)) + [n, n + 1],  # 122 pins
                 [4], [9, 10]]
        grid = (40, 24, 2)
    if kind == "single":
        sizes, nets, macros = sizes[:1], [], []
    if kind == "nz1":
        grid = (16, 16, 1)
    if kind == "zfixed":
        zf = list(range(0, n, 5))
    ni = len(sizes)
    P_ = sum(len(e) for e in nets)
    off = np.zeros((P_, 4))
    off[:, 0] = rng.uniform(-0.5, 0.5, P_)
    off[:, 1] = rng.uniform(-0.5, 0.5, P_)
    off[:, 2] = 0.8 * off[:, 0]
    off[:, 3] = 0.8 * off[:, 1]
    p = problem(sizes, nets=nets, offsets=off, die=die, grid=grid, macros=macros, z_fixed=zf,
                gamma=4.0 * 74.0 / grid[0])
    dz = dz_of(p)
    x = rng.uniform(die[0] + 5, die[2] - 5, ni)
    y = rng.uniform(die[1] + 5, die[3] - 5, ni)
    z = rng.uniform(dz / 4, 3 * dz / 4, ni)
    if kind == "alltop":
        z[:] = 0.75 * dz
    if kind == "allbottom":
        z[:] = 0.25 * dz
    if kind == "zmid":
        z[::3] = dz / 2
    if kind == "outside":
        x[:10] = die[0] - 1.0
        x[10:20] = die[2] + 0.5
        x[n] = die[0] + 1.0  # macro hanging out of the region
    return p, x, y, z


EDGE = ["default", "nonets", "single", "alltop", "allbottom", "zmid", "outside", "hifanout", "nz1",
        "zfixed"]


@pytest.mark.parametrize("kind", EDGE)
def test_fp64_edge_cases(kind):
    p, x, y, z = _edge(kind)
    _check_fp64(p, x, y, z)


@pytest.mark.parametrize("kind", EDGE)
def test_fp32_edge_cases(kind):
    p, x, y, z = _edge(kind)
    _check_fp32(p, x, y, z)


def test_positions_from_device_tensors_and_device_gradients():
    """Device (torch CUDA) positions and gradients give the host results."""
    torch = pytest.importorskip("torch")
    from paper_2403_09070_gb300 import place3d as P
    p = synth.make_problem("cells_2k")
    ref = run_gpu(p, p["x"], p["y"], p["z"], "fp64", maps=False)
    with P.Place3D(p, precision="fp64", stream=torch.cuda.current_stream()) as h:
        xs = [torch.tensor(p[k], device="cuda", dtype=torch.float64) for k in ("x", "y", "z")]
        h.set_positions(*xs)
        gs = [torch.empty(p["n_inst"], device="cuda", dtype=torch.float64) for _ in range(3)]
        r = h.eval(*gs)
    # the wirelength sums use floating-point atomics: equal up to summation order
    assert r["obj"] == pytest.approx(ref["res"]["obj"], rel=1e-12)
    for t, k in zip(gs, ("gx", "gy", "gz")):
        np.testing.assert_allclose(t.cpu().numpy(), ref[k], rtol=1e-12, atol=1e-12 * np.abs(ref[k]).max())


@pytest.mark.parametrize("kind", ["default", "outside", "hifanout"])
@pytest.mark.parametrize("flags", [2, 4])  # Theorem 1 suffix-sum adjoint / direct bin-parallel gather
def test_macro_gather_forms(kind, flags):
    p, x, y, z = _edge(kind)
    _check_fp64(p, x, y, z, flags=flags)
    _check_fp32(p, x, y, z, flags=flags)


def test_macro_gather_forms_cells_2k():
    p = synth.make_problem("cells_2k")
    for flags in (2, 4):
        _check_fp64(p, p["x"], p["y"], p["z"], flags=flags)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotuned_forms_keep_parity(precision):
    """Every reduction form the autotuner may pick gives the oracle's result."""
    p = synth.make_problem("cells_200k")
    if precision == "fp64":
        g, _ = _check_fp64(p, p["x"], p["y"], p["z"], maps=False, autotune=True)
    else:
        g, _ = _check_fp32(p, p["x"], p["y"], p["z"], autotune=True)
    assert all(G * ppl >= d or (G, ppl, d) == (1, 1, 2) for d, G, ppl in g["forms"] if G > 0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_reduction_form(precision):
    """Each (lanes per net, pins per lane) form of every degree bucket gives
    the same wirelength parts as the oracle."""
    from paper_2403_09070_gb300 import place3d as P
    p, x, y, z = _edge("hifanout")
    rng = np.random.default_rng(3)
    n = p["n_inst"]
    dt = np.float64 if precision == "fp64" else np.float32
    xs = [np.asarray(a, dt) for a in (x, y, z)]
    ref = None
    with P.Place3D(p, precision=precision) as h:
        h.set_positions(*xs)
        forms = h.wl_forms()
        from oracle import Oracle
        w = Oracle(p, alpha=h.alpha).wirelength(*[a.astype(np.float64) for a in xs])
        for bi, (dmax, G, ppl) in enumerate(forms):
            if G == 0:
                continue
            for (g2, p2) in P.WL_FORMS:
                if (g2, p2) == (1, 1) and dmax != 2:
                    continue  # the closed-form kernel serves 2-pin nets only
                if g2 * p2 < dmax and (g2, p2) != (1, 1):
                    continue
                h.set_wl_form(bi, g2, p2)
                h.eval()
                parts = h.wl_parts()
                tol = 1e-9 if precision == "fp64" else 1e-4
                for k in ("gx", "gy", "gwaz", "gfd"):
                    assert rel_l2(parts[k], w[k]) < tol, (bi, g2, p2, k)
            h.set_wl_form(bi, G, ppl)


@pytest.mark.parametrize("kind", ["default", "outside", "hifanout", "zfixed", "nz1", "single", "nonets"])
def test_tiled_path_edge_cases(kind):
    """The tile-sorted scatter/gather (forced with PLACE3D_FLAG_TILES on these
    small problems, where the default is per cell) on the edge cases:
    bit-exact map, FP64 1e-9, FP32 bars."""
    p, x, y, z = _edge(kind)
    _check_fp64(p, x, y, z, flags=16)
    _check_fp32(p, x, y, z, flags=16)


@pytest.mark.parametrize("positions", ["uniform", "center"])
def test_tiled_path_cells_2k(positions):
    p = synth.make_problem("cells_2k", positions=positions)
    _check_fp64(p, p["x"], p["y"], p["z"], flags=16)
    _check_fp32(p, p["x"], p["y"], p["z"], flags=16)


@pytest.mark.parametrize("kind", ["default", "outside", "hifanout", "zfixed", "nz1"])
def test_per_cell_scatter_gather_path(kind):
    """The per-cell scatter/gather (PLACE3D_FLAG_NO_TILES: one thread per
    cell, global int64 atomics and field loads) matches the oracle like the
    default tile-sorted path (bit-exact map included)."""
    p, x, y, z = _edge(kind)
    _check_fp64(p, x, y, z, flags=32)
    _check_fp32(p, x, y, z, flags=32)


@pytest.mark.parametrize("positions", ["uniform", "center"])
def test_per_cell_path_cells_200k(positions):
    """The per-cell path at 256x256x4 with clustered and uniform cells."""
    p = synth.make_problem("cells_200k", positions=positions)
    _check_fp64(p, p["x"], p["y"], p["z"], maps=True, flags=32)
    _check_fp32(p, p["x"], p["y"], p["z"], flags=32)


def test_tiles_with_wide_cells():
    """A few cells 7 bins wide among 1-2-bin ones: the tile windows' halo
    grows to 4 bins and the map stays bit-exact."""
    rng = np.random.default_rng(3)
    die = (0.0, 0.0, 400.0, 300.0)
    grid = (80, 60, 2)
    n = 600
    sizes = [(float(rng.integers(1, 9)), 1.0, 0.0, 0.0) for _ in range(n)]
    sizes = [(w, h, 0.8 * w, 0.8 * h) for (w, h, _, _) in sizes]
    for k in range(0, n, 97):
        sizes[k] = (35.0, 2.0, 28.0, 1.6)  # 7 bins wide: halo 4
    nets = [list(rng.choice(n, size=int(rng.integers(2, 6)), replace=False)) for _ in range(700)]
    P_ = sum(len(e) for e in nets)
    p = problem(sizes, nets=nets, offsets=np.zeros((P_, 4)), die=die, grid=grid, gamma=20.0)
    dz = dz_of(p)
    x = rng.uniform(die[0], die[2], n)
    y = rng.uniform(die[1], die[3], n)
    z = rng.uniform(dz / 4, 3 * dz / 4, n)
    _check_fp64(p, x, y, z, flags=16)
    _check_fp32(p, x, y, z, flags=16)


def _with_big_nets(sizes=(300, 1500, 2004), seed=9):
    """cells_2k plus nets of the given pin counts on distinct instances (the
    largest covers every instance): nets above 128 pins are split into
    chunks of 1,024 pins, so these take one, two and two chunks."""
    p = synth.make_problem("cells_2k")
    rng = np.random.default_rng(seed)
    n = p["n_inst"]
    ns = list(np.asarray(p["net_start"], np.int64))
    pins = list(np.asarray(p["pin_inst"], np.int64))
    offs = [list(np.asarray(p[k], np.float64)) for k in ("off_bx", "off_by", "off_tx", "off_ty")]
    for d in sizes:
        inst = rng.choice(n, size=d, replace=False)
        ox = rng.uniform(-0.5, 0.5, d)
        oy = rng.uniform(-0.4, 0.4, d)
        pins += list(inst)
        for lst, v in zip(offs, (ox, oy, 0.8 * ox, 0.8 * oy)):
            lst += list(v)
        ns.append(ns[-1] + d)
    q = dict(p)
    q["net_start"] = np.asarray(ns, np.int32)
    q["pin_inst"] = np.asarray(pins, np.int32)
    for k, lst in zip(("off_bx", "off_by", "off_tx", "off_ty"), offs):
        q[k] = np.asarray(lst, np.float64)
    q["n_net"] = len(ns) - 1
    q["n_pin"] = int(ns[-1])
    return q


def test_high_fanout_nets_split_across_blocks():
    """Nets of 300, 1,500 and 2,004 pins, each split into 1,024-pin chunks
    handled by separate blocks whose partial extremes and WA sums are merged
    per net: FP64 within 1e-9 of the oracle (incremental FD included, which
    needs the exact 1st/2nd extremes across chunks), FP32 within its bar."""
    q = _with_big_nets()
    _check_fp64(q, q["x"], q["y"], q["z"])
    _check_fp32(q, q["x"], q["y"], q["z"])


# ---- dummy fillers (Sec. III-A): pinless instances, z-fixed ones with a zero z-gradient ----
def _with_fillers(wl, u, positions, seed=5):
    from oracle import Oracle
    p = synth.make_problem(wl, positions=positions)
    fp = Oracle(p).filler_plan(p["z"], *u)  # counts from the oracle's plan
    return synth.append_fillers(p, fp, seed=seed, positions=positions)


@pytest.mark.parametrize("positions", ["center", "uniform"])
def test_fillers_cells_2k_fp64(positions):
    q = _with_fillers("cells_2k", (0.8, 0.7), positions)
    g, r = _check_fp64(q, q["x"], q["y"], q["z"])
    zf = q["z_fixed"].astype(bool)
    assert zf.sum() > 1000 and np.all(g["gz"][zf] == 0.0)
    assert np.abs(g["gx"][q["fillers"]["first"]:]).max() > 0  # fillers feel the field


@pytest.mark.parametrize("positions", ["center", "uniform"])
def test_fillers_cells_2k_fp32(positions):
    q = _with_fillers("cells_2k", (0.8, 0.7), positions)
    g, r = _check_fp32(q, q["x"], q["y"], q["z"])
    assert np.all(g["gz"][q["z_fixed"].astype(bool)] == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_tc"])
@pytest.mark.parametrize("positions", ["center", "uniform"])
def test_density_overflow(precision, positions):
    """The overflow by-product (sum of max(rho - 1, 0) over the sum of rho,
    target density 1) against its definition on the oracle's fixed-point map."""
    wl = "cells_200k" if precision == "fp32_tc" else "cells_2k"
    p = synth.make_problem(wl, positions=positions)
    dt = np.float64 if precision == "fp64" else np.float32
    x, y, z = (np.asarray(p[k], dt).astype(np.float64) for k in ("x", "y", "z"))
    g = run_gpu(p, x, y, z, precision, maps=False)
    from oracle import Oracle
    rho = Oracle(p).density_fixed(x, y, z, use_float=precision != "fp64") * Q
    expect = np.maximum(rho - 1.0, 0.0).sum() / rho.sum()
    assert g["res"]["overflow"] == pytest.approx(expect, rel=1e-10 if precision == "fp64" else 1e-5, abs=1e-12)
    if positions == "center":
        assert g["res"]["overflow"] > 0.05  # the clustered start overflows
