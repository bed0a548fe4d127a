"""CUDA-graph evaluation and batches of independent instances in one graph
launch (batching row): results equal the plain evaluation's."""
import numpy as np
import pytest

from paper_2403_09070_gb300 import place3d as P
from paper_2403_09070_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _plain(p, precision, x, y, z):
    dt = np.float64 if precision == "fp64" else np.float32
    with P.Place3D(p, precision=precision) as h:
        h.set_positions(*(np.asarray(a, dt) for a in (x, y, z)))
        g = [np.zeros(p["n_inst"], dt) for _ in range(3)]
        r = h.eval(*g)
    return r, g


@pytest.mark.parametrize("precision,wl", [("fp64", "cells_2k"), ("fp32_tc", "cells_200k")])
def test_eval_graph_replays_with_new_positions(precision, wl):
    p = synth.make_problem(wl)
    dt = torch.float64 if precision == "fp64" else torch.float32
    h = P.Place3D(p, precision=precision, stream=torch.cuda.current_stream())
    xyz = [torch.tensor(p[k], device="cuda", dtype=dt) for k in ("x", "y", "z")]
    g = [torch.empty(p["n_inst"], device="cuda", dtype=dt) for _ in range(3)]
    rng = np.random.default_rng(5)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for it in range(3):
        if it:
            x, y, z = synth.draw_positions(rng, p, "uniform")
            for t, a in zip(xyz, (x, y, z)):
                t.copy_(torch.as_tensor(a, dtype=dt))
        h.eval_graph(*xyz, *g)
        r = h.get_result()
        ref, gref = _plain(p, precision, *(t.cpu().numpy() for t in xyz))
        assert r["obj"] == pytest.approx(ref["obj"], rel=tol)
        for a, b in zip(g, gref):
            np.testing.assert_allclose(a.cpu().numpy(), b, rtol=tol, atol=tol * np.abs(b).max())
    h.close()


def test_batch_of_uneven_instances_in_one_graph():
    probs = synth.make_batch(count=6, seed=7, n_min=3000, n_max=40000)
    hs, xyz, gs = [], [], []
    for p in probs:
        prec = "fp32_tc" if p["nx"] % 128 == 0 else "fp32"
        hs.append(P.Place3D(p, precision=prec))
        xyz.append([torch.tensor(p[k], device="cuda", dtype=torch.float32) for k in ("x", "y", "z")])
        gs.append([torch.empty(p["n_inst"], device="cuda", dtype=torch.float32) for _ in range(3)])
    b = P.Batch(hs)
    for rep in range(2):
        b.eval(*[[v[k] for v in xyz] for k in range(3)], *[[v[k] for v in gs] for k in range(3)])
        torch.cuda.synchronize()
        assert b.shared_stages() == 1  # the wirelength stage: one launch per stage for all instances
        for p, h, v, g in zip(probs, hs, xyz, gs):
            prec = "fp32_tc" if p["nx"] % 128 == 0 else "fp32"
            r = h.get_result()
            ref, gref = _plain(p, prec, *(t.cpu().numpy() for t in v))
            assert r["obj"] == pytest.approx(ref["obj"], rel=1e-5)
            for a, c in zip(g, gref):
                np.testing.assert_allclose(a.cpu().numpy(), c, rtol=1e-4, atol=1e-4 * np.abs(c).max())
    b.close()
    for h in hs:
        h.close()


def test_batch_sees_set_params_of_one_instance():
    """A batch graph captured before place3d_set_params on one of its handles
    evaluates that instance with the new gamma and lambda, the others
    unchanged."""
    probs = synth.make_batch(count=3, seed=11, n_min=3000, n_max=8000)
    hs = [P.Place3D(p, precision="fp32") for p in probs]
    xyz = [[torch.tensor(p[k], device="cuda", dtype=torch.float32) for k in ("x", "y", "z")] for p in probs]
    gs = [[torch.empty(p["n_inst"], device="cuda", dtype=torch.float32) for _ in range(3)] for p in probs]
    b = P.Batch(hs)
    args = [[v[k] for v in xyz] for k in range(3)] + [[v[k] for v in gs] for k in range(3)]
    b.eval(*args)
    torch.cuda.synchronize()
    before = [h.get_result()["obj"] for h in hs]
    p1 = probs[1]
    hs[1].set_params(gamma=1.5 * p1["gamma"], gamma_z=0.0, alpha=hs[1].alpha, lam=3 * p1["lam"])
    b.eval(*args)
    torch.cuda.synchronize()
    for i, (p, h, v, g) in enumerate(zip(probs, hs, xyz, gs)):
        r = h.get_result()
        with P.Place3D(p, precision="fp32") as hr:
            if i == 1:
                hr.set_params(gamma=1.5 * p["gamma"], gamma_z=0.0, alpha=hr.alpha, lam=3 * p["lam"])
            hr.set_positions(*(t.cpu().numpy() for t in v))
            gref = [np.zeros(p["n_inst"], np.float32) for _ in range(3)]
            ref = hr.eval(*gref)
        assert r["obj"] == pytest.approx(ref["obj"], rel=1e-5)
        if i != 1:
            assert r["obj"] == pytest.approx(before[i], rel=1e-6)
        else:
            assert abs(r["obj"] - before[i]) > 1e-3 * abs(before[i])
        for a, c in zip(g, gref):
            np.testing.assert_allclose(a.cpu().numpy(), c, rtol=1e-4, atol=1e-4 * np.abs(c).max())
    b.close()
    for h in hs:
        h.close()


def test_autotuned_plan_keeps_results_and_transfers():
    """place3d_autotune regroups the degree classes and picks the forms and
    the tensor-core tile widths (comparing candidate plans by whole
    evaluations at the current positions, which get_result then reports);
    the results stay those of the default plan
    (up to summation order), and the plan set on a second handle
    (place3d_set_wl_plan, place3d_set_tc_tiles) reproduces them."""
    p = synth.make_problem("cells_200k")
    x, y, z = (np.asarray(p[k], np.float32) for k in ("x", "y", "z"))
    n = p["n_inst"]
    with P.Place3D(p, precision="fp32_tc") as h:
        h.set_positions(x, y, z)
        g0 = [np.zeros(n, np.float32) for _ in range(3)]
        r0 = h.eval(*g0)
        default = h.wl_forms()
        h.autotune(1)
        ra = h.get_result()  # the autotuner's timed evaluations at these positions
        plan, tiles = h.wl_forms(), h.tc_tiles()
        g1 = [np.zeros(n, np.float32) for _ in range(3)]
        r1 = h.eval(*g1)
    maxdeg = int(np.diff(p["net_start"]).max())
    assert [f[0] for f in default][:5] == [2, 4, 8, 16, 32] and default[-1][0] == maxdeg
    assert len(tiles) == 4 and set(tiles) <= {64, 128}
    assert plan[-1][0] == default[-1][0]  # every degree is covered
    assert r1["obj"] == pytest.approx(r0["obj"], rel=1e-5)
    assert ra["obj"] == pytest.approx(r0["obj"], rel=1e-5)
    for a, b in zip(g1, g0):
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-4 * np.abs(b).max())
    with P.Place3D(p, precision="fp32_tc") as h2:
        h2.set_wl_plan(plan)
        h2.set_tc_tiles(tiles)
        assert h2.wl_forms() == plan and h2.tc_tiles() == tiles
        h2.set_positions(x, y, z)
        g2 = [np.zeros(n, np.float32) for _ in range(3)]
        r2 = h2.eval(*g2)
        assert r2["obj"] == pytest.approx(r1["obj"], rel=1e-6)
        with pytest.raises(P.Place3DError):
            h2.set_wl_plan([(3, 1, 4)])  # leaves classes uncovered
        with pytest.raises(P.Place3DError):
            h2.set_tc_tiles([64, 96, 64, 64])
        h2.set_wl_plan([])
        assert h2.wl_forms() == default


@pytest.mark.parametrize("cols", [[64, 64, 64, 64], [128, 128, 128, 128], [128, 64, 64, 128]])
def test_tensor_core_tile_widths_agree(cols):
    """Every tile width of the tensor-core products gives the same fields."""
    p = synth.make_problem("cells_200k")
    x, y, z = (np.asarray(p[k], np.float32) for k in ("x", "y", "z"))
    out = []
    for c in ([64, 64, 64, 64], cols):
        with P.Place3D(p, precision="fp32_tc") as h:
            h.set_tc_tiles(c)
            h.set_positions(x, y, z)
            r = h.eval()
            out.append((r["energy"], h.copy_map(P.MAP_EX)))
    assert out[1][0] == pytest.approx(out[0][0], rel=1e-6)
    np.testing.assert_allclose(out[1][1], out[0][1], rtol=1e-5, atol=1e-5 * np.abs(out[0][1]).max())


def test_fp64_batch_runs_each_instance_on_its_own():
    """An FP64 batch has no shared stage (each instance's graph branch runs
    its whole evaluation) and equals the plain evaluations."""
    probs = synth.make_batch(count=3, seed=13, n_min=3000, n_max=9000)
    hs = [P.Place3D(p, precision="fp64") for p in probs]
    xyz = [[torch.tensor(p[k], device="cuda", dtype=torch.float64) for k in ("x", "y", "z")] for p in probs]
    gs = [[torch.empty(p["n_inst"], device="cuda", dtype=torch.float64) for _ in range(3)] for p in probs]
    b = P.Batch(hs)
    b.eval(*[[v[k] for v in xyz] for k in range(3)], *[[v[k] for v in gs] for k in range(3)])
    torch.cuda.synchronize()
    assert b.shared_stages() == 0
    for p, h, v, g in zip(probs, hs, xyz, gs):
        ref, gref = _plain(p, "fp64", *(t.cpu().numpy() for t in v))
        assert h.get_result()["obj"] == pytest.approx(ref["obj"], rel=1e-10)
        for a, c in zip(g, gref):
            np.testing.assert_allclose(a.cpu().numpy(), c, rtol=1e-10, atol=1e-10 * np.abs(c).max())
    b.close()
    for h in hs:
        h.close()
