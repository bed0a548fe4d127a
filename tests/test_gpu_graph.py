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
