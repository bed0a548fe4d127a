"""GPU parity of the multi-die 2D mode (eq. 2d-place) through the C ABI
against the oracle: bit-exact fixed-point layer maps, FP64 within 1e-9, FP32
and FP32_TC within 2e-5 (objective) and 1e-4 (gradient L2); HBT pins in
both partial nets, per-layer weights, high-fanout nets, and CUDA graphs
that see a parameter change made after their capture."""
import numpy as np
import pytest

from gpu_harness import rel_l2, rel_max
from oracle import Oracle
from paper_2403_09070_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LAM = (2e-3, 5e-3, 1e-2)


def _problem2d(wl="cells_2k", seed=3, big_net=0, **kw):
    p = synth.make_problem(wl, **kw)
    if big_net:
        # one extra net over big_net distinct instances (a high-fanout, crossing net)
        rng = np.random.default_rng(seed)
        ins = rng.choice(p["n_inst"], big_net, replace=False).astype(np.int32)
        p["pin_inst"] = np.concatenate([p["pin_inst"], ins])
        p["net_start"] = np.concatenate([p["net_start"], [p["net_start"][-1] + big_net]]).astype(np.int32)
        for k in ("off_bx", "off_by", "off_tx", "off_ty"):
            p[k] = np.concatenate([p[k], np.zeros(big_net)])
        p["n_net"] += 1
        p["n_pin"] += big_net
    return synth.to_problem2d(p, seed=seed, lam_layer=LAM)


def _run(q, precision, pos=None, flags=0):
    from paper_2403_09070_gb300 import place3d as P
    dt = np.float64 if precision == "fp64" else np.float32
    x, y, z = (np.asarray(q[k] if pos is None else pos[i], dt) for i, k in enumerate(("x", "y", "z")))
    with P.Place3D(q, precision=precision, flags=flags) as h:
        h.set_positions(x, y, z)
        g = [np.zeros(q["n_inst"], dt) for _ in range(3)]
        r = h.eval(*g)
        qmap = h.copy_map(P.MAP_RHO_FIXED)
    return r, g, qmap, [a.astype(np.float64) for a in (x, y, z)]


def _check(q, precision, flags=0):
    r, g, qmap, (x, y, z) = _run(q, precision, flags=flags)
    o = Oracle(q)
    assert np.array_equal(qmap, o.density_fixed(x, y, z, use_float=precision != "fp64")), "2D fixed-point maps"
    if precision == "fp64":
        ref = o.eval2d(x, y, z, density_mode=1)
        for k, kr in (("obj", "obj"), ("wl_bi", "wl"), ("hpwl_d2d", "hpwl_d2d")):
            assert r[k] == pytest.approx(ref[kr], rel=1e-9), k
        for l, kr in enumerate(("e_bot", "e_top", "e_hbt")):
            assert r["energy_layer"][l] == pytest.approx(ref[kr], rel=1e-9), kr
        assert rel_max(g[0], ref["gx"]) < 1e-9 and rel_max(g[1], ref["gy"]) < 1e-9
    else:
        ref = o.eval2d(x, y, z, density_mode=0)
        assert r["obj"] == pytest.approx(ref["obj"], rel=2e-5)
        assert r["hpwl_d2d"] == pytest.approx(ref["hpwl_d2d"], rel=1e-6)
        for l, kr in enumerate(("e_bot", "e_top", "e_hbt")):
            assert r["energy_layer"][l] == pytest.approx(ref[kr], rel=1e-4), kr
        assert rel_l2(g[0], ref["gx"]) < 1e-4 and rel_l2(g[1], ref["gy"]) < 1e-4
    assert r["n_cross"] == ref["n_cross"] == len(q["hbt_nets"])
    assert np.all(g[2] == 0)  # the partition is fixed: no z-gradient
    hbt = q["is_hbt"].astype(bool)
    assert np.abs(g[0][hbt]).max() > 0  # HBTs feel both partial nets and their layer
    return r, g


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_2d_cells_2k(precision):
    _check(_problem2d(), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_2d_tiled_density_path(precision):
    """The tile-sorted scatter and gather forced in 2D mode (PLACE3D_FLAG_TILES;
    the default there is per cell): every instance in one layer, HBTs on the
    third, the same maps and gradients."""
    _check(_problem2d(), precision, flags=16)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_2d_high_fanout_net(precision):
    q = _problem2d(big_net=300)
    assert np.diff(q["net_start"]).max() > 128  # the block form's bucket
    _check(q, precision)


def test_2d_cells_200k_tensor_cores():
    _check(_problem2d("cells_200k", seed=5), "fp32_tc")


def test_2d_layer_weights_seen_by_captured_graph():
    """set_layer_weights changes the objective by the weighted layer
    energies, and a graph captured before the change picks the new weights
    up (the weights are read from device memory at run time)."""
    from paper_2403_09070_gb300 import place3d as P
    q = _problem2d()
    n = q["n_inst"]
    xyz = [torch.tensor(q[k], device="cuda", dtype=torch.float64) for k in ("x", "y", "z")]
    gs = [torch.empty(n, device="cuda", dtype=torch.float64) for _ in range(3)]
    with P.Place3D(q, precision="fp64") as h:
        h.eval_graph(*xyz, *gs)
        r1 = h.get_result()
        h.set_layer_weights(0.0, 0.0, 0.0)
        h.eval_graph(*xyz, *gs)
        r0 = h.get_result()
        assert r0["obj"] == pytest.approx(r0["wl_bi"], rel=1e-12)
        assert r1["obj"] == pytest.approx(r0["wl_bi"] + sum(l * e for l, e in zip(LAM, r0["energy_layer"])),
                                          rel=1e-12)


def test_graph_sees_set_params():
    """3D mode: a graph captured before place3d_set_params evaluates with the
    new gamma and lambda afterwards (gamma is a kernel argument: the graph is
    re-captured and updated in place at its next launch; lambda is read from
    device memory)."""
    from paper_2403_09070_gb300 import place3d as P
    p = synth.make_problem("cells_2k")
    n = p["n_inst"]
    xyz = [torch.tensor(p[k], device="cuda", dtype=torch.float64) for k in ("x", "y", "z")]
    gs = [torch.empty(n, device="cuda", dtype=torch.float64) for _ in range(3)]
    with P.Place3D(p, precision="fp64") as h:
        h.eval_graph(*xyz, *gs)
        h.set_params(gamma=2.0 * p["gamma"], gamma_z=0.0, alpha=h.alpha, lam=5 * p["lam"])
        h.eval_graph(*xyz, *gs)
        rg = h.get_result()
        gg = [t.cpu().numpy() for t in gs]
        h.set_positions(*xyz)
        ge = [np.zeros(n) for _ in range(3)]
        re = h.eval(*ge)
    assert rg["obj"] == pytest.approx(re["obj"], rel=1e-12)
    for a, b in zip(gg, ge):
        assert rel_max(a, b) < 1e-12


def test_2d_result_to_device_matches_host_result():
    from paper_2403_09070_gb300 import place3d as P
    q = _problem2d()
    with P.Place3D(q, precision="fp32") as h:
        h.set_positions(*(np.asarray(q[k], np.float32) for k in ("x", "y", "z")))
        r = h.eval(*[np.zeros(q["n_inst"], np.float32) for _ in range(3)])
        dev = torch.zeros(10, dtype=torch.float64, device="cuda")
        h.result_to_device(dev)
        v = dev.cpu().numpy()
    keys = ("obj", "wl_bi", "wl_z", "energy", "hpwl_d2d", "n_cross")
    for k, got in zip(keys, v[:6]):
        assert got == pytest.approx(r[k], rel=1e-12), k
    assert r["energy"] == pytest.approx(sum(r["energy_layer"]), rel=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_2d_one_die_no_hbts(precision):
    """Every instance on the bottom die: no crossing net, no HBT, the top and
    HBT layers empty (zero energy), each net one partial net."""
    p = synth.make_problem("cells_2k")
    zlo, _ = synth.depth_range(p)
    q = synth.to_problem2d(p, z=np.full(p["n_inst"], zlo), lam_layer=LAM)
    assert len(q["hbt_nets"]) == 0 and q["n_inst"] == p["n_inst"]
    r, g, qmap, (x, y, z) = _run(q, precision)
    o = Oracle(q)
    assert np.array_equal(qmap, o.density_fixed(x, y, z, use_float=precision != "fp64"))
    ref = o.eval2d(x, y, z, density_mode=1 if precision == "fp64" else 0)
    tol = 1e-9 if precision == "fp64" else 2e-5
    assert r["obj"] == pytest.approx(ref["obj"], rel=tol)
    assert r["n_cross"] == 0 and r["energy_layer"][1] == 0 and r["energy_layer"][2] == 0
    assert r["energy_layer"][0] > 0
    assert rel_l2(g[0], ref["gx"]) < (1e-9 if precision == "fp64" else 1e-4)


def test_lambda_change_keeps_graph_gamma_change_recaptures():
    """A new lambda is read from device memory by the captured graph (no new
    capture, results equal a fresh plain evaluation); a new gamma re-captures
    once."""
    from paper_2403_09070_gb300 import place3d as P
    p = synth.make_problem("cells_2k")
    n = p["n_inst"]
    xyz = [torch.tensor(p[k], device="cuda", dtype=torch.float64) for k in ("x", "y", "z")]
    gs = [torch.empty(n, device="cuda", dtype=torch.float64) for _ in range(3)]

    def plain(gamma, lam):
        with P.Place3D(dict(p, gamma=gamma, lam=lam), precision="fp64") as hp:
            hp.set_positions(*xyz)
            g = [np.zeros(n) for _ in range(3)]
            return hp.eval(*g), g

    with P.Place3D(p, precision="fp64") as h:
        h.eval_graph(*xyz, *gs)
        c0 = h.graph_captures()
        for lam in (3 * p["lam"], 10 * p["lam"]):
            h.set_params(gamma=p["gamma"], gamma_z=0.0, alpha=h.alpha, lam=lam)
            h.eval_graph(*xyz, *gs)
            r, g = h.get_result(), [t.cpu().numpy() for t in gs]
            assert h.graph_captures() == c0
            rp, gp = plain(p["gamma"], lam)
            assert r["obj"] == pytest.approx(rp["obj"], rel=1e-12)
            for a, b in zip(g, gp):
                assert rel_max(a, b) < 1e-12
        h.set_params(gamma=2 * p["gamma"], gamma_z=0.0, alpha=h.alpha, lam=lam)
        h.eval_graph(*xyz, *gs)
        assert h.graph_captures() == c0 + 1
        rp, _ = plain(2 * p["gamma"], lam)
        assert h.get_result()["obj"] == pytest.approx(rp["obj"], rel=1e-12)
