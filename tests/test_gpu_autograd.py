"""Differentiation row: the torch.autograd wrapper, central finite differences
on 64 sampled coordinates at the 1M-cell workload, and a Nesterov placement
loop with the 3D mixed-size preconditioner (eq. improved-precond)."""
import numpy as np
import pytest

from paper_2403_09070_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autograd_matches_eval_gradient():
    from paper_2403_09070_gb300 import place3d as P
    from paper_2403_09070_gb300.autograd import Place3DObjective
    p = synth.make_problem("cells_2k")
    m = Place3DObjective(p, precision="fp64")
    xyz = [torch.tensor(p[k], device="cuda", dtype=torch.float64, requires_grad=True) for k in ("x", "y", "z")]
    f = m(*xyz)
    (3.0 * f).backward()
    with P.Place3D(p, precision="fp64", alpha=m.alpha) as h:
        h.set_positions(*[t.detach() for t in xyz])
        g = [np.zeros(p["n_inst"]) for _ in range(3)]
        r = h.eval(*g)
    assert float(f.detach()) == pytest.approx(r["obj"], rel=1e-12)
    for t, ref in zip(xyz, g):
        np.testing.assert_allclose(t.grad.cpu().numpy(), 3.0 * ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    s = m.last_scalars()
    assert s["wl_bi"] == pytest.approx(r["wl_bi"], rel=1e-12)


def test_finite_differences_64_coordinates_1m():
    """x and y gradients of the wirelength objective (lambda = 0: the density
    gradient is a field gather by design) against central differences of the
    forward, FP64 path, 1M cells, 64 sampled instances."""
    from paper_2403_09070_gb300.autograd import Place3DObjective
    p = synth.make_problem("cells_1m")
    m = Place3DObjective(p, precision="fp64")
    m.set_params(lam=0.0)
    xyz = [torch.tensor(p[k], device="cuda", dtype=torch.float64, requires_grad=True) for k in ("x", "y", "z")]
    f = m(*xyz)
    f.backward()
    grads = [t.grad.clone() for t in xyz]
    rng = np.random.default_rng(64)
    deg = np.bincount(np.asarray(p["pin_inst"]), minlength=p["n_inst"])
    cand = np.nonzero((deg > 0) & (p["is_macro"] == 0))[0]
    sample = rng.choice(cand, 64, replace=False)
    ok, total = 0, 0
    with torch.no_grad():
        base = [t.detach().clone() for t in xyz]
        for i in sample:
            for a in (0, 1):
                fd = []
                for hstep in (0.5, 0.25):
                    v = [b.clone() for b in base]
                    v[a][i] += hstep
                    fp = float(m(*v))
                    v[a][i] -= 2 * hstep
                    fm = float(m(*v))
                    fd.append((fp - fm) / (2 * hstep))
                g = float(grads[a][i])
                total += 1
                # a kink of the bistratal max inside the stencil makes the two steps disagree
                if abs(fd[0] - fd[1]) > 1e-3 * max(1.0, abs(g)):
                    continue
                assert abs(fd[1] - g) <= 2e-3 * max(1.0, abs(g)), (i, a, fd, g)
                ok += 1
    assert ok >= 0.9 * total, (ok, total)


def _overflow(h, p, g):
    q = h.copy_map(0).astype(np.float64) * 2.0 ** -36
    vol_b = g["wb"] * g["hb"] * g["db"]
    cells = (p["w_bot"] * p["h_bot"]).sum() * 0.5 * g["dz"]
    return float(np.maximum(q - 1.0, 0.0).sum() * vol_b / cells)


@pytest.mark.parametrize("fused", [True, False])
def test_nesterov_loop_spreads_a_clustered_start(fused):
    """From the paper's initialisation (normal about the centre) the
    preconditioned Nesterov loop (device helpers, and the torch statement of
    it) cuts the density overflow and keeps every centre inside the region
    with z in [d_z/4, 3 d_z/4]."""
    from paper_2403_09070_gb300.nesterov import NesterovPlacer, preconditioner
    p = synth.make_problem("cells_2k", positions="center")
    pl = NesterovPlacer(p, precision="fp32", lam_mult=1.05)
    pl.obj.set_params(lam=1e-4)
    g = pl.g
    ov0 = None
    x, y, z = p["x"], p["y"], p["z"]
    pl.obj.handle.set_positions(*(np.asarray(a, np.float32) for a in (x, y, z)))
    pl.obj.handle.eval()
    ov0 = _overflow(pl.obj.handle, p, g)
    u, hist = (pl.run if fused else pl.run_reference)(x, y, z, iters=200, log_every=50)
    uu = u.cpu().numpy().astype(np.float64)
    pl.obj.handle.set_positions(*(np.asarray(a, np.float32) for a in uu))
    pl.obj.handle.eval()
    ov1 = _overflow(pl.obj.handle, p, g)
    assert ov1 < 0.5 * ov0, (ov0, ov1, hist)
    assert np.all(uu[2] >= 0.25 * g["dz"] - 1e-4) and np.all(uu[2] <= 0.75 * g["dz"] + 1e-4)
    assert np.all(uu[0] >= p["xl"] - 1e-4) and np.all(uu[0] <= p["xh"] + 1e-4)
    assert all(np.isfinite(hh[1]) for hh in hist)
    # eq. improved-precond on a hand-made case
    pins = torch.tensor([0.0, 5.0, 0.0], device="cuda")
    mac = torch.tensor([False, True, True], device="cuda")
    q = torch.tensor([10.0, 10.0, 10.0], device="cuda")
    H = preconditioner(pins, mac, q, 0.01).cpu().numpy()
    np.testing.assert_allclose(H, [1.0, 5.1, 1.0])


def test_fused_nesterov_follows_the_torch_loop():
    """The device-helper loop and the torch loop take the same steps: FP64,
    from the same clustered start, positions after 1, 5 and 12 iterations
    agree to 1e-9 of the region size (they differ only in the order of the
    floating-point atomics and reductions)."""
    from paper_2403_09070_gb300.nesterov import NesterovPlacer
    p = synth.make_problem("cells_2k", positions="center")
    span = max(p["xh"] - p["xl"], p["yh"] - p["yl"])
    for iters in (1, 5, 12):
        out = []
        for fused in (True, False):
            pl = NesterovPlacer(p, precision="fp64", lam_mult=1.1)
            pl.obj.set_params(lam=1e-4)
            u, _ = (pl.run if fused else pl.run_reference)(p["x"], p["y"], p["z"], iters=iters, log_every=0)
            out.append(u.cpu().numpy())
            pl.obj.handle.close()
        assert np.abs(out[0] - out[1]).max() < 1e-9 * span, iters


def test_nesterov_helpers_reject_misuse():
    """The device Nesterov helpers need a 3D handle, the handle's precision
    on CUDA tensors, and a last evaluation whose gradient the handle kept
    (not eval_graph, not device gradient arrays of the other precision)."""
    from paper_2403_09070_gb300 import place3d as P
    p = synth.make_problem("cells_2k")
    n = p["n_inst"]
    xyz = [torch.tensor(p[k], device="cuda", dtype=torch.float32) for k in ("x", "y", "z")]
    g = torch.zeros((3, n), device="cuda", dtype=torch.float32)
    with P.Place3D(p, precision="fp32") as h:
        h.set_positions(*xyz)
        with pytest.raises(P.Place3DError):  # no evaluation yet
            h.nesterov_init(g, 1.0)
        # device gradient arrays of the other precision: written directly, not kept
        h.eval(*[torch.empty(n, device="cuda", dtype=torch.float64) for _ in range(3)])
        with pytest.raises(P.Place3DError):
            h.nesterov_precondition(g)
        h.eval(*[torch.empty(n, device="cuda") for _ in range(3)])  # kept in the handle, then copied
        h.nesterov_precondition(g)
        h.eval(sync=False)  # gradient kept in the handle
        with pytest.raises(ValueError):
            h.nesterov_init(g.double(), 1.0)  # wrong precision
        with pytest.raises(P.Place3DError):
            h.nesterov_init(g, 0.0)  # init_step must be > 0
        h.nesterov_init(g, 1.0)
        assert h.nesterov_step() > 0
        gs = [torch.empty(n, device="cuda") for _ in range(3)]
        h.eval_graph(*xyz, *gs)
        with pytest.raises(P.Place3DError):
            h.nesterov_precondition(g)
    q = synth.to_problem2d(p, seed=3)
    with P.Place3D(q, precision="fp32") as h2:
        h2.set_positions(*(torch.tensor(q[k], device="cuda", dtype=torch.float32) for k in ("x", "y", "z")))
        h2.eval(sync=False)
        with pytest.raises(P.Place3DError):
            h2.nesterov_init(torch.zeros((3, q["n_inst"]), device="cuda"), 1.0)
