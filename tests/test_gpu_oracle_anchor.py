"""GPU results that sit on top of the evaluation, checked against the FP64
oracle rather than against the library itself: the autograd wrapper's
gradient, the alpha dp^(z)/dz part of the depth gradient (central
differences, Sec. II-B eq. wl-model), the device Nesterov loop (a host loop
whose gradients come from the oracle), every instance of the 24-instance
batch (one graph launch), and the FP64 path at 1M cells against the
fixed-point replica at the FP64 bar."""
import math

import numpy as np
import pytest

from gpu_harness import Q, rel_l2, rel_max
from oracle import Oracle
from paper_2403_09070_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autograd_gradient_matches_oracle_cells_200k_fp32_tc():
    """torch.autograd over the fused evaluation (FP32 with tensor-core
    transforms) against the FP64 oracle at the same float32 positions:
    objective within 2e-5, each gradient component within 1e-4 (L2)."""
    from paper_2403_09070_gb300.autograd import Place3DObjective
    p = synth.make_problem("cells_200k")
    m = Place3DObjective(p, precision="fp32_tc")
    xyz = [torch.tensor(p[k], device="cuda", dtype=torch.float32, requires_grad=True) for k in ("x", "y", "z")]
    f = m(*xyz)
    (2.0 * f).backward()
    x64 = [t.detach().double().cpu().numpy() for t in xyz]
    r = Oracle(p, alpha=m.alpha).eval(*x64, density_mode=0)
    assert float(f.detach()) == pytest.approx(r["obj"], rel=2e-5)
    for t, k in zip(xyz, ("gx", "gy", "gz")):
        e = rel_l2(t.grad.double().cpu().numpy(), 2.0 * r[k])
        assert e < 1e-4, (k, e)
    m.handle.close()


def test_depth_wirelength_gradient_central_differences():
    """The alpha dp^(z)/dz part of the z-gradient is a true derivative of the
    objective: with lambda = 0 the objective depends on z_i only through
    alpha p^_e(z) while z_i stays on its die, so central differences of the
    FP64 objective in z_i equal alpha * dp^(z)/dz_i of the GPU (and of the
    oracle); and the GPU's final z-gradient is g * FD + alpha * dp^(z)/dz
    (eq. fda-normalize)."""
    from paper_2403_09070_gb300 import place3d as P
    p = synth.make_problem("cells_200k")
    x, y, z = (np.asarray(p[k], np.float64) for k in ("x", "y", "z"))
    with P.Place3D(p, precision="fp64") as h:
        alpha = h.alpha
        h.set_params(gamma=p["gamma"], gamma_z=0.0, alpha=alpha, lam=0.0)
        dz = h.geometry()["dz"]
        h.set_positions(x, y, z)
        g = [np.zeros(p["n_inst"]) for _ in range(3)]
        r = h.eval(*g)
        wl = h.wl_parts()
        # eq. fda-normalize: z-gradient = g * FD + alpha dp(z)/dz (lambda = 0)
        zf = np.asarray(p["z_fixed"], bool)
        dec = np.where(zf, 0.0, r["g_scale"] * wl["gfd"] + alpha * wl["gwaz"])
        assert rel_max(g[2], dec) < 1e-12
        o = Oracle(p, alpha=alpha)
        ow = o.wirelength(x, y, z)
        assert rel_max(wl["gwaz"], ow["gwaz"]) < 1e-9
        rng = np.random.default_rng(17)
        deg = np.bincount(np.asarray(p["pin_inst"]), minlength=p["n_inst"])
        step = 0.25
        cand = np.nonzero((deg > 0) & ~zf & (np.abs(z - 0.5 * dz) > 4 * step))[0]
        sample = rng.choice(cand, 64, replace=False)
        for i in sample:
            fd = []
            for hh in (2 * step, step):
                zp = z.copy()
                zp[i] += hh
                h.set_positions(x, y, zp)
                fp = h.eval()["obj"]
                zp[i] -= 2 * hh
                h.set_positions(x, y, zp)
                fm = h.eval()["obj"]
                fd.append((fp - fm) / (2 * hh))
            ref = alpha * ow["gwaz"][i]
            tol = 1e-4 * max(1.0, abs(ref))
            assert abs(fd[1] - ref) <= tol, (i, fd, ref)
            assert abs(fd[1] - alpha * wl["gwaz"][i]) <= tol
            assert abs(fd[0] - ref) <= 4 * tol  # the wider stencil agrees too (second order)


def _oracle_nesterov(p, alpha, lam0, lam_mult, init_step, iters, dz):
    """The preconditioned Nesterov loop (Sec. III-A, eq. improved-precond,
    projection to the region and z in [d_z/4, 3 d_z/4]) in numpy, with each
    gradient from the FP64 oracle (fixed-point density replica)."""
    o = Oracle(p, alpha=alpha)
    n = p["n_inst"]
    lo = np.array([p["xl"], p["yl"], 0.25 * dz])[:, None]
    hi = np.array([p["xh"], p["yh"], 0.75 * dz])[:, None]
    proj = lambda v: np.clip(v, lo, hi)
    mac = np.asarray(p["is_macro"], bool)
    zf = np.asarray(p["z_fixed"], bool)
    pins = np.bincount(np.asarray(p["pin_inst"]), minlength=n).astype(np.float64)
    wt, ht, wb, hb = (np.asarray(p[k], np.float64) for k in ("w_top", "h_top", "w_bot", "h_bot"))

    def grad(v, lam):
        o.s.lam = lam
        r = o.eval(v[0], v[1], v[2], density_mode=1)
        G = np.stack([r["gx"], r["gy"], r["gz"]])
        top = v[2] > 0.5 * dz
        q = np.where(top, wt * ht, wb * hb) * (0.5 * dz)
        H = np.maximum(lam * q + np.where(mac, pins, 0.0), 1.0)
        g = G / H
        g[2] = np.where(zf, 0.0, g[2])
        return g

    lam = lam0
    u = proj(np.stack([np.asarray(p[k], np.float64) for k in ("x", "y", "z")]))
    v = u.copy()
    g = grad(v, lam)
    step = init_step / max(np.abs(g).max(), 1e-30)
    a = 1.0
    for _ in range(iters):
        a_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * a * a))
        u_new = proj(v - step * g)
        v_new = proj(u_new + ((a - 1.0) / a_new) * (u_new - u))
        dv2 = float(((v_new - v) ** 2).sum())
        g_new = grad(v_new, lam)
        dg2 = float(((g_new - g) ** 2).sum())
        if dv2 > 0 and dg2 > 0:
            step = math.sqrt(dv2 / dg2)
        u, v, g, a = u_new, v_new, g_new, a_new
        lam *= lam_mult
    return u


@pytest.mark.parametrize("positions", ["center", "uniform"])
def test_device_nesterov_loop_follows_oracle_loop(positions):
    """FP64, cells_2k: the device-helper Nesterov loop (place3d_nesterov_*)
    and the host loop driven by oracle gradients give the same positions
    after 1, 3 and 5 iterations, within 1e-9 of the region size."""
    from paper_2403_09070_gb300.nesterov import NesterovPlacer
    p = synth.make_problem("cells_2k", positions=positions)
    span = max(p["xh"] - p["xl"], p["yh"] - p["yl"])
    for iters in (1, 3, 5):
        pl = NesterovPlacer(p, precision="fp64", lam_mult=1.1)
        pl.obj.set_params(lam=1e-4)
        u, _ = pl.run(p["x"], p["y"], p["z"], iters=iters, log_every=0)
        got = u.cpu().numpy()
        ref = _oracle_nesterov(p, pl.obj.alpha, 1e-4, 1.1, pl.init_step, iters, pl.g["dz"])
        pl.obj.handle.close()
        assert np.abs(got - ref).max() < 1e-9 * span, (iters, np.abs(got - ref).max())
        assert np.abs(got - np.stack([p["x"], p["y"], p["z"]])).max() > 1e-3  # it moved


def test_batch24_every_instance_matches_oracle():
    """The 24 uneven instances of the batching workload (5k-300k cells, grids
    64x64x2 to 512x512x4), evaluated by ONE batch graph launch (the
    wirelength stage shared by all instances, one launch per stage): every
    instance's fixed-point map equals the oracle's float replica bit for bit,
    its objective is within 2e-5 and each gradient component within 1e-4
    (L2) of the FP64 oracle."""
    from paper_2403_09070_gb300 import place3d as P
    probs = synth.make_batch(24, seed=4)
    hs, xyz, gs = [], [], []
    for p in probs:
        prec = "fp32_tc" if p["nx"] % 128 == 0 else "fp32"
        hs.append(P.Place3D(p, precision=prec))
        xyz.append([torch.tensor(p[k], device="cuda", dtype=torch.float32) for k in ("x", "y", "z")])
        gs.append([torch.empty(p["n_inst"], device="cuda", dtype=torch.float32) for _ in range(3)])
    b = P.Batch(hs)
    b.eval(*[[v[k] for v in xyz] for k in range(3)], *[[v[k] for v in gs] for k in range(3)])
    torch.cuda.synchronize()
    assert b.shared_stages() == 1  # the wirelength stage shared by the 24 instances
    for p, h, v, g in zip(probs, hs, xyz, gs):
        r = h.get_result()
        qmap = h.copy_map(P.MAP_RHO_FIXED)
        x32 = [t.double().cpu().numpy() for t in v]
        o = Oracle(p, alpha=h.alpha)
        ref = o.eval(*x32, density_mode=0)
        assert np.array_equal(qmap, o.density_fixed(*x32, use_float=True)), p["n_inst"]
        assert r["obj"] == pytest.approx(ref["obj"], rel=2e-5), p["n_inst"]
        assert r["n_cross"] == ref["n_cross"]
        for a, k in zip(g, ("gx", "gy", "gz")):
            e = rel_l2(a.cpu().numpy(), ref[k])
            assert e < 1e-4, (p["n_inst"], k, e)
    b.close()
    for h in hs:
        h.close()


def test_fp64_cells_1m_against_fixed_point_replica():
    """The FP64 path at 1M cells (512x512x4) against the oracle with the
    double fixed-point replica: map bit for bit, fields, wirelength parts,
    scalars and the gradient within 1e-9 relative."""
    from paper_2403_09070_gb300 import place3d as P
    p = synth.make_problem("cells_1m")
    x, y, z = (np.asarray(p[k], np.float64) for k in ("x", "y", "z"))
    with P.Place3D(p, precision="fp64") as h:
        h.set_positions(x, y, z)
        g = [np.zeros(p["n_inst"]) for _ in range(3)]
        res = h.eval(*g)
        qmap = h.copy_map(P.MAP_RHO_FIXED)
        E = [h.copy_map(m) for m in (P.MAP_EX, P.MAP_EY, P.MAP_EZ)]
        wl = h.wl_parts()
        alpha = h.alpha
    o = Oracle(p, alpha=alpha)
    q = o.density_fixed(x, y, z, use_float=False)
    assert np.array_equal(qmap, q)
    pe = o.poisson(q * Q)
    for a, k in zip(E, ("ex", "ey", "ez")):
        assert rel_max(a, pe[k]) < 1e-9, k
    w = o.wirelength(x, y, z)
    for k in ("gx", "gy", "gwaz", "gfd"):
        assert rel_max(wl[k], w[k]) < 1e-9, k
    r = o.eval(x, y, z, density_mode=1)
    for k, kr in (("obj", "obj"), ("wl_bi", "wl_bi"), ("wl_z", "wl_z"), ("energy", "energy"),
                  ("hpwl_d2d", "hpwl_d2d"), ("g_scale", "g_scale")):
        assert res[k] == pytest.approx(r[kr], rel=1e-9), k
    assert res["n_cross"] == r["n_cross"]
    for a, k in zip(g, ("gx", "gy", "gz")):
        assert rel_max(a, r[k]) < 1e-9, k
