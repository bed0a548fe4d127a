"""GPU tests of the tensor-core path: the split-BF16 tcgen05 product against
an FP64 product, and the PLACE3D_FP32_TC evaluation against the oracle
(objective within 2e-5 relative, gradient L2 within 1e-4 relative)."""
import numpy as np
import pytest

from gpu_harness import rel_l2, rel_max, run_gpu, run_oracle
from helpers import dz_of, problem
from paper_2403_09070_gb300 import place3d as P
from paper_2403_09070_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K,batches", [(128, 64, 64, 1), (256, 128, 512, 3), (512, 1024, 512, 2)])
def test_tc_product_matches_fp64(M, N, K, batches):
    """Split-BF16 operands with FP32 accumulation reproduce the FP64 product
    to ~1e-5 of its scale (the hi*hi + hi*lo + lo*hi terms)."""
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(batches, M, K)).astype(np.float32)
    W = np.cos(np.pi * np.outer(np.arange(N) % K, np.arange(K) + 0.5) / K).astype(np.float32)
    out, err = P.tc_selftest(A, W)
    assert err == 0
    ref = np.einsum("bmk,nk->bnm", A.astype(np.float64), W.astype(np.float64))
    e = np.abs(out - ref).max() / np.abs(ref).max()
    assert e < 2e-5, e


def _check_tc(prob, x, y, z):
    x32, y32, z32 = (np.asarray(a, np.float32).astype(np.float64) for a in (x, y, z))
    g = run_gpu(prob, x32, y32, z32, "fp32_tc")
    o, r = run_oracle(prob, x32, y32, z32, g["alpha"], density_mode=0)
    assert np.array_equal(g["q"], o.density_fixed(x32, y32, z32, use_float=True))
    assert g["res"]["obj"] == pytest.approx(r["obj"], rel=2e-5)
    assert g["res"]["energy"] == pytest.approx(r["energy"], rel=1e-4)
    for k in ("gx", "gy", "gz"):
        assert rel_l2(g[k], r[k]) < 1e-4, (k, rel_l2(g[k], r[k]))
    pe = o.poisson(o.density_direct(x32, y32, z32))
    for k in ("ex", "ey", "ez"):
        assert rel_l2(g[k], pe[k]) < 1e-4, (k, rel_l2(g[k], pe[k]))


@pytest.mark.parametrize("positions", ["uniform", "center"])
def test_fp32_tc_cells_200k(positions):
    p = synth.make_problem("cells_200k", positions=positions)
    _check_tc(p, p["x"], p["y"], p["z"])


def test_fp32_tc_rectangular_grid_nz3():
    """N_x != N_y, N_z = 3, region origin off zero, macros near the edge."""
    rng = np.random.default_rng(31)
    n = 3000
    sizes = [(float(rng.integers(1, 9)), 1.0, 0.0, 0.0) for _ in range(n)]
    sizes = [(w, h, 0.8 * w, 0.8 * h) for (w, h, _, _) in sizes] + [(40.0, 30.0, 32.0, 24.0)] * 3
    nets = [list(rng.choice(n + 3, size=int(rng.integers(2, 12)), replace=False)) for _ in range(3500)]
    P_ = sum(len(e) for e in nets)
    off = np.zeros((P_, 4))
    off[:, 0] = rng.uniform(-0.5, 0.5, P_)
    off[:, 2] = 0.8 * off[:, 0]
    die = (-50.0, 20.0, -50.0 + 400.0, 20.0 + 300.0)
    p = problem(sizes, nets=nets, offsets=off, die=die, grid=(128, 256, 3), macros=[n, n + 1, n + 2],
                gamma=4 * 400.0 / 128)
    dz = dz_of(p)
    x = rng.uniform(die[0] + 2, die[2] - 2, n + 3)
    y = rng.uniform(die[1] + 2, die[3] - 2, n + 3)
    z = rng.uniform(dz / 4, 3 * dz / 4, n + 3)
    x[n] = die[0] + 5.0
    _check_tc(p, x, y, z)


def test_fp32_tc_rejects_unaligned_grid():
    p = synth.make_problem("cells_2k")  # 64 x 64 bins
    with pytest.raises(P.Place3DError) as ei:
        P.Place3D(p, precision="fp32_tc")
    assert ei.value.code == -7


def _precision_study(name, p, x, y, z, alpha, ref):
    """Errors of the FP64 and FP32 paths (and of the FP32_TC result passed in
    by the caller) against the FP64 oracle's evaluation `ref` at the same
    positions: relative errors of the scalars, relative L2 and max-norm
    errors of the gradient.  Printed as one JSON line (pytest -s)."""
    import json
    out = {}
    for m in ("fp64", "fp32"):
        g = run_gpu(p, x, y, z, m, alpha=alpha, maps=False)
        e = {k: abs(g["res"][k] - ref[k]) / max(abs(ref[k]), 1e-300)
             for k in ("obj", "wl_bi", "wl_z", "energy", "hpwl_d2d")}
        e["n_cross_equal"] = g["res"]["n_cross"] == ref["n_cross"]
        for k in ("gx", "gy", "gz"):
            e[k + "_rel_l2"] = rel_l2(g[k], ref[k])
            e[k + "_rel_max"] = rel_max(g[k], ref[k])
        out[m] = e
    print("PRECISION", json.dumps({"workload": name, "reference": "FP64 oracle, direct density definition",
                                   "modes": out}))
    return out


def _tc_errors(g, ref):
    e = {k: abs(g["res"][k] - ref[k]) / max(abs(ref[k]), 1e-300) for k in ("obj", "wl_bi", "wl_z", "energy", "hpwl_d2d")}
    for k in ("gx", "gy", "gz"):
        e[k + "_rel_l2"] = rel_l2(g[k], ref[k])
        e[k + "_rel_max"] = rel_max(g[k], ref[k])
    return e


def test_fp32_tc_full_size_bench_configuration():
    """The bench's workload and launch configuration (1M cells, 512x512x4,
    FP32_TC, autotuned reduction forms) against the full FP64 oracle; with the
    FP64 and FP32 paths at the same positions for the precision study."""
    import json
    p = synth.make_problem("cells_1m")
    x32, y32, z32 = (np.asarray(p[k], np.float32).astype(np.float64) for k in ("x", "y", "z"))
    g = run_gpu(p, x32, y32, z32, "fp32_tc", autotune=True)
    o, r = run_oracle(p, x32, y32, z32, g["alpha"], density_mode=0)
    print("PRECISION", json.dumps({"workload": "cells_1m", "modes": {"fp32_tc": _tc_errors(g, r)}}))
    study = _precision_study("cells_1m", p, x32, y32, z32, g["alpha"], r)
    assert study["fp64"]["obj"] < 1e-8 and study["fp64"]["gx_rel_l2"] < 1e-8
    assert study["fp32"]["obj"] < 2e-5 and study["fp32"]["gx_rel_l2"] < 1e-4
    assert np.array_equal(g["q"], o.density_fixed(x32, y32, z32, use_float=True))
    assert g["res"]["obj"] == pytest.approx(r["obj"], rel=2e-5)
    assert g["res"]["n_cross"] == r["n_cross"]
    assert g["res"]["hpwl_d2d"] == pytest.approx(r["hpwl_d2d"], rel=1e-6)
    for k in ("gx", "gy", "gz"):
        assert rel_l2(g[k], r[k]) < 1e-4, (k, rel_l2(g[k], r[k]))


def test_fp32_tc_cells_200k_with_fillers():
    """cells_200k with the fillers of eqs. filler-vol / free-filler-vol at
    u+ = u- = 0.8 (about 4.3M pinless instances, spread over the region)."""
    from oracle import Oracle
    p = synth.make_problem("cells_200k")
    fp = Oracle(p).filler_plan(p["z"], 0.8, 0.8)
    q = synth.append_fillers(p, fp, seed=7, positions="uniform")
    assert q["n_inst"] > 4_000_000
    _check_tc(q, q["x"], q["y"], q["z"])


def test_fp32_tc_large_skewed_configuration():
    """4M cells + 200 macros, 4.2M nets plus 200 high-fanout nets of 2k-20k
    pins (one block per net), 1024x1024x4 bins, FP32_TC with autotuned forms,
    against the full FP64 oracle (about a minute of CPU time)."""
    p = synth.make_problem("cells_4m_skewed")
    assert np.diff(p["net_start"]).max() >= 2000
    x32, y32, z32 = (np.asarray(p[k], np.float32).astype(np.float64) for k in ("x", "y", "z"))
    g = run_gpu(p, x32, y32, z32, "fp32_tc", autotune=True)
    assert any(f[1] == 0 for f in g["forms"])  # the block form ran
    o, r = run_oracle(p, x32, y32, z32, g["alpha"], density_mode=0)
    import json
    print("PRECISION", json.dumps({"workload": "cells_4m_skewed", "modes": {"fp32_tc": _tc_errors(g, r)}}))
    study = _precision_study("cells_4m_skewed", p, x32, y32, z32, g["alpha"], r)
    assert study["fp64"]["obj"] < 1e-8 and study["fp64"]["gx_rel_l2"] < 1e-8
    assert study["fp32"]["obj"] < 2e-5 and study["fp32"]["gx_rel_l2"] < 1e-4
    assert np.array_equal(g["q"], o.density_fixed(x32, y32, z32, use_float=True))
    assert g["res"]["obj"] == pytest.approx(r["obj"], rel=2e-5)
    assert g["res"]["n_cross"] == r["n_cross"]
    assert g["res"]["hpwl_d2d"] == pytest.approx(r["hpwl_d2d"], rel=1e-6)
    for k in ("gx", "gy", "gz"):
        assert rel_l2(g[k], r[k]) < 1e-4, (k, rel_l2(g[k], r[k]))


def test_tc_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: the producer arms nothing, the
    bounded mbarrier wait runs out (about 0.1 s), the kernel returns an error
    status the host reads, and the context still computes correctly."""
    rc, code = P.tc_timeout_selftest(200_000_000)
    assert rc == -6 and code in (1, 2, 3), (rc, code)
    rng = np.random.default_rng(1)
    A = rng.normal(size=(1, 128, 64)).astype(np.float32)
    W = np.cos(np.pi * np.outer(np.arange(64), np.arange(64) + 0.5) / 64).astype(np.float32)
    out, err = P.tc_selftest(A, W)
    assert err == 0
    ref = np.einsum("bmk,nk->bnm", A.astype(np.float64), W.astype(np.float64))
    assert np.abs(out - ref).max() / np.abs(ref).max() < 2e-5
