"""Whole-objective pins of the oracle (eq. analytical-placement with the
wirelength of eq. wl-model and the eDensity3D penalty): invariances and the
special cases that reduce it to its parts."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2403_09070_gb300 import synth


@pytest.fixture(scope="module")
def prob():
    return synth.make_problem("cells_2k")


def test_origin_shift_invariance(prob):
    """Moving the die outline and every position by the same offset leaves
    the objective and the gradient unchanged."""
    o = Oracle(prob)
    r = o.eval(prob["x"], prob["y"], prob["z"], density_mode=0)
    q = synth.make_problem("cells_2k", origin=(137.0, -42.5))
    o2 = Oracle(q, alpha=o.alpha)
    r2 = o2.eval(q["x"], q["y"], q["z"], density_mode=0)
    assert r2["obj"] == pytest.approx(r["obj"], rel=1e-10)
    for k in ("gx", "gy", "gz"):
        np.testing.assert_allclose(r2[k], r[k], rtol=1e-7, atol=1e-9 * np.abs(r[k]).max())


def test_density_modes_agree(prob):
    """The fixed-point density replica changes the objective by rounding only."""
    o = Oracle(prob)
    r0 = o.eval(prob["x"], prob["y"], prob["z"], density_mode=0)
    r1 = o.eval(prob["x"], prob["y"], prob["z"], density_mode=1)
    r2 = o.eval(prob["x"], prob["y"], prob["z"], density_mode=2)
    assert r1["energy"] == pytest.approx(r0["energy"], rel=1e-9)
    assert r2["energy"] == pytest.approx(r0["energy"], rel=1e-5)
    np.testing.assert_allclose(r1["gx"], r0["gx"], rtol=1e-6, atol=1e-9 * np.abs(r0["gx"]).max())


def test_lambda_zero_is_wirelength_only(prob):
    q = dict(prob, lam=0.0)
    o = Oracle(q)
    r = o.eval(q["x"], q["y"], q["z"])
    w = o.wirelength(q["x"], q["y"], q["z"])
    assert r["obj"] == pytest.approx(w["wl_bi"] + o.alpha * w["wl_z"], rel=1e-14)
    np.testing.assert_allclose(r["gx"], w["gx"], rtol=1e-14)


def test_z_fixed_instances_have_zero_z_gradient(prob):
    q = dict(prob)
    zf = np.zeros(q["n_inst"], np.uint8)
    zf[::7] = 1
    q["z_fixed"] = zf
    r = Oracle(q).eval(q["x"], q["y"], q["z"])
    assert np.all(r["gz"][zf == 1] == 0.0)
    assert np.any(r["gz"][zf == 0] != 0.0)


def test_energy_matches_poisson_of_density(prob):
    o = Oracle(prob)
    r = o.eval(prob["x"], prob["y"], prob["z"], density_mode=0)
    e = o.poisson(o.density_direct(prob["x"], prob["y"], prob["z"]))["energy"]
    assert r["energy"] == pytest.approx(e, rel=1e-14)
