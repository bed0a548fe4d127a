"""Host arrays through the C ABI: page-locked host positions and gradients
are read and written by the kernels directly over the CPU-GPU link (no
staging copies), pageable ones go through device copies.  Every combination
must give the device path's results (the same kernels compute; only where
the data lives differs, so the results differ only by the order of the
floating-point gradient atomics), also when the same pinned buffers are
reused across evaluations with new contents."""
import numpy as np
import pytest

from paper_2403_09070_gb300 import place3d as P
from paper_2403_09070_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _arrays(kind, vals, dt):
    if kind == "pageable":
        return [np.array(v, dtype=np.float64 if dt == torch.float64 else np.float32) for v in vals]
    t = [torch.tensor(np.asarray(v), dtype=dt) for v in vals]
    if kind == "pinned":
        return [a.pin_memory() for a in t]
    return [a.cuda() for a in t]


def _np(a):
    return a.cpu().numpy() if torch.is_tensor(a) else np.asarray(a)


@pytest.mark.parametrize("flags", [0, P.FLAG_TILES])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_host_memory_kinds_agree(precision, flags):
    """flags = PLACE3D_FLAG_TILES: the tiled scatter; device gradients then
    come from the tiled gather, page-locked host ones from the per-cell
    gather (whose host stores overlap its work): the same results."""
    p = synth.make_problem("cells_2k")
    n = p["n_inst"]
    dt = torch.float64 if precision == "fp64" else torch.float32
    tol = 1e-12 if precision == "fp64" else 1e-5
    rng = np.random.default_rng(3)
    pos_sets = [[p["x"], p["y"], p["z"]], list(synth.draw_positions(rng, p, "uniform"))]
    with P.Place3D(p, precision=precision, flags=flags) as h:
        ref = []
        for pos in pos_sets:
            xyz = _arrays("device", pos, dt)
            g = _arrays("device", [np.zeros(n)] * 3, dt)
            h.set_positions(*xyz)
            r = h.eval(*g)
            ref.append((r["obj"], [_np(a) for a in g]))
        for kin in ("pageable", "pinned"):
            for kout in ("pageable", "pinned"):
                g = _arrays(kout, [np.zeros(n)] * 3, dt)
                xyz = _arrays(kin, pos_sets[0], dt)
                for (obj, gref), pos in zip(ref, pos_sets):
                    new = _arrays(kin, pos, dt)
                    for a, b in zip(xyz, new):  # same buffers, new contents
                        a[...] = b
                    h.set_positions(*xyz)
                    r = h.eval(*g)
                    assert r["obj"] == pytest.approx(obj, rel=tol), (kin, kout)
                    for a, b in zip(g, gref):
                        np.testing.assert_allclose(_np(a), b, rtol=tol, atol=tol * np.abs(b).max(),
                                                   err_msg=f"{kin} -> {kout}")
