"""Failure detection on the GPU without faulting it: device allocation
failures injected through a fake of the failing call (place3d_create
returns OOM, frees what it allocated, and the next create works), and
position checks (non-finite or out-of-range coordinates under
PLACE3D_FLAG_CHECKS return OUT_OF_RANGE)."""
import numpy as np
import pytest

from paper_2403_09070_gb300 import place3d as P
from paper_2403_09070_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("nth", [1, 2, 7, 19, 30])
def test_injected_allocation_failure(nth):
    p = synth.make_problem("cells_2k")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    P.debug_fail_alloc(nth)
    try:
        with pytest.raises(P.Place3DError) as ei:
            P.Place3D(p, precision="fp32")
        assert ei.value.code == -5  # OOM
    finally:
        P.debug_fail_alloc(0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 8 << 20  # nothing left allocated (allocator granularity aside)
    with P.Place3D(p, precision="fp32") as h:  # the next create and evaluation work
        h.set_positions(*(np.asarray(p[k], np.float32) for k in ("x", "y", "z")))
        r = h.eval()
        assert np.isfinite(r["obj"]) and r["obj"] > 0


@pytest.mark.parametrize("bad", ["nan_x", "inf_y", "z_low", "z_high"])
def test_checked_positions(bad):
    p = synth.make_problem("cells_2k")
    x, y, z = (np.asarray(p[k], np.float64).copy() for k in ("x", "y", "z"))
    zlo, zhi = synth.depth_range(p)
    if bad == "nan_x":
        x[17] = np.nan
    elif bad == "inf_y":
        y[3] = np.inf
    elif bad == "z_low":
        z[5] = 0.5 * zlo
    else:
        z[5] = zhi + 0.5 * zlo
    with P.Place3D(p, precision="fp64", flags=P.FLAG_CHECKS) as h:
        with pytest.raises(P.Place3DError) as ei:
            h.set_positions(x, y, z)
        assert ei.value.code == -3  # OUT_OF_RANGE
        h.set_positions(*(np.asarray(p[k], np.float64) for k in ("x", "y", "z")))  # still usable
        assert np.isfinite(h.eval()["obj"])
