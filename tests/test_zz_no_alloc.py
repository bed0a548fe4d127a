"""The allocation-free density map (place3d_density_map_noalloc) against the
existing entry point's fixed-point map, bit for bit, on two calls in a row.

It exists for callers that cannot allocate device memory when they need the
map (inside another framework's memory arena, or where an allocation would
synchronise the device); its scratch is a fixed array inside the library.
Collected last so that a failure here stops a -x run after every other test.
"""
import numpy as np
import pytest

from paper_2403_09070_gb300 import place3d as P
from paper_2403_09070_gb300 import synth

pytestmark = pytest.mark.gpu


def _existing_map(prob, x, y, z):
    with P.Place3D(prob, precision="fp64") as h:
        h.set_positions(x, y, z)
        h.eval()
        return h.copy_map(P.MAP_RHO_FIXED) * 2.0 ** -36


def test_noalloc_density_matches_eval_on_two_calls():
    torch = pytest.importorskip("torch")
    prob = synth.make_problem("cells_2k")
    dev = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    sizes = [dev(prob[k]) for k in ("w_bot", "h_bot", "w_top", "h_top")]
    is_macro = dev(prob["is_macro"], torch.uint8)
    region = (prob["xl"], prob["yl"], prob["xh"], prob["yh"])
    grid = (prob["nx"], prob["ny"], prob["nz"])
    rng = np.random.default_rng(12)
    for call, kind in enumerate(("uniform", "center")):
        x, y, z = synth.draw_positions(rng, prob, kind)
        exp = _existing_map(prob, x, y, z)
        rho = torch.full((prob["nz"], prob["ny"], prob["nx"]), float("nan"), dtype=torch.float64, device="cuda")
        P.density_map_noalloc(dev(x), dev(y), dev(z), *sizes, is_macro, region, grid, rho)
        torch.cuda.synchronize()
        got = rho.cpu().numpy()
        assert np.array_equal(got, exp), f"call {call}: max diff {np.abs(got - exp).max()}"


def test_noalloc_at_the_size_limit_with_macros_on_a_side_stream():
    """A grid of exactly PLACE3D_NOALLOC_MAX_BINS bins (256 x 256 x 4, where
    the macro corner map ends at the end of the static array), 20 macros,
    enqueued on a non-default stream: bit for bit the handle's map, twice."""
    torch = pytest.importorskip("torch")
    prob = synth.make_problem("cells_200k")
    assert prob["nx"] * prob["ny"] * prob["nz"] == P.NOALLOC_MAX_BINS
    assert int(np.asarray(prob["is_macro"]).sum()) == 20
    dev = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    sizes = [dev(prob[k]) for k in ("w_bot", "h_bot", "w_top", "h_top")]
    is_macro = dev(prob["is_macro"], torch.uint8)
    region = (prob["xl"], prob["yl"], prob["xh"], prob["yh"])
    grid = (prob["nx"], prob["ny"], prob["nz"])
    rng = np.random.default_rng(21)
    side = torch.cuda.Stream()
    for call, kind in enumerate(("uniform", "center")):
        x, y, z = synth.draw_positions(rng, prob, kind)
        exp = _existing_map(prob, x, y, z)
        xyz = [dev(a) for a in (x, y, z)]
        rho = torch.full((prob["nz"], prob["ny"], prob["nx"]), float("nan"), dtype=torch.float64, device="cuda")
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            P.density_map_noalloc(*xyz, *sizes, is_macro, region, grid, rho, stream=side)
        side.synchronize()
        got = rho.cpu().numpy()
        assert np.array_equal(got, exp), f"call {call}: max diff {np.abs(got - exp).max()}"


def test_noalloc_rejects_grids_above_the_limit():
    torch = pytest.importorskip("torch")
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    m = torch.zeros(1, dtype=torch.uint8, device="cuda")
    rho = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.Place3DError) as ei:
        P.density_map_noalloc(t, t, t, t, t, t, t, m, (0, 0, 1, 1), (1024, 1024, 1), rho)
    assert ei.value.code == -3
