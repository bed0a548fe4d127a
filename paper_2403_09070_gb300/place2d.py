"""Host set-up of the multi-die 2D global placement (Sec. V-B, eq. 2d-place).

After the 3D placement fixes the partition, every crossing-die net gets one
HBT at the centre of its optimal region (eq. optimal-region: per axis, the
interval between max{lo+, lo-} and min{hi+, hi-} of the top and bottom pins'
bounding boxes, in either order), and each die receives dummy fillers whose
total area is the die area minus the area of the instances on it (Sec. V-B
fillers).  The result is a PLACE3D_MODE_2D problem for the library.

Filler footprint on a die (the same reading as the 3D fillers): the mean
standard-cell width x height on that die; count = area / footprint, rounded.
The HBT layer gets no fillers (its instances are the HBTs alone).
"""
from __future__ import annotations

import numpy as np

from . import synth


def _pins(prob, x, y, top):
    pi = np.asarray(prob["pin_inst"], np.int64)
    t = top[pi]
    px = x[pi] + np.where(t, prob["off_tx"], prob["off_bx"])
    py = y[pi] + np.where(t, prob["off_ty"], prob["off_by"])
    return px, py, t


def hbt_positions(prob: dict, x=None, y=None, z=None):
    """Centres of eq. optimal-region for the crossing nets of a 3D problem at
    (x, y, z), in net order (the order synth.to_problem2d appends HBTs in).
    Returns (hx, hy, net ids)."""
    x = np.asarray(prob["x"] if x is None else x, np.float64)
    y = np.asarray(prob["y"] if y is None else y, np.float64)
    z = np.asarray(prob["z"] if z is None else z, np.float64)
    zlo, zhi = synth.depth_range(prob)
    top = z > 0.5 * (zlo + zhi)
    ns = np.asarray(prob["net_start"], np.int64)
    deg = np.diff(ns)
    net_of = np.repeat(np.arange(deg.size), deg)
    px, py, t = _pins(prob, x, y, top)
    nt = np.bincount(net_of, weights=t.astype(np.float64), minlength=deg.size)
    cross = np.nonzero((nt > 0) & (nt < deg))[0]
    out = []
    for v in (px, py):
        big = np.finfo(np.float64).max
        lo = [np.full(deg.size, big), np.full(deg.size, big)]
        hi = [np.full(deg.size, -big), np.full(deg.size, -big)]
        for side, m in ((1, t), (0, ~t)):
            np.minimum.at(lo[side], net_of[m], v[m])
            np.maximum.at(hi[side], net_of[m], v[m])
        a = np.maximum(lo[0], lo[1])[cross]
        b = np.minimum(hi[0], hi[1])[cross]
        out.append(0.5 * (np.minimum(a, b) + np.maximum(a, b)))
    return out[0], out[1], cross


def die_filler_plan(prob2d: dict) -> dict:
    """Filler counts and footprints of the two dies of a 2D problem: total
    filler area = die area - area of the die's instances (footprints of
    that die); HBTs are not on a die."""
    z = np.asarray(prob2d["z"], np.float64)
    wb = (prob2d["xh"] - prob2d["xl"]) / prob2d["nx"]
    hb = (prob2d["yh"] - prob2d["yl"]) / prob2d["ny"]
    dz = prob2d["nz"] * 0.5 * (wb + hb)
    hbt = np.asarray(prob2d.get("is_hbt", np.zeros(z.size)), bool)
    top = (z > 0.5 * dz) & ~hbt
    bot = ~top & ~hbt
    mac = np.asarray(prob2d["is_macro"], bool)
    zf = np.asarray(prob2d.get("z_fixed", np.zeros(z.size)), bool)
    std = ~mac & ~zf & ~hbt
    area = (prob2d["xh"] - prob2d["xl"]) * (prob2d["yh"] - prob2d["yl"])
    fp = {}
    for name, on, w, h in (("top", top, "w_top", "h_top"), ("bot", bot, "w_bot", "h_bot")):
        W = np.asarray(prob2d[w], np.float64)
        H = np.asarray(prob2d[h], np.float64)
        free = max(area - float(np.sum((W * H)[on])), 0.0)
        fw = float(W[std].mean()) if std.any() else 0.0
        fh = float(H[std].mean()) if std.any() else 0.0
        fp[f"w_{name}"], fp[f"h_{name}"] = fw, fh
        fp[f"n_{name}"] = int(np.floor(free / (fw * fh) + 0.5)) if fw * fh > 0 else 0
        fp[f"area_{name}"] = free
    fp["n_free"] = 0
    return fp


def from_3d(prob: dict, x=None, y=None, z=None, lam_layer=None, fillers: bool = True, seed: int = 0,
            positions: str = "uniform") -> dict:
    """The PLACE3D_MODE_2D problem of a 3D placement: partition from z, one
    HBT per crossing net at its optimal-region centre, and (optionally) the
    dies' fillers spread over the region ("uniform") or about its centre."""
    hx, hy, _ = hbt_positions(prob, x, y, z)
    q = synth.to_problem2d(prob, x, y, z, hbt_xy=(hx, hy), lam_layer=lam_layer)
    if fillers:
        q = synth.append_fillers(q, die_filler_plan(q), seed=seed, positions=positions)
    return q
