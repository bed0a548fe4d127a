"""Dummy fillers of the 3D placer (Sec. III-A).

Two filler kinds join the instance table as pinless instances:

* z-fixed fillers, one set per die, of total volume (1/2) d_x d_y d_z (1 - u)
  for the die's maximum utilisation u (eq. filler-vol).  They start at depth
  3 d_z / 4 (top) or d_z / 4 (bottom) and their z-gradient is held at zero
  (the ``z_fixed`` mask of the C ABI), so a die filled past u pushes
  instances to the other die;
* free fillers for the remaining white space, d_x d_y d_z minus the z-fixed
  fillers and the instances' volume vol_a, clamped at zero
  (eq. free-filler-vol).  They move in z like standard cells.

vol_a is taken at the initial positions: each instance is a cuboid of depth
d_z / 2 with the footprint of the die it starts on (eq. std-size-tech; the
linear macro size of eq. macro-size-tech).  Fillers on one die share one
footprint: the mean standard-cell width and height on that die (standard
cells = instances that are neither macros nor z-fixed).  A set's count is its
volume over one filler's volume rounded to the nearest integer; a free filler
counts the mean of the two dies' filler volumes.  Every instance, fillers
included, starts normal about the region's centre (Sec. III-A
initialisation): sigma = 0.1 of each extent in x and y, and for free fillers
0.2 of the movable depth range [d_z / 4, 3 d_z / 4] in z.
"""
from __future__ import annotations

import numpy as np

from . import synth


def _geometry(prob: dict):
    dx = prob["xh"] - prob["xl"]
    dy = prob["yh"] - prob["yl"]
    db = 0.5 * (dx / prob["nx"] + dy / prob["ny"])
    return dx, dy, prob["nz"] * db


def _footprint(prob: dict, z: np.ndarray, dz: float):
    """Per-instance width and height on the die given by z (eqs.
    std-size-tech, macro-size-tech)."""
    top = (z - 0.5 * dz) > 0.0
    t = np.clip(2.0 * z / dz - 0.5, 0.0, 1.0)
    mac = np.asarray(prob["is_macro"]).astype(bool)
    wb, hb = np.asarray(prob["w_bot"], np.float64), np.asarray(prob["h_bot"], np.float64)
    wt, ht = np.asarray(prob["w_top"], np.float64), np.asarray(prob["h_top"], np.float64)
    w = np.where(mac, t * wt + (1.0 - t) * wb, np.where(top, wt, wb))
    h = np.where(mac, t * ht + (1.0 - t) * hb, np.where(top, ht, hb))
    return w, h


def plan(prob: dict, u_top: float, u_bot: float, z=None) -> dict:
    """Volumes, per-die footprints and counts of the fillers (eqs. filler-vol,
    free-filler-vol) for the instances at depths z (default prob["z"])."""
    z = np.asarray(prob["z"] if z is None else z, np.float64)
    dx, dy, dz = _geometry(prob)
    depth = 0.5 * dz
    V = dx * dy * dz
    w, h = _footprint(prob, z, dz)
    vol_a = float(np.sum(w * h * depth))
    std = ~np.asarray(prob["is_macro"]).astype(bool)
    zf = prob.get("z_fixed")
    if zf is not None:
        std &= ~np.asarray(zf).astype(bool)
    n_std = int(std.sum())
    mean = lambda k: float(np.mean(np.asarray(prob[k], np.float64)[std])) if n_std else 0.0
    wt, ht, wb, hb = mean("w_top"), mean("h_top"), mean("w_bot"), mean("h_bot")
    vf_t = 0.5 * V * (1.0 - u_top)
    vf_b = 0.5 * V * (1.0 - u_bot)
    vfr = max(V - (vf_t + vf_b + vol_a), 0.0)
    unit_t, unit_b = wt * ht * depth, wb * hb * depth
    unit_fr = 0.5 * (unit_t + unit_b)
    count = lambda v, u: int(np.floor(v / u + 0.5)) if u > 0.0 else 0
    return dict(vol_a=vol_a, vol_f_top=vf_t, vol_f_bot=vf_b, vol_fr=vfr,
                w_top=wt, h_top=ht, w_bot=wb, h_bot=hb,
                n_top=count(vf_t, unit_t), n_bot=count(vf_b, unit_b), n_free=count(vfr, unit_fr))


def insert(prob: dict, u_top: float, u_bot: float, seed: int = 0, positions: str = "center") -> dict:
    """A copy of prob with the fillers of ``plan`` appended after its
    instances (pinless: the netlist is unchanged), in the order top z-fixed,
    bottom z-fixed, free, at their initial positions.  The returned dict
    carries the plan under "fillers".  positions="uniform" spreads the
    fillers over the region instead (a mid-placement state)."""
    return synth.append_fillers(prob, plan(prob, u_top, u_bot), seed, positions)
