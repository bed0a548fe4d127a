"""Seeded synthetic placement problems shaped like the paper's benchmarks.

This module only *draws* inputs: netlists (pin/net CSR), per-die instance
sizes, pin offsets and positions.  It holds none of the placement method's
arithmetic (no density, no wirelength, no transform), so that both the CUDA
path and the CPU oracle can take their inputs from it without sharing any part
of the computation they are compared on.

The paper's ICCAD 2023 contest cases and RISC-V designs (Tab. "benchmark-stat",
Tab. "risc-stat") are not available; these recipes stand in for them:

* net degree: 2 (55 %), 3-4 (25 %), 5-16 (17 %), 17-64 (3 %), P(d) ~ d^-2
  inside each bucket (about 4.2 pins per net);
* every pin of a net sits on a distinct instance drawn uniformly; macros take
  1 % of the pins ("macros have many pins", Sec. III-A preconditioning text);
* pin offsets uniform inside the bottom-die footprint, top offsets 0.8x;
* std cells: bottom width uniform in 1..8 sites of 1.0, height (row) 1.0; top
  die scaled by 0.8 in both dimensions (heterogeneous technology nodes);
* macros: squares whose total area is 20 % of one die, split equally, 0.8x on
  the top die;
* positions: x, y uniform inside the die, z uniform in [d_z/4, 3 d_z/4]
  ("uniform") or normal about the centre with sigma = 0.1 of each extent
  ("center", the paper's initialisation, Sec. III-A free fillers text);
* gamma = 4 bin widths, lambda = 1e-3, HBT cost beta = 10, HBT pitch 1.0,
  row heights 0.8 (top) / 1.0 (bottom).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Degree buckets (inclusive ranges) and their probabilities.
_DEG_BUCKETS = ((2, 2, 0.55), (3, 4, 0.25), (5, 16, 0.17), (17, 64, 0.03))


@dataclasses.dataclass(frozen=True)
class Workload:
    """Sizes of one synthetic workload."""

    name: str
    n_std: int
    n_macro: int
    n_net: int
    die: float  # square die side, both dies share the outline
    nx: int
    ny: int
    nz: int
    seed: int
    n_hifanout: int = 0  # extra nets with log-uniform 2k..20k pins


WORKLOADS = {
    # 2,000 std cells + 4 macros, 2,100 nets, 200x200 dies, 64x64x2 bins.
    "cells_2k": Workload("cells_2k", 2000, 4, 2100, 200.0, 64, 64, 2, 1),
    # 200k std cells + 20 macros, 210k nets, 3,000x3,000 dies, 256x256x4 bins.
    "cells_200k": Workload("cells_200k", 200_000, 20, 210_000, 3000.0, 256, 256, 4, 2),
    # 1M std cells + 60 macros, 1.05M nets, 6,700x6,700 dies, 512x512x4 bins.
    "cells_1m": Workload("cells_1m", 1_000_000, 60, 1_050_000, 6700.0, 512, 512, 4, 3),
    # 4M std cells + 200 macros, 4.2M nets + 200 high-fanout nets, 1024x1024x4.
    "cells_4m_skewed": Workload("cells_4m_skewed", 4_000_000, 200, 4_200_000, 13400.0,
                                1024, 1024, 4, 5, n_hifanout=200),
}


def _degrees(rng: np.random.Generator, n: int) -> np.ndarray:
    probs = np.array([b[2] for b in _DEG_BUCKETS])
    which = rng.choice(len(_DEG_BUCKETS), size=n, p=probs / probs.sum())
    deg = np.empty(n, dtype=np.int64)
    for k, (lo, hi, _) in enumerate(_DEG_BUCKETS):
        sel = np.nonzero(which == k)[0]
        d = np.arange(lo, hi + 1)
        w = 1.0 / d.astype(np.float64) ** 2
        deg[sel] = rng.choice(d, size=sel.size, p=w / w.sum())
    return deg


def _distinct_pins(rng, net_start, n_std, n_macro, macro_frac):
    """Draw one instance per pin so that no net holds an instance twice."""
    n_net = net_start.size - 1
    deg = np.diff(net_start)
    P = int(net_start[-1])
    net_of = np.repeat(np.arange(n_net, dtype=np.int64), deg)
    n_inst = n_std + n_macro

    def draw(k):
        if n_macro > 0:
            mac = rng.random(k) < macro_frac
            return np.where(mac, n_std + rng.integers(0, n_macro, k), rng.integers(0, n_std, k))
        return rng.integers(0, n_std, k)

    inst = draw(P)
    for it in range(200):
        key = net_of * n_inst + inst
        order = np.argsort(key, kind="stable")
        dup = np.zeros(P, dtype=bool)
        ks = key[order]
        dup[order[1:]] = ks[1:] == ks[:-1]
        nd = int(dup.sum())
        if nd == 0:
            return inst
        idx = np.nonzero(dup)[0]
        if it < 100:
            inst[idx] = draw(nd)
        else:  # fall back to std cells only (a net asked for more macros than exist)
            inst[idx] = rng.integers(0, n_std, nd)
    raise RuntimeError("could not draw distinct pins")


def make_problem(wl: Workload | str, positions: str = "uniform", origin=(0.0, 0.0),
                 seed: int | None = None, n_std: int | None = None,
                 n_net: int | None = None) -> dict:
    """Return a problem dict (numpy arrays + scalars) and positions x, y, z.

    Keys follow the C ABI's ``place3d_problem`` field names.  ``positions`` is
    "uniform" or "center".  ``origin`` shifts the die outline (and positions).
    ``n_std``/``n_net`` override the workload's counts (smaller samples).
    """
    if isinstance(wl, str):
        wl = WORKLOADS[wl]
    if n_std is not None or n_net is not None:
        wl = dataclasses.replace(wl, n_std=n_std or wl.n_std, n_net=n_net or wl.n_net)
    rng = np.random.default_rng(wl.seed if seed is None else seed)
    d = float(wl.die)
    n_std, n_mac = wl.n_std, wl.n_macro
    n_inst = n_std + n_mac

    # --- sizes (bottom die; top die 0.8x) ---
    w_bot = np.empty(n_inst)
    h_bot = np.empty(n_inst)
    w_bot[:n_std] = rng.integers(1, 9, n_std).astype(np.float64)
    h_bot[:n_std] = 1.0
    if n_mac:
        side = math.sqrt(0.2 * d * d / n_mac)
        w_bot[n_std:n_std + n_mac] = side
        h_bot[n_std:n_std + n_mac] = side
    w_top = 0.8 * w_bot
    h_top = 0.8 * h_bot
    is_macro = np.zeros(n_inst, dtype=np.uint8)
    is_macro[n_std:n_std + n_mac] = 1
    z_fixed = np.zeros(n_inst, dtype=np.uint8)

    # --- netlist ---
    deg = _degrees(rng, wl.n_net)
    if wl.n_hifanout:
        hf = np.exp(rng.uniform(math.log(2000), math.log(20000), wl.n_hifanout)).astype(np.int64)
        deg = np.concatenate([deg, hf])
    net_start = np.zeros(deg.size + 1, dtype=np.int64)
    np.cumsum(deg, out=net_start[1:])
    pin_inst = _distinct_pins(rng, net_start, n_std, n_mac, 0.01)

    # --- instance order: interleave macros among cells ---
    perm = rng.permutation(n_inst)  # new index of old instance k is perm[k]
    inv = np.empty_like(perm)
    inv[perm] = np.arange(n_inst)
    w_bot, h_bot, w_top, h_top = (a[inv] for a in (w_bot, h_bot, w_top, h_top))
    is_macro, z_fixed = is_macro[inv], z_fixed[inv]
    pin_inst = perm[pin_inst]

    # --- pin offsets inside the bottom footprint; top offsets 0.8x ---
    P = pin_inst.size
    off_bx = (rng.random(P) - 0.5) * w_bot[pin_inst]
    off_by = (rng.random(P) - 0.5) * h_bot[pin_inst]
    off_tx = 0.8 * off_bx
    off_ty = 0.8 * off_by

    prob = dict(
        n_inst=n_inst, is_macro=is_macro, z_fixed=z_fixed,
        w_bot=w_bot, h_bot=h_bot, w_top=w_top, h_top=h_top,
        n_net=int(deg.size), n_pin=int(P),
        net_start=net_start.astype(np.int32), pin_inst=pin_inst.astype(np.int32),
        off_bx=off_bx, off_by=off_by, off_tx=off_tx, off_ty=off_ty,
        xl=float(origin[0]), yl=float(origin[1]),
        xh=float(origin[0]) + d, yh=float(origin[1]) + d,
        nx=wl.nx, ny=wl.ny, nz=wl.nz,
        gamma=4.0 * d / wl.nx, gamma_z=0.0, lam=1e-3,
        beta=10.0, w_hbt=1.0, rh_top=0.8, rh_bot=1.0,
        workload=wl.name,
    )
    x, y, z = draw_positions(rng, prob, positions)
    prob["x"], prob["y"], prob["z"] = x, y, z
    return prob


def depth_range(prob: dict) -> tuple[float, float]:
    """(z_lo, z_hi) = (d_z/4, 3 d_z/4) of the problem's grid (Sec. V-A bin depth)."""
    wb = (prob["xh"] - prob["xl"]) / prob["nx"]
    hb = (prob["yh"] - prob["yl"]) / prob["ny"]
    dz = prob["nz"] * 0.5 * (wb + hb)
    return 0.25 * dz, 0.75 * dz


def draw_positions(rng: np.random.Generator, prob: dict, kind: str = "uniform"):
    n = prob["n_inst"]
    xl, yl, xh, yh = prob["xl"], prob["yl"], prob["xh"], prob["yh"]
    zlo, zhi = depth_range(prob)
    w = np.maximum(prob["w_bot"], prob["w_top"])
    h = np.maximum(prob["h_bot"], prob["h_top"])
    if kind == "uniform":
        x = xl + w / 2 + rng.random(n) * np.maximum(xh - xl - w, 0.0)
        y = yl + h / 2 + rng.random(n) * np.maximum(yh - yl - h, 0.0)
        z = zlo + rng.random(n) * (zhi - zlo)
    elif kind == "center":
        x = np.clip(rng.normal(0.5 * (xl + xh), 0.1 * (xh - xl), n), xl, xh)
        y = np.clip(rng.normal(0.5 * (yl + yh), 0.1 * (yh - yl), n), yl, yh)
        z = np.clip(rng.normal(0.5 * (zlo + zhi), 0.2 * (zhi - zlo), n), zlo, zhi)
    else:
        raise ValueError(kind)
    return x, y, z


def append_fillers(prob: dict, fp: dict, seed: int = 0, positions: str = "center") -> dict:
    """A copy of prob with pinless filler instances appended: fp["n_top"]
    top z-fixed fillers at depth 3 d_z / 4, fp["n_bot"] bottom z-fixed fillers
    at d_z / 4, then fp["n_free"] free fillers; footprints fp["w_top"] x
    fp["h_top"] on the top die and fp["w_bot"] x fp["h_bot"] on the bottom
    one (a z-fixed filler keeps its own die's footprint in both tables).
    positions="center": x, y normal about the region's centre (sigma 0.1 of
    each extent), free fillers' z normal about d_z / 2 (sigma 0.2 of
    [d_z/4, 3 d_z/4]); "uniform": x, y uniform over the region, free
    fillers' z uniform in [d_z/4, 3 d_z/4].
    The counts and footprints are inputs: this draws positions and builds
    arrays only.  The result carries fp under "fillers" with the first
    filler's index."""
    n0 = int(prob["n_inst"])
    nt, nb, nf = int(fp["n_top"]), int(fp["n_bot"]), int(fp["n_free"])
    nfill = nt + nb + nf
    zlo, zhi = depth_range(prob)
    rng = np.random.default_rng(seed)
    out = dict(prob)

    def cat(k, vals, dt):
        return np.concatenate([np.asarray(prob[k], dt), np.asarray(vals, dt)])

    wt, ht = np.full(nfill, float(fp["w_top"])), np.full(nfill, float(fp["h_top"]))
    wb, hb = np.full(nfill, float(fp["w_bot"])), np.full(nfill, float(fp["h_bot"]))
    wb[:nt], hb[:nt] = fp["w_top"], fp["h_top"]
    wt[nt:nt + nb], ht[nt:nt + nb] = fp["w_bot"], fp["h_bot"]
    out["w_top"], out["h_top"] = cat("w_top", wt, np.float64), cat("h_top", ht, np.float64)
    out["w_bot"], out["h_bot"] = cat("w_bot", wb, np.float64), cat("h_bot", hb, np.float64)
    out["is_macro"] = cat("is_macro", np.zeros(nfill), np.uint8)
    zf0 = prob.get("z_fixed")
    zf0 = np.zeros(n0, np.uint8) if zf0 is None else np.asarray(zf0, np.uint8)
    out["z_fixed"] = np.concatenate([zf0, np.ones(nt + nb, np.uint8), np.zeros(nf, np.uint8)])
    if prob.get("is_hbt") is not None:  # a 2D problem: fillers are not HBTs
        out["is_hbt"] = np.concatenate([np.asarray(prob["is_hbt"], np.uint8), np.zeros(nfill, np.uint8)])
    xl, yl, xh, yh = prob["xl"], prob["yl"], prob["xh"], prob["yh"]
    fz = np.empty(nfill)
    fz[:nt] = zhi
    fz[nt:nt + nb] = zlo
    if positions == "center":
        fx = np.clip(rng.normal(0.5 * (xl + xh), 0.1 * (xh - xl), nfill), xl, xh)
        fy = np.clip(rng.normal(0.5 * (yl + yh), 0.1 * (yh - yl), nfill), yl, yh)
        fz[nt + nb:] = np.clip(rng.normal(0.5 * (zlo + zhi), 0.2 * (zhi - zlo), nf), zlo, zhi)
    elif positions == "uniform":
        fx = xl + rng.random(nfill) * (xh - xl)
        fy = yl + rng.random(nfill) * (yh - yl)
        fz[nt + nb:] = zlo + rng.random(nf) * (zhi - zlo)
    else:
        raise ValueError(positions)
    for k, v in (("x", fx), ("y", fy), ("z", fz)):
        if k in prob:
            out[k] = cat(k, v, np.float64)
    out["n_inst"] = n0 + nfill
    out["fillers"] = dict(fp, first=n0)
    return out


def make_batch(count: int = 24, seed: int = 4, n_min: int = 5000, n_max: int = 300_000) -> list:
    """Independent instances of uneven size: cell counts log-uniform in
    [n_min, n_max], macros 0.01 % of the cells (at least 1), nets 1.05 x the
    cells with the usual degree mix, dies 3,000 * sqrt(n / 200k) wide, grids
    N_x = N_y = the power of two nearest sqrt(n) clamped to [64, 512] and
    N_z = 2 for N_x <= 128, else 4."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        nm = max(1, int(round(1e-4 * n)))
        nxy = int(min(512, max(64, 2 ** round(math.log2(math.sqrt(n))))))
        wl = Workload(f"batch{k}", n, nm, int(1.05 * n), 3000.0 * math.sqrt(n / 200_000.0), nxy, nxy,
                      2 if nxy <= 128 else 4, seed * 1000 + k)
        out.append(make_problem(wl))
    return out


def to_problem2d(prob: dict, x=None, y=None, z=None, hbt_xy=None, seed: int = 0, lam_layer=None) -> dict:
    """The multi-die 2D form of a 3D problem at positions (x, y, z) (default
    the problem's own): the partition is the one z gives (top iff z > d_z/2
    of the 3D grid), the grid keeps N_x x N_y with N_z = 3 layers (bottom die,
    top die, HBT layer), and every net with pins on both dies gets one HBT
    instance (is_hbt = 1, a w_hbt x w_hbt square, no offsets) whose pin ends
    that net's pin list.  hbt_xy: (x, y) arrays of the HBT centres in
    crossing-net order, or None for uniform random centres in the region.
    z is rewritten to d_z/4 (bottom) or 3 d_z/4 (top) of the 3-layer grid.
    This only assembles arrays; it computes nothing of the method."""
    x = np.asarray(prob["x"] if x is None else x, np.float64)
    y = np.asarray(prob["y"] if y is None else y, np.float64)
    z = np.asarray(prob["z"] if z is None else z, np.float64)
    n = int(prob["n_inst"])
    zlo3, zhi3 = depth_range(prob)
    top = z > 0.5 * (zlo3 + zhi3)
    ns = np.asarray(prob["net_start"], np.int64)
    pi = np.asarray(prob["pin_inst"], np.int64)
    deg = np.diff(ns)
    net_of = np.repeat(np.arange(deg.size), deg)
    t_cnt = np.bincount(net_of, weights=top[pi].astype(np.float64), minlength=deg.size)
    cross = np.nonzero((t_cnt > 0) & (t_cnt < deg))[0]
    nh = cross.size
    rng = np.random.default_rng(seed)
    if hbt_xy is None:
        hx = prob["xl"] + rng.random(nh) * (prob["xh"] - prob["xl"])
        hy = prob["yl"] + rng.random(nh) * (prob["yh"] - prob["yl"])
    else:
        hx, hy = (np.asarray(a, np.float64) for a in hbt_xy)
    # netlist: the HBT pin appended to each crossing net
    extra = np.zeros(deg.size, np.int64)
    extra[cross] = 1
    new_deg = deg + extra
    new_ns = np.zeros(deg.size + 1, np.int64)
    np.cumsum(new_deg, out=new_ns[1:])
    P2 = int(new_ns[-1])
    new_pi = np.empty(P2, np.int64)
    offs = {k: np.zeros(P2) for k in ("off_bx", "off_by", "off_tx", "off_ty")}
    dst = np.repeat(new_ns[:-1], deg) + (np.arange(pi.size) - np.repeat(ns[:-1], deg))
    new_pi[dst] = pi
    for k in offs:
        offs[k][dst] = np.asarray(prob[k], np.float64)
    new_pi[new_ns[cross + 1] - 1] = n + np.arange(nh)
    w = float(prob.get("w_hbt", 1.0))
    wb = (prob["xh"] - prob["xl"]) / prob["nx"]
    hb = (prob["yh"] - prob["yl"]) / prob["ny"]
    dz2 = 3 * 0.5 * (wb + hb)
    out = dict(prob)
    for k in ("w_bot", "h_bot", "w_top", "h_top"):
        out[k] = np.concatenate([np.asarray(prob[k], np.float64), np.full(nh, w)])
    out["is_macro"] = np.concatenate([np.asarray(prob["is_macro"], np.uint8), np.zeros(nh, np.uint8)])
    zf = prob.get("z_fixed")
    out["z_fixed"] = np.concatenate([np.zeros(n, np.uint8) if zf is None else np.asarray(zf, np.uint8),
                                     np.zeros(nh, np.uint8)])
    out["is_hbt"] = np.concatenate([np.zeros(n, np.uint8), np.ones(nh, np.uint8)])
    out["n_inst"] = n + nh
    out["net_start"] = new_ns.astype(np.int32)
    out["pin_inst"] = new_pi.astype(np.int32)
    out["n_pin"] = P2
    out.update(offs)
    out["nz"] = 3
    out["mode"] = 1
    out["lam_layer"] = tuple(lam_layer) if lam_layer is not None else (prob["lam"],) * 3
    out["x"] = np.concatenate([x, hx])
    out["y"] = np.concatenate([y, hy])
    out["z"] = np.concatenate([np.where(top, 0.75 * dz2, 0.25 * dz2), np.full(nh, 0.5 * dz2)])
    out["hbt_nets"] = cross.astype(np.int64)
    return out
