"""Small hand-built problems for tests (inputs only, no method arithmetic)."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def problem(sizes, nets=(), offsets=None, die=(0.0, 0.0, 10.0, 10.0), grid=(8, 8, 2),
            macros=(), z_fixed=(), gamma=1.0, gamma_z=0.0, lam=1e-3):
    """sizes: list of (w_bot, h_bot, w_top, h_top); nets: list of instance lists;
    offsets: per pin (obx, oby, otx, oty) in net order, default zeros."""
    n = len(sizes)
    s = np.asarray(sizes, dtype=np.float64).reshape(n, 4) if n else np.zeros((0, 4))
    is_macro = np.zeros(n, np.uint8)
    is_macro[list(macros)] = 1
    zf = np.zeros(n, np.uint8)
    zf[list(z_fixed)] = 1
    net_start = np.zeros(len(nets) + 1, np.int32)
    for e, pins in enumerate(nets):
        net_start[e + 1] = net_start[e] + len(pins)
    pin_inst = np.array([i for pins in nets for i in pins], np.int32)
    P = pin_inst.size
    off = np.zeros((P, 4)) if offsets is None else np.asarray(offsets, np.float64).reshape(P, 4)
    return dict(n_inst=n, is_macro=is_macro, z_fixed=zf,
                w_bot=s[:, 0].copy(), h_bot=s[:, 1].copy(), w_top=s[:, 2].copy(), h_top=s[:, 3].copy(),
                n_net=len(nets), n_pin=P, net_start=net_start, pin_inst=pin_inst,
                off_bx=off[:, 0].copy(), off_by=off[:, 1].copy(),
                off_tx=off[:, 2].copy(), off_ty=off[:, 3].copy(),
                xl=die[0], yl=die[1], xh=die[2], yh=die[3], nx=grid[0], ny=grid[1], nz=grid[2],
                gamma=gamma, gamma_z=gamma_z, lam=lam, beta=10.0, w_hbt=1.0, rh_top=0.8, rh_bot=1.0)


def dz_of(p):
    wb = (p["xh"] - p["xl"]) / p["nx"]
    hb = (p["yh"] - p["yl"]) / p["ny"]
    return p["nz"] * 0.5 * (wb + hb)


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows
