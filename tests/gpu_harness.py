"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle import Oracle
from paper_2403_09070_gb300 import place3d as P

Q = 2.0 ** -36


def rel_max(a, b):
    """max |a - b| / max |b| (0 when both are 0)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.abs(b).max() if b.size else 0.0
    num = np.abs(a - b).max() if b.size else 0.0
    return 0.0 if num == 0 else num / max(den, 1e-300)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    num = np.linalg.norm(a - b)
    return 0.0 if num == 0 else num / max(den, 1e-300)


def run_gpu(prob, x, y, z, precision="fp64", alpha=None, maps=True, pos_dtype=None, flags=0,
            autotune=False):
    """Create a handle, evaluate once, return scalars, gradient, maps."""
    with P.Place3D(prob, precision=precision, alpha=alpha, flags=flags) as h:
        dt = pos_dtype or (np.float64 if precision == "fp64" else np.float32)
        h.set_positions(np.asarray(x, dt), np.asarray(y, dt), np.asarray(z, dt))
        if autotune:
            h.autotune(1)
        gdt = np.float64 if precision == "fp64" else np.float32
        g = [np.zeros(prob["n_inst"], gdt) for _ in range(3)]
        r = h.eval(*g)
        out = dict(res=r, gx=g[0], gy=g[1], gz=g[2], alpha=h.alpha)
        if maps:
            out["q"] = h.copy_map(P.MAP_RHO_FIXED)
            out["ex"], out["ey"], out["ez"] = (h.copy_map(m) for m in (P.MAP_EX, P.MAP_EY, P.MAP_EZ))
            out["wl"] = h.wl_parts()
        out["launches"] = h.launches_per_eval()
        out["forms"] = h.wl_forms()
    return out


def run_oracle(prob, x, y, z, alpha, density_mode=1, fd_mode=1):
    o = Oracle(prob, alpha=alpha)
    r = o.eval(x, y, z, density_mode=density_mode, fd_mode=fd_mode)
    return o, r
