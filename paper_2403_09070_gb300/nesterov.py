"""Nesterov placement loop over the place3d evaluation (Sec. III-A, the
gradient-based 3D global placement of Fig. overall-flow).

Per iteration: gradient at the reference solution, 3D mixed-size
preconditioning (eq. improved-precond), a Nesterov step with the step length
predicted from a Lipschitz estimate, and projection of the centres into the
region with z in [d_z/4, 3 d_z/4] (Sec. III-A movable range).  The density
weight lambda grows geometrically.

`run` drives the loop through the library's device helpers
(place3d_nesterov_update / _precondition: the step length never leaves the
GPU, no host synchronisation per iteration); `run_reference` is the same
loop written with torch operations over the autograd wrapper, kept as the
readable statement of the method and as the fused loop's test reference.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .autograd import Place3DObjective


def preconditioner(pins_per_inst, is_macro, q, lam):
    """Eq. improved-precond: H_ii = max(1, |E_i| + lambda q_i) for macros,
    max(1, lambda q_i) for every other instance."""
    return torch.where(is_macro, torch.clamp(pins_per_inst + lam * q, min=1.0), torch.clamp(lam * q, min=1.0))


class NesterovPlacer:
    def __init__(self, prob: dict, precision: str = "fp32_tc", device: int = 0, lam_mult: float = 1.05,
                 init_step_bins: float = 0.5):
        self.obj = Place3DObjective(prob, precision=precision, device=device)
        dev = torch.device("cuda", device)
        dt = self.obj.dtype
        self.p = prob
        g = self.obj.handle.geometry()
        self.g = g
        self.dev, self.dt = dev, dt
        t = lambda a, d=dt: torch.tensor(np.ascontiguousarray(a), dtype=d, device=dev)
        self.is_macro = t(prob["is_macro"], torch.bool)
        self.z_fixed = t(prob["z_fixed"], torch.bool) if prob.get("z_fixed") is not None else None
        self.w = (t(prob["w_bot"]), t(prob["w_top"]))
        self.h = (t(prob["h_bot"]), t(prob["h_top"]))
        pins = np.bincount(np.asarray(prob["pin_inst"]), minlength=prob["n_inst"]).astype(np.float64)
        self.pins = t(pins)
        self.lo = (prob["xl"], prob["yl"], 0.25 * g["dz"])
        self.hi = (prob["xh"], prob["yh"], 0.75 * g["dz"])
        self.lam_mult = lam_mult
        self.init_step = init_step_bins * min(g["wb"], g["hb"])

    def _q(self, z):
        top = z > 0.5 * self.g["dz"]
        w = torch.where(top, self.w[1], self.w[0])
        h = torch.where(top, self.h[1], self.h[0])
        return w * h * (0.5 * self.g["dz"])  # instance volume (Sec. III-A)

    def _project(self, v):
        for a in range(3):
            v[a].clamp_(self.lo[a], self.hi[a])
        return v

    def _grad(self, v):
        v = v.detach().requires_grad_(True)
        f = self.obj(v[0], v[1], v[2])
        (gv,) = torch.autograd.grad(f, v)
        H = preconditioner(self.pins, self.is_macro, self._q(v[2].detach()), self.obj.lam)
        gv = gv / H
        if self.z_fixed is not None:
            gv[2] = torch.where(self.z_fixed, torch.zeros_like(gv[2]), gv[2])
        return f.detach(), gv

    def run(self, x, y, z, iters: int = 100, log_every: int = 10, callback=None):
        """The loop on the device helpers.  Returns the final positions (a
        [3][n] tensor) and a history of (iter, obj, wl_bi, hpwl_d2d, energy,
        lambda); logging synchronises, every log_every iterations."""
        h = self.obj.handle
        n = self.p["n_inst"]
        u = self._project(torch.stack([torch.as_tensor(a, dtype=self.dt, device=self.dev) for a in (x, y, z)]))
        u = u.contiguous()
        v = u.clone()
        g = torch.empty((3, n), dtype=self.dt, device=self.dev)
        h.set_positions(v[0], v[1], v[2])
        h.eval(sync=False)  # the gradient stays in the handle, where the helpers read it
        h.nesterov_init(g, self.init_step)
        a = 1.0
        hist = []
        for k in range(iters):
            a_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * a * a))
            h.nesterov_update(u, v, g, (a - 1.0) / a_new)  # also the next positions
            h.eval(sync=False)
            h.nesterov_precondition(g)
            a = a_new
            if log_every and (k % log_every == 0 or k == iters - 1):
                h.result_to_device(self.obj.scalars)
                s = self.obj.last_scalars()
                hist.append((k, s["obj"], s["wl_bi"], s["hpwl_d2d"], s["energy"], self.obj.lam))
                if callback:
                    callback(k, s)
            self.obj.set_params(lam=self.obj.lam * self.lam_mult)
        return u, hist

    def run_reference(self, x, y, z, iters: int = 100, log_every: int = 10, callback=None):
        """The same loop with torch operations.  Returns the final positions
        and a history of (iter, obj, wl_bi, hpwl_d2d, energy, lambda)."""
        u = self._project(torch.stack([torch.as_tensor(a, dtype=self.dt, device=self.dev) for a in (x, y, z)]))
        v = u.clone()
        a = 1.0
        f, gv = self._grad(v)
        step = self.init_step / max(float(gv.abs().max()), 1e-30)
        hist = []
        for k in range(iters):
            u_new = self._project(v - step * gv)
            a_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * a * a))
            v_new = self._project(u_new + ((a - 1.0) / a_new) * (u_new - u))
            f_new, g_new = self._grad(v_new)
            # Lipschitz step-size estimate in FP64 (the positions and gradients may be FP32)
            dv = float(torch.linalg.vector_norm((v_new - v).double()))
            dg = float(torch.linalg.vector_norm((g_new - gv).double()))
            if dg > 0 and dv > 0:
                step = dv / dg  # inverse Lipschitz estimate
            u, v, gv, a = u_new, v_new, g_new, a_new
            if log_every and (k % log_every == 0 or k == iters - 1):
                s = self.obj.last_scalars()
                hist.append((k, s["obj"], s["wl_bi"], s["hpwl_d2d"], s["energy"], self.obj.lam))
                if callback:
                    callback(k, s)
            self.obj.set_params(lam=self.obj.lam * self.lam_mult)
        return u, hist
