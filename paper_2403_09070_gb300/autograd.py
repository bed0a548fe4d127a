"""torch.autograd wrapper of the place3d evaluation (differentiation row of the
hot path: a torch optimiser drives placement through the CUDA kernels).

The forward enqueues ONE fused evaluation of the C ABI: the objective of eq.
analytical-placement and its gradient come out of the same sweep (the
per-net WA exponentials are recomputed per pin in registers, never stored,
so there is no per-pin state beyond the netlist itself).  The gradient is
saved and the backward scales it by the incoming gradient.

Note the z component is the paper's normalised finite-difference depth
gradient plus alpha dp^(z)/dz plus lambda dU/dz (eqs. fda-grad,
fda-normalize), not the derivative of the returned objective: the bistratal
wirelength is a step function of z (Sec. III-A).  Likewise the density part
of every component is the field gather (force q_i E_i), which approximates
the derivative of the discrete energy.
"""
from __future__ import annotations

import torch

from . import place3d as P


class Place3DFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, y, z, handle, scalars):
        g = [torch.empty_like(x) for _ in range(3)]
        handle.set_positions(x, y, z)
        handle.eval(*g, sync=False)
        handle.result_to_device(scalars)
        ctx.save_for_backward(*g)
        return scalars[0].to(x.dtype).clone()

    @staticmethod
    def backward(ctx, go):
        gx, gy, gz = ctx.saved_tensors
        return go * gx, go * gy, go * gz, None, None


class Place3DObjective(torch.nn.Module):
    """f(x, y, z) of one placement problem as a differentiable torch module.

    precision: "fp64", "fp32" or "fp32_tc"; positions are CUDA tensors of the
    matching dtype (float64 for fp64, float32 otherwise)."""

    def __init__(self, prob: dict, precision: str = "fp32_tc", device: int = 0, alpha=None, flags: int = 0):
        super().__init__()
        self.handle = P.Place3D(prob, precision=precision, device=device,
                                stream=torch.cuda.current_stream(device), alpha=alpha, flags=flags)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.scalars = torch.zeros(10, dtype=torch.float64, device=f"cuda:{device}")
        self.gamma, self.gamma_z = float(prob["gamma"]), float(prob.get("gamma_z", 0.0))
        self.alpha, self.lam = self.handle.alpha, float(prob["lam"])

    def set_params(self, gamma=None, lam=None, gamma_z=None, alpha=None):
        self.gamma = self.gamma if gamma is None else float(gamma)
        self.lam = self.lam if lam is None else float(lam)
        self.gamma_z = self.gamma_z if gamma_z is None else float(gamma_z)
        self.alpha = self.alpha if alpha is None else float(alpha)
        self.handle.set_params(self.gamma, self.gamma_z, self.alpha, self.lam)

    def forward(self, x, y, z):
        return Place3DFunction.apply(x, y, z, self.handle, self.scalars)

    def last_scalars(self) -> dict:
        """The last evaluation's scalars (synchronises)."""
        keys = ("obj", "wl_bi", "wl_z", "energy", "hpwl_d2d", "n_cross", "g_scale", "s_x", "s_y", "s_z")
        return dict(zip(keys, self.scalars.tolist()))
