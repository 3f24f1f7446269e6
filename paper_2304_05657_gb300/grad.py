"""Gradients of flame observables with respect to the model parameters
theta = (ln A, Ta, T_wall, u_in), behind a torch.autograd.Function.

The forward pass runs the coupled step in the library's tangent precision
(every state value carries its four derivatives, propagated exactly through
the discrete step), so the gradient is ready when the forward pass ends;
backward only scales it by the incoming gradient.  With four parameters
this needs one pass and no stored trajectory.  precision "tangent" is FP64
throughout; "tangent_mixed" runs the forward pass in FP32 (FP64 Arrhenius
above T_fp64) and accumulates the objective and its gradient in FP64.
precision "adjoint" computes the same gradient of the flame position in
reverse mode (the discrete adjoint, FP64, checkpoints every
`checkpoint_every` steps and recomputation of each segment).
"""
from __future__ import annotations

import math

import numpy as np

from . import lbfd


def apply_theta(cfg: dict, theta) -> dict:
    """Configuration with theta = (ln A, Ta, T_wall, u_in) substituted;
    T_wall sets every isothermal wall face and the solid temperature."""
    lnA, Ta, Tw, u_in = (float(t) for t in theta)
    out = dict(cfg)
    out["A"] = math.exp(lnA)
    out["Ta"] = Ta
    out["T_wall"] = [Tw if b == "wall_isothermal" else cfg["T_wall"][f] for f, b in enumerate(cfg["bc"])]
    out["T_solid"] = Tw if cfg["solid_isothermal"] else cfg["T_solid"]
    out["u_in"] = u_in
    return out


def theta_of(cfg: dict):
    walls = [cfg["T_wall"][f] for f, b in enumerate(cfg["bc"]) if b == "wall_isothermal"]
    Tw = walls[0] if walls else cfg["T_solid"]
    return np.array([math.log(cfg["A"]), cfg["Ta"], Tw, cfg["u_in"]])


def run_tangent(cfg: dict, solid, T0, Y0, steps: int, objective: int = lbfd.OBJ_FLAME_POSITION, theta=None,
                precision: str = "tangent", checkpoint_every: int = 200):
    """J after `steps` steps from (T0, Y0, g = 0) and dJ/dtheta."""
    if precision == "adjoint":
        return run_adjoint(cfg, solid, T0, Y0, steps, objective, theta, checkpoint_every)
    if precision not in ("tangent", "tangent_mixed"):
        raise ValueError(precision)
    c = apply_theta(cfg, theta) if theta is not None else dict(cfg)
    c["precision"] = precision
    s = lbfd.Solver(c, solid)
    s.init_fields(T0, Y0)
    s.step(steps)
    J, g = s.gradient(objective)
    s.close()
    return J, g


def run_adjoint(cfg: dict, solid, T0, Y0, steps: int, objective: int = lbfd.OBJ_FLAME_POSITION, theta=None,
                checkpoint_every: int = 200):
    """The same (J, dJ/dtheta) by the discrete adjoint (FP64)."""
    c = apply_theta(cfg, theta) if theta is not None else dict(cfg)
    c["precision"] = "fp64"
    s = lbfd.Solver(c, solid)
    s.init_fields(T0, Y0)
    J, g = s.adjoint_gradient(steps, checkpoint_every, objective)
    s.close()
    return J, g


try:
    import torch

    class FlameObjective(torch.autograd.Function):
        """J(theta) = flame position (or heat release) after `steps` steps.

        forward(theta[4] float64 tensor, cfg, solid, T0, Y0, steps, objective,
        precision)."""

        @staticmethod
        def forward(ctx, theta, cfg, solid, T0, Y0, steps, objective=lbfd.OBJ_FLAME_POSITION, precision="tangent"):
            J, g = run_tangent(cfg, solid, T0, Y0, int(steps), int(objective), theta.detach().cpu().numpy(),
                               precision)
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            return theta.new_tensor(J)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None, None, None, None, None, None, None

except ImportError:  # torch is optional for the C-ABI user
    FlameObjective = None
