"""Gradients of flame observables with respect to the model parameters
theta = (ln A, Ta, T_wall, u_in), behind a torch.autograd.Function.

Two ways through the library:
  - forward mode ("tangent", "tangent_mixed"): every state value carries its
    four derivatives through the discrete step, so the gradient is ready
    when the forward pass ends and backward only scales it;
  - the discrete adjoint ("adjoint": FP64, "adjoint_mixed": FP32 forward
    pass with the adjoint and the gradient accumulated in FP64): the
    forward pass advances the state keeping a checkpoint every
    `checkpoint_every` steps and returns J; backward sweeps the steps in
    reverse (each segment recomputed from its checkpoint) with the
    incoming gradient as the adjoint's seed.
Objectives: flame position x_f [m] (Sec. IV.A), total heat release
(forward mode only), and the quenching distance (a heat-release-weighted
soft minimum of the distance to the cold walls, for the dead zone of
Sec. IV.A).
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


ADJOINT = {"adjoint": "fp64", "adjoint_mixed": "mixed"}


def run_tangent(cfg: dict, solid, T0, Y0, steps: int, objective: int = lbfd.OBJ_FLAME_POSITION, theta=None,
                precision: str = "tangent", checkpoint_every: int = 200):
    """J after `steps` steps from (T0, Y0, g = 0) and dJ/dtheta."""
    if precision in ADJOINT:
        return run_adjoint(cfg, solid, T0, Y0, steps, objective, theta, checkpoint_every, ADJOINT[precision])
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


def adjoint_solver(cfg: dict, solid, T0, Y0, theta=None, checkpoint_every: int = 200, forward: str = "fp64"):
    """A handle at (T0, Y0, g = 0) with theta applied, ready to record."""
    c = apply_theta(cfg, theta) if theta is not None else dict(cfg)
    c["precision"] = forward
    s = lbfd.Solver(c, solid)
    s.init_fields(T0, Y0)
    s.adjoint_setup(checkpoint_every)
    return s


def run_adjoint(cfg: dict, solid, T0, Y0, steps: int, objective: int = lbfd.OBJ_FLAME_POSITION, theta=None,
                checkpoint_every: int = 200, forward: str = "fp64"):
    """The same (J, dJ/dtheta) by the discrete adjoint; forward "fp64" or
    "mixed" (FP32 forward pass, FP64 adjoint)."""
    s = adjoint_solver(cfg, solid, T0, Y0, theta, checkpoint_every, forward)
    J, g = s.adjoint_run(steps, objective)
    s.close()
    return J, g


try:
    import torch

    class FlameObjective(torch.autograd.Function):
        """J(theta) = an objective after `steps` steps from (T0, Y0, g = 0).

        forward(theta[4] float64 tensor, cfg, solid, T0, Y0, steps, objective,
        precision, checkpoint_every).  precision "tangent"/"tangent_mixed":
        forward mode, the gradient is computed with J.  "adjoint"/
        "adjoint_mixed": forward keeps only checkpoints, backward runs the
        reverse sweep seeded with the incoming gradient."""

        @staticmethod
        def forward(ctx, theta, cfg, solid, T0, Y0, steps, objective=lbfd.OBJ_FLAME_POSITION, precision="tangent",
                    checkpoint_every=200):
            th = theta.detach().cpu().numpy()
            ctx.solver = None
            if precision in ADJOINT:
                s = adjoint_solver(cfg, solid, T0, Y0, th, int(checkpoint_every), ADJOINT[precision])
                J = s.adjoint_record(int(steps), int(objective))
                ctx.solver = s
                ctx.save_for_backward(theta)
            else:
                J, g = run_tangent(cfg, solid, T0, Y0, int(steps), int(objective), th, precision)
                ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            return theta.new_tensor(J)

        @staticmethod
        def backward(ctx, grad_out):
            (saved,) = ctx.saved_tensors
            if ctx.solver is not None:
                g = ctx.solver.adjoint_backward(float(grad_out))
                ctx.solver.close()
                ctx.solver = None
                return (torch.as_tensor(g, dtype=saved.dtype, device=saved.device),) + (None,) * 8
            return (grad_out * saved,) + (None,) * 8

except ImportError:  # torch is optional for the C-ABI user
    FlameObjective = None
