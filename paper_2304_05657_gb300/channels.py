"""Host-side observables of the channel studies (Sec. IV.A): per-channel
flame position and heat release of a batch of channels packed along y,
flame speed from the flame position history, the quenching width, and the
inflow control that holds a flame in place (the flow rate "dynamically set
to match the flame propagation speed").

All reductions run on the GPU (lbfd_diagnostics_rows); this module only
keeps histories and does the bookkeeping.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def channel_diagnostics(solver, segments) -> list:
    """Diagnostics of every channel (segments = [(y0, y1), ...])."""
    return [solver.diagnostics(rows=seg) for seg in segments]


@dataclass
class FlameSpeedTracker:
    """Flame speed S_F = u_in - dx_f/dt of each channel (lattice units),
    x_f the unburnt length; converted to m/s with dx/dt."""

    segments: list
    times: list = field(default_factory=list)
    xf: list = field(default_factory=list)
    hrr: list = field(default_factory=list)
    u_in: list = field(default_factory=list)

    def record(self, solver, step: int):
        d = channel_diagnostics(solver, self.segments)
        self.times.append(step)
        self.xf.append([c["x_f"] for c in d])
        self.hrr.append([c["heat_release"] for c in d])
        self.u_in.append(solver.cfg["u_in"])

    def flame_speed(self, window: int = 5) -> np.ndarray:
        """Mean S_F over the last `window` records, per channel (lattice)."""
        t = np.asarray(self.times[-window:], dtype=np.float64)
        x = np.asarray(self.xf[-window:], dtype=np.float64)
        u = np.asarray(self.u_in[-window:], dtype=np.float64)
        if len(t) < 2:
            raise ValueError("need at least two records")
        slope = np.polyfit(t - t[0], x, 1)[0]
        return u.mean() - slope

    def burning(self, rel: float = 1e-3) -> np.ndarray:
        """Channels whose heat release is above rel x the largest one."""
        h = np.asarray(self.hrr[-1])
        return h > rel * max(h.max(), 1e-300)


def dead_zone(peak, wall_distance, rel: float = 0.1) -> float:
    """Dead-zone thickness delta_dead of one channel (Sec. IV.A): the
    smallest distance between the reaction front (the peak heat release of
    each column across the channel) and a wall, over the columns where the
    front burns (peak >= rel x the channel's largest); nan when nothing
    burns.  Inputs: the two arrays of lbfd_column_peaks for the channel."""
    peak = np.asarray(peak, dtype=np.float64)
    top = peak.max() if peak.size else 0.0
    if not top > 0.0:
        return float("nan")
    sel = peak >= rel * top
    return float(np.asarray(wall_distance, dtype=np.float64)[sel].min())


def channel_dead_zones(solver, segments, rel: float = 0.1) -> list:
    """delta_dead [cells] of every channel (segments = [(y0, y1), ...])."""
    return [dead_zone(*solver.column_peaks(seg), rel=rel) for seg in segments]


def quenching_width(widths, burning) -> float:
    """Smallest width that still burns, given per-channel burning flags of
    channels sorted by width (nan if none burns)."""
    w = np.asarray(widths, dtype=np.float64)
    b = np.asarray(burning, dtype=bool)
    return float(w[b].min()) if b.any() else float("nan")


@dataclass
class InflowController:
    """Proportional-integral control of the inlet velocity on the flame
    position, in incremental form: u_k = u_{k-1} + kp (e_k - e_{k-1}) +
    ki e_k with e = x_target - x_f.  If the flame drifts downstream (x_f
    above the target) the inflow slows down, and vice versa.  The flame
    position integrates u_in - S_F, so this PI loop settles with x_f at the
    target and u_in equal to the flame speed."""

    x_target: float          # unburnt length to hold [cells]
    kp: float = 1e-3         # per cell of error change
    ki: float = 2e-5         # per cell of error and per update
    u_min: float = 0.0
    u_max: float = 0.1
    last_err: float | None = None

    def update(self, solver, rows=None) -> float:
        xf = solver.diagnostics(rows=rows)["x_f"]
        err = self.x_target - xf  # > 0: flame too close to the inlet -> more inflow
        de = 0.0 if self.last_err is None else err - self.last_err
        self.last_err = err
        u = solver.cfg["u_in"] + self.kp * de + self.ki * err
        u = float(min(max(u, self.u_min), self.u_max))
        solver.set_inlet_velocity(u)
        return u


def hold_flame(solver, controller: InflowController, steps: int, every: int = 50, rows=None):
    """Advance `steps` steps, updating the inlet velocity every `every`
    steps; returns the (step, x_f, u_in) history."""
    hist = []
    done = 0
    while done < steps:
        n = min(every, steps - done)
        solver.step(n)
        done += n
        u = controller.update(solver, rows)
        hist.append((solver.steps_done, solver.diagnostics(rows=rows)["x_f"], u))
    return hist
