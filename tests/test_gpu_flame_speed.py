"""Flame speed of the mixed-precision form (FP32 storage and arithmetic,
FP64 Arrhenius source above 1000 K) against the FP64 oracle: within 0.5 %.

The flame speed is S_F = u_in - dx_f/dt (Sec. IV.A: the flame is located
from its unburnt fuel; x_f is the unburnt length), with dx_f/dt the
least-squares slope of x_f sampled over a window, which averages out the
acoustic ringing of the expanding gas.  Two flames: the 256x32 adiabatic
channel ignited at the inlet (2000 steps, window 1000-2000), and the 1-D
planar flame held near its place by an inflow below its speed (the
standard grid of the oracle's convergence test)."""
import numpy as np
import pytest

from paper_2304_05657_gb300 import inputs

pytestmark = pytest.mark.gpu


def speed(ts, xs, u_in):
    return u_in - np.polyfit(ts, xs, 1)[0]


def history(sim, steps0, chunk, nsamp, step, diag):
    step(sim, steps0)
    ts, xs = [], []
    for i in range(nsamp + 1):
        ts.append(i * chunk)
        xs.append(diag(sim))
        if i < nsamp:
            step(sim, chunk)
    return np.array(ts), np.array(xs)


def gpu_history(lbfd, cfg, solid, T, Y, precision, steps0, chunk, nsamp):
    s = lbfd.Solver(dict(cfg, precision=precision), solid)
    s.init_fields(T, Y)
    out = history(s, steps0, chunk, nsamp, lambda m, n: m.step_graph(n) if n else None,
                  lambda m: m.diagnostics()["x_f"])
    s.close()
    return out


def oracle_history(oracle_mod, cfg, solid, T, Y, steps0, chunk, nsamp):
    import os

    oracle_mod.set_threads(os.cpu_count() or 1)
    try:
        o = oracle_mod.Sim(cfg, solid)
        o.set_state(T, Y)
        return history(o, steps0, chunk, nsamp, lambda m, n: m.step(n) if n else None,
                       lambda m: m.diagnostics()["x_f"])
    finally:
        oracle_mod.set_threads(1)


def test_channel_flame_speed_mixed_vs_oracle(lbfd_lib, oracle_mod):
    cfg, solid, T, Y = inputs.channel(nx=256, ny=32)
    T, Y = inputs.ignition_fields(cfg, solid, 0, 20, burnt=False)
    args = (1000, 50, 20)
    to, xo = oracle_history(oracle_mod, cfg, solid, T, Y, *args)
    tm, xm = gpu_history(lbfd_lib, cfg, solid, T, Y, "mixed", *args)
    td, xd = gpu_history(lbfd_lib, cfg, solid, T, Y, "fp64", *args)
    So, Sm, Sd = (speed(t, x, cfg["u_in"]) for t, x in ((to, xo), (tm, xm), (td, xd)))
    assert So > 0.01  # the flame runs (and pushes fresh gas out of the outlet)
    assert abs(Sm - So) <= 5e-3 * abs(So), (Sm, So)
    assert abs(Sd - So) <= 1e-9 * abs(So), (Sd, So)


def test_planar_flame_speed_mixed_vs_oracle(lbfd_lib, oracle_mod):
    nx = 120
    cfg = inputs.base_config(dim=2, nx=nx, ny=1, u_in=0.0018,
                             bc=["inlet", "outlet_pressure", "periodic", "periodic", "periodic", "periodic"])
    T_ad = cfg["T_in"] + cfg["Q"] * cfg["Y_in"][0] / cfg["cp"]
    solid = np.zeros((1, nx), np.uint8)
    T, Y = inputs.ignition_fields(cfg, solid, nx - 30, nx + 10, T_hot=T_ad, burnt=True)
    args = (20000, 250, 80)
    to, xo = oracle_history(oracle_mod, cfg, solid, T, Y, *args)
    tm, xm = gpu_history(lbfd_lib, cfg, solid, T, Y, "mixed", *args)
    So, Sm = speed(to, xo, cfg["u_in"]), speed(tm, xm, cfg["u_in"])
    assert 0.002 < So < 0.003
    assert abs(Sm - So) <= 5e-3 * So, (Sm, So)
