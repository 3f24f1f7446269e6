"""Host-side logic that needs no GPU: the synthetic input recipes, the
channel bookkeeping (flame speed, burning flags, quenching width, inflow
control) against a stand-in solver, the parameter plumbing of the gradient
wrapper, and the bench's traffic record lookup."""
import json
import math

import numpy as np
import pytest

import bench
from paper_2304_05657_gb300 import channels, grad, inputs


def test_batched_channels_recipe():
    cfg, solid, T, Y, seg = inputs.batched_channels()
    widths = [y1 - y0 for y0, y1 in seg]
    assert widths == list(range(16, 197, 12))  # 16 widths, 16 .. 196 step 12
    ny, nx = solid.shape
    assert nx == 1024 and ny == sum(widths) + len(widths) - 1
    for (y0, y1), (z0, _) in zip(seg[:-1], seg[1:]):  # one solid row between channels
        assert z0 == y1 + 1 and solid[y1].all()
    assert not solid[seg[0][0]:seg[0][1]].any()
    fluid = solid == 0
    assert np.allclose(Y.sum(axis=0)[fluid.ravel()], 1.0, atol=1e-12)
    assert T[fluid.ravel()].min() >= cfg["T_in"] - 1e-9


def test_sphere_packing_is_seeded_and_hits_its_porosity():
    a = inputs.sphere_packing(nx=48, ny=24, nz=24, x_range=(8, 40), r_range=(3.0, 5.0), seed=11)
    b = inputs.sphere_packing(nx=48, ny=24, nz=24, x_range=(8, 40), r_range=(3.0, 5.0), seed=11)
    c = inputs.sphere_packing(nx=48, ny=24, nz=24, x_range=(8, 40), r_range=(3.0, 5.0), seed=12)
    assert np.array_equal(a[1], b[1]) and not np.array_equal(a[1], c[1])
    slab = a[1][:, :, 8:40]
    porosity = 1.0 - slab.mean()
    assert 0.75 <= porosity <= 0.80
    assert not a[1][:, :, :8].any() and not a[1][:, :, 40:].any()


class FakeSolver:
    """The two calls the channel helpers make, with a flame front that moves
    at a set speed against the inflow."""

    def __init__(self, S_L):
        self.cfg = {"u_in": 0.0}
        self.S_L = S_L
        self.x = 50.0
        self.steps_done = 0

    def step(self, n):
        # the front moves upstream at S_L through gas moving downstream at
        # u_in: the unburnt length changes at u_in - S_L
        self.x += n * (self.cfg["u_in"] - self.S_L)
        self.steps_done += n

    def diagnostics(self, rows=None):
        return {"x_f": self.x, "heat_release": 1.0}

    def set_inlet_velocity(self, u):
        self.cfg["u_in"] = u


def test_flame_speed_tracker_recovers_the_front_speed():
    s = FakeSolver(S_L=0.004)
    s.cfg["u_in"] = 0.001
    tr = channels.FlameSpeedTracker(segments=[None])
    for _ in range(6):
        tr.record(s, s.steps_done)
        s.step(100)
    # S_F = u_in - dx_f/dt recovers S_L
    assert tr.flame_speed(window=5)[0] == pytest.approx(0.004, abs=1e-12)


def test_burning_flags_and_quenching_width():
    tr = channels.FlameSpeedTracker(segments=[0, 1, 2, 3])
    tr.hrr.append([0.0, 1e-9, 0.5, 1.0])
    assert list(tr.burning(rel=1e-3)) == [False, False, True, True]
    assert channels.quenching_width([16, 28, 40, 52], [False, False, True, True]) == 40.0
    assert math.isnan(channels.quenching_width([16, 28], [False, False]))


def test_inflow_controller_holds_the_front():
    """On a front that integrates u_in - S_L the controller settles: x_f at
    the target and u_in at the flame speed (an accumulating P + I form, which
    integrates the error twice, keeps oscillating on this plant)."""
    s = FakeSolver(S_L=0.004)
    ctl = channels.InflowController(x_target=50.0)
    hist = channels.hold_flame(s, ctl, steps=40000, every=50)
    assert abs(hist[-1][1] - 50.0) < 1e-3  # the front is held
    assert hist[-1][2] == pytest.approx(0.004, rel=1e-3)  # u_in equals the flame speed
    xs = [h[1] for h in hist[-100:]]
    assert max(xs) - min(xs) < 1e-3  # no limit cycle


def test_theta_round_trip():
    cfg, solid, T, Y = inputs.channel(nx=32, ny=10, walls="isothermal", T_wall=350.0)
    th = grad.theta_of(cfg)
    c2 = grad.apply_theta(cfg, th + np.array([0.1, 100.0, 5.0, 0.001]))
    assert grad.theta_of(c2) == pytest.approx(th + np.array([0.1, 100.0, 5.0, 0.001]), rel=1e-14)
    assert c2["A"] == pytest.approx(cfg["A"] * math.exp(0.1), rel=1e-14)
    assert all(t == 355.0 for t, b in zip(c2["T_wall"], c2["bc"]) if b == "wall_isothermal")
    with pytest.raises(ValueError):
        grad.run_tangent(cfg, solid, T, Y, 1, precision="fp64")


def test_traffic_record_only_for_the_recorded_sources(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 64 and h == bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"w": {"csrc_sha256": h, "precision": "mixed", "dram_bytes_per_step": {"5": 100.0},
                 "warp_instructions_per_step": {"5": 7.0}, "scale_to_workload": 2.0}}
    (prof / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.measured_traffic("w", 5, "mixed")[0] == 200.0
    assert bench.measured_instructions("w", 5, "mixed") == 14.0
    assert bench.measured_traffic("w", 6, "mixed")[0] is None
    assert bench.measured_traffic("w", 5, "fp64")[0] is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.measured_traffic("w", 5, "mixed")[0] is None
    assert bench.measured_instructions("w", 5, "mixed") is None


def test_dead_zone_from_column_peaks():
    """delta_dead is the smallest front-to-wall distance over the columns
    whose peak heat release is at least 10 % of the channel's largest."""
    from paper_2304_05657_gb300 import channels

    peak = np.array([0.0, 0.05, 1.0, 2.0, 0.3, 0.01])
    dist = np.array([0.5, 0.5, 3.5, 6.5, 2.5, 0.5])
    assert channels.dead_zone(peak, dist) == 2.5  # columns 2, 3, 4 burn
    assert channels.dead_zone(peak, dist, rel=0.6) == 6.5
    assert np.isnan(channels.dead_zone(np.zeros(4), np.ones(4)))
