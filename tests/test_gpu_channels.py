"""Batched channels, per-channel diagnostics and inflow control on the GPU."""
import numpy as np
import pytest

from paper_2304_05657_gb300 import channels, inputs

pytestmark = pytest.mark.gpu


def test_row_diagnostics_equal_separate_oracle_channels(lbfd_lib, oracle_mod):
    """Each channel of a packed batch gives the diagnostics of the same
    channel run alone by the oracle (the solid separators are isothermal
    walls at the wall temperature, so the problems are independent)."""
    widths = [5, 8, 13]
    cfg, solid, T, Y, seg = inputs.batched_channels(widths=widths, length=45, ignite=(10, 25), closed_end=False,
                                                     u_in=0.01)
    s = lbfd_lib.Solver(cfg, solid)
    s.init_fields(T, Y)
    s.step(40)
    got = channels.channel_diagnostics(s, seg)
    for (y0, y1), w, d in zip(seg, widths, got):
        c1, s1, T1, Y1 = inputs.channel(nx=45, ny=w, walls="isothermal", T_wall=cfg["T_wall"][2], ignite=(10, 25))
        o = oracle_mod.Sim(c1, s1)
        o.set_state(T[y0 * 45:y1 * 45], Y[:, y0 * 45:y1 * 45])
        o.step(40)
        do = o.diagnostics()
        for key in ("x_f", "mass", "heat_release", "fuel_consumption", "T_max"):
            assert abs(d[key] - do[key]) <= 1e-11 * max(1.0, abs(do[key])), (w, key, d[key], do[key])
        assert d["n_fluid"] == do["n_fluid"] and d["x_hrr_max"] == do["x_hrr_max"]
    whole = s.diagnostics()
    assert abs(sum(d["mass"] for d in got) - whole["mass"]) <= 1e-11 * whole["mass"]
    assert sum(d["n_fluid"] for d in got) == whole["n_fluid"]


def test_set_inlet_velocity_matches_oracle_two_phases(lbfd_lib, oracle_mod):
    cfg, solid, T, Y = inputs.channel(nx=70, ny=14, ignite=(20, 40))
    s = lbfd_lib.Solver(cfg, solid)
    s.init_fields(T, Y)
    s.step_graph(30)
    s.set_inlet_velocity(0.025)
    s.step_graph(30)  # the captured graph must see the new velocity
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y)
    o.step(30)
    To, Yo, go = o.get_state()
    o2 = oracle_mod.Sim(dict(cfg, u_in=0.025), solid)
    o2.set_state(To, Yo, go)
    o2.step(30)
    To, Yo, go = o2.get_state()
    Tg, Yg, gg = s.get_state()
    assert np.linalg.norm(Tg - To) <= 1e-10 * np.linalg.norm(To)
    assert np.linalg.norm(gg - go) <= 1e-10 * np.linalg.norm(go)


def test_inflow_controller_holds_the_flame(lbfd_lib):
    """The flame of a 120x12 adiabatic channel, ignited 20 cells upstream of
    the target position, is brought to the target and held there: after
    14 000 steps the unburnt length is within 0.5 cells of the target and the
    inlet velocity has settled (its last 20 updates within 5e-5), i.e. it
    equals the flame speed (about 0.0125 in lattice units here)."""
    cfg, solid, T, Y = inputs.channel(nx=120, ny=12, walls="adiabatic", u_in=0.01, ignite=(40, 60))
    s = lbfd_lib.Solver(cfg, solid)
    s.init_fields(T, Y)
    x0 = s.diagnostics()["x_f"]
    target = x0 + 20.0
    ctl = channels.InflowController(x_target=target)
    hist = channels.hold_flame(s, ctl, steps=14000, every=50)
    assert abs(hist[-1][1] - target) < 0.5, hist[-1]
    us = [h[2] for h in hist[-20:]]
    assert max(us) - min(us) < 5e-5, us
    assert all(0.0 <= h[2] <= 0.1 for h in hist)


def test_batched_channels_show_a_quenching_width(lbfd_lib):
    """The benchmark's 16 channels (widths 16..196, isothermal 300 K walls,
    mixed precision) after 20 000 steps: the narrow channels quench and the
    wide ones burn, with one transition (a quenching width, Sec. IV.A), and
    among the burning channels the flame speed S_F = u_in - dx_f/dt grows
    with the width (the widest at least twice the narrowest burning one)."""
    cfg, solid, T, Y, seg = inputs.batched_channels()
    s = lbfd_lib.Solver(dict(cfg, precision="mixed"), solid)
    s.init_fields(T, Y)
    tr = channels.FlameSpeedTracker(segments=seg)
    for n in range(0, 20001, 1000):
        if n:
            s.step_graph(1000)
        tr.record(s, n)
    burning = tr.burning()
    widths = [y1 - y0 for y0, y1 in seg]
    first = int(np.argmax(burning))
    assert 3 <= first <= len(widths) - 3, burning  # some quench, some burn
    assert not burning[:first].any() and burning[first:].all(), burning  # one transition
    qw = channels.quenching_width(widths, burning)
    assert qw == widths[first]
    S_F = tr.flame_speed(window=5)
    burn = S_F[first:]
    assert np.all(burn[1:] > 0.0)
    assert burn[-1] >= 2.0 * burn[0]


def test_column_peaks_and_dead_zone_match_the_oracle(lbfd_lib, oracle_mod):
    """The reaction front per column of each channel of a packed batch
    (peak heat release across the channel and its distance to the nearer
    wall): FP64 GPU against the oracle after 60 steps, peaks to 1e-11 of the
    channel's largest, distances exactly; delta_dead equal."""
    widths = [8, 13, 20]
    cfg, solid, T, Y, seg = inputs.batched_channels(widths=widths, length=60, ignite=(15, 30), closed_end=False,
                                                     u_in=0.01)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=31, T_amp=20.0)
    s = lbfd_lib.Solver(cfg, solid)
    s.set_state(T, Y, g)
    s.step(60)
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(60)
    for rows in seg:
        pg, dg = s.column_peaks(rows)
        po, do = o.column_peaks(rows)
        assert np.abs(pg - po).max() <= 1e-11 * po.max()
        assert np.array_equal(dg, do)
        assert channels.dead_zone(pg, dg) == channels.dead_zone(po, do)
    assert len(channels.channel_dead_zones(s, seg)) == 3
