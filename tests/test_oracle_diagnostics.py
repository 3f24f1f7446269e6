"""Pins of the oracle's reductions (a11: flame position, mass, heat
release, fuel consumption, maximum temperature, the centre-line argmax of
the heat release, the non-finite count) against values computed here from
the state alone, and against closed forms.

The definitions are the paper's observables (Sec. IV.A flame position from
the unburnt fuel, Sec. IV.C consumption speed from the integrated fuel
consumption, Eq. 40) in this build's single-step model: rho from the ideal-gas
EOS rho = (T_in/T)(W/W_in), q = A dt max(Y_F,0) max(Y_O,0) exp(-Ta/T),
heat release rho (Q/cp) q."""
import numpy as np
import pytest

from paper_2304_05657_gb300 import inputs


def numpy_diagnostics(cfg, solid, T, Y, g):
    """The reductions written with numpy array operations over the fluid
    cells (no loop, no oracle code)."""
    dim = cfg["dim"]
    shape = (cfg["nz"], cfg["ny"], cfg["nx"]) if dim == 3 else (1, cfg["ny"], cfg["nx"])
    fl = solid.reshape(shape) == 0
    T3 = T.reshape(shape)
    Y3 = Y.reshape((5,) + shape)
    g3 = g.reshape((g.shape[0],) + shape)
    finite = np.isfinite(T3) & np.isfinite(Y3).all(axis=0) & np.isfinite(g3).all(axis=0)
    good = fl & finite
    W = np.asarray(cfg["W"])[:, None, None, None]
    Yin = np.asarray(cfg["Y_in"])
    invW = np.where(good, (np.where(good, Y3, 0.0) / W).sum(axis=0), 1.0)
    invW_in = (Yin / np.asarray(cfg["W"])).sum()
    Tg = np.where(good, T3, 1.0)
    rho = (cfg["T_in"] / Tg) * (invW_in / invW)
    yf = np.clip(np.where(good, Y3[cfg["fuel"]], 0.0), 0.0, None)
    yo = np.clip(np.where(good, Y3[cfg["oxidiser"]], 0.0), 0.0, None)
    q = cfg["A"] * cfg["dt"] * yf * yo * np.exp(-cfg["Ta"] / Tg)
    hrr = np.where(good, rho * cfg["Q"] / cfg["cp"] * q, 0.0)
    section = fl[:, :, 0].sum()
    out = {
        "x_f": np.where(good, Y3[cfg["fuel"]], 0.0).sum() / (Yin[cfg["fuel"]] * section),
        "mass": np.where(good, rho, 0.0).sum(),
        "heat_release": hrr.sum(),
        "fuel_consumption": np.where(good, rho * q, 0.0).sum(),
        "T_max": np.where(good, T3, -np.inf).max(),
        "n_nonfinite": float((fl & ~finite).sum()),
        "n_fluid": float(fl.sum()),
    }
    zc, yc = cfg["nz"] // 2 if dim == 3 else 0, cfg["ny"] // 2
    line = np.where(good[zc, yc], hrr[zc, yc], -np.inf)
    out["x_hrr_max"] = float(np.flatnonzero(line == line.max())[0]) if good[zc, yc].any() else -1.0
    return out


def random_state(cfg, solid, seed):
    rng = np.random.default_rng(seed)
    N = solid.size
    Q = 9 if cfg["dim"] == 2 else 27
    T = rng.uniform(300.0, 2300.0, N)
    Y = rng.uniform(0.0, 1.0, (5, N))
    Y /= Y.sum(axis=0)
    Y[0, rng.random(N) < 0.1] *= -0.01  # a few slightly negative fuel fractions (clipped in q only)
    g = rng.uniform(-1e-3, 1e-3, (Q, N))
    return T, Y, g


@pytest.mark.parametrize("dim", [2, 3])
def test_diagnostics_equal_the_definitions(oracle_mod, dim):
    if dim == 2:
        cfg = inputs.base_config(dim=2, nx=37, ny=12)
        rng = np.random.default_rng(3)
        solid = (rng.random((12, 37)) < 0.15).astype(np.uint8)
    else:
        cfg = inputs.base_config(dim=3, nx=15, ny=8, nz=6,
                                 bc=["inlet", "outlet_pressure", "periodic", "periodic", "periodic", "periodic"])
        rng = np.random.default_rng(4)
        solid = (rng.random((6, 8, 15)) < 0.2).astype(np.uint8)
    solid[..., 0] = 0
    solid.reshape(-1)[5] = 1  # a solid cell in the x = 0 section
    T, Y, g = random_state(cfg, solid, 7 + dim)
    # a tie on the centre line: two cells with the same state (the smaller x wins)
    shape = solid.shape
    zc = shape[0] // 2 if dim == 3 else None
    yc = cfg["ny"] // 2
    line = (np.arange(cfg["nx"]) + cfg["nx"] * (yc + cfg["ny"] * (zc or 0)))
    line = line[solid.ravel()[line] == 0]
    a, b = line[3], line[-2]
    Y[0, line] *= 0.01  # the rest of the line burns slowly
    Y[:, line] /= Y[:, line].sum(axis=0)
    T[a] = T[b] = 2200.0
    Y[:, a] = Y[:, b] = [0.3, 0.3, 0.05, 0.05, 0.3]
    # two fluid cells with non-finite values (counted, left out of every sum)
    fluid = np.flatnonzero(solid.ravel() == 0)
    T[fluid[7]] = np.nan
    g[2, fluid[9]] = np.inf
    sim = oracle_mod.Sim(cfg, solid)
    sim.set_state(T, Y, g)
    got = sim.diagnostics()
    ref = numpy_diagnostics(cfg, solid, T, Y, g)
    for key in ("x_f", "mass", "heat_release", "fuel_consumption", "T_max"):
        assert abs(got[key] - ref[key]) <= 1e-13 * abs(ref[key]), (key, got[key], ref[key])
    assert got["n_nonfinite"] == ref["n_nonfinite"] == 2.0
    assert got["n_fluid"] == ref["n_fluid"] == float((solid == 0).sum())
    assert got["x_hrr_max"] == ref["x_hrr_max"] == float(a % cfg["nx"])


def test_diagnostics_closed_forms(oracle_mod):
    """A uniform inlet-state gas has rho = 1 in every fluid cell (the EOS
    reference), so the mass is the fluid cell count; unburnt gas upstream of
    column x_b and burnt gas (no fuel) beyond gives x_f = x_b exactly; the
    heat release is Q/cp times the fuel consumption; a cold mixture has no
    centre-line maximum other than its first fluid cell."""
    nx, ny = 50, 9
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny)
    solid = np.zeros((ny, nx), np.uint8)
    solid[4, 10:20] = 1  # a solid block: the section at x = 0 stays fully fluid
    N = nx * ny
    T = np.full(N, cfg["T_in"])
    Y = np.tile(np.asarray(cfg["Y_in"])[:, None], (1, N))
    sim = oracle_mod.Sim(cfg, solid)
    sim.set_state(T, Y)
    d = sim.diagnostics()
    nfl = float((solid == 0).sum())
    assert d["mass"] == pytest.approx(nfl, rel=1e-14)
    assert d["n_fluid"] == nfl and d["n_nonfinite"] == 0
    # fluid cells per column: the x_f normalisation uses the x = 0 section (ny cells)
    assert d["x_f"] == pytest.approx(nfl / ny, rel=1e-14)
    # burnt beyond x_b (no fuel), unburnt before, no solid: x_f = x_b
    x_b = 31
    solid0 = np.zeros((ny, nx), np.uint8)
    Yb = inputs.burnt_Y(cfg["Y_in"])
    xs = np.tile(np.arange(nx), ny)
    Y2 = np.where(xs[None, :] < x_b, np.asarray(cfg["Y_in"])[:, None], np.asarray(Yb)[:, None])
    T2 = np.where(xs < x_b, 1500.0, 2000.0)
    sim2 = oracle_mod.Sim(cfg, solid0)
    sim2.set_state(T2, Y2)
    d2 = sim2.diagnostics()
    assert d2["x_f"] == pytest.approx(x_b, rel=1e-14)
    assert d2["heat_release"] == pytest.approx(cfg["Q"] / cfg["cp"] * d2["fuel_consumption"], rel=1e-13)
    assert d2["T_max"] == 2000.0
    # every hot unburnt cell on the centre line has the same rate: ties go to x = 0
    assert d2["x_hrr_max"] == 0.0


def test_column_peaks_closed_form(oracle_mod):
    """A front drawn by hand: in column x the only reacting cell is at row
    r(x) of a band y0 <= y < y1, so the peak is that cell's heat release and
    the distance is min(r - y0 + 1/2, y1 - 1/2 - r); a column with two equal
    peaks reports the smaller row."""
    nx, ny = 12, 15
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny)
    solid = np.zeros((ny, nx), np.uint8)
    solid[9, :] = 1  # a separator: the band is rows 10..14
    y0, y1 = 10, 15
    T = np.full((ny, nx), 300.0)
    rows = [10, 11, 12, 13, 14, 12, 11, 10, 13, 14, 12, 11]
    for x, r in enumerate(rows):
        T[r, x] = 1500.0 + 10.0 * x
    T[12, 4] = T[11, 4] = 1600.0  # a tie in column 4: rows 11 and 12 (distances 1.5 and 2.5)
    T[14, 4] = 300.0
    Y = np.tile(np.asarray(cfg["Y_in"])[:, None], (1, nx * ny))
    sim = oracle_mod.Sim(cfg, solid)
    sim.set_state(T.ravel(), Y)
    peak, dist = sim.column_peaks((y0, y1))
    for x, r in enumerate(rows):
        if x == 4:
            r = 11
        assert dist[x] == min(r - y0 + 0.5, y1 - 0.5 - r), (x, dist[x])
    assert np.all(peak > 0) and np.argmax(peak) == nx - 1
