"""Pins of the curved-wall treatment (Sec. III): interpolated bounce-back
with the wall distance q of each cut link (Eq. 29-30) and image-point
ghost values by Shepard inverse-distance weighting (Eq. 34-38), against
exact solutions whose walls lie between grid points; the staircase
treatment of the same mask misses them by the wall offset."""
import numpy as np
import pytest

from paper_2304_05657_gb300 import inputs

CS2 = 1.0 / 3.0


def plates(nx, ny, a, b, **over):
    """Fluid between half-space walls y < a and y > b (cell centres y + 1/2)."""
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny, A=0.0, **over)
    yc = np.arange(ny) + 0.5
    solid = np.zeros((ny, nx), np.uint8)
    solid[(yc < a) | (yc > b), :] = 1
    prims = [(1, 0.0, -1.0, 0.0, -a), (1, 0.0, 1.0, 0.0, b)]
    return cfg, solid, prims


def poiseuille_profile(oracle_mod, curved, a=1.3, b=12.6, nx=72, ny=14, steps=5000):
    cfg, solid, prims = plates(nx, ny, a, b, u_in=0.01,
                               bc=["inlet", "outlet_pressure", "periodic", "periodic", "periodic", "periodic"])
    T = np.full(nx * ny, 300.0)
    Y = np.tile(np.array(cfg["Y_in"])[:, None], (1, nx * ny))
    sim = oracle_mod.Sim(cfg, solid)
    if curved:
        sim.set_geometry(prims)
    sim.set_state(T, Y)
    sim.step(steps)
    _, _, g = sim.get_state()
    gm = g.reshape(9, ny, nx)
    cx = np.array([i % 3 - 1 for i in range(9)], dtype=np.float64)
    ux = np.tensordot(cx, gm, axes=1)[:, nx // 2] / CS2  # rho = 1
    fluid = solid[:, nx // 2] == 0
    y = np.arange(ny)[fluid] + 0.5
    u = ux[fluid]
    flux = u.sum()
    H = b - a
    exact = 6.0 * (flux / H) * (y - a) * (b - y) / H ** 2  # same flux, true walls
    return np.abs(u - exact).max() / exact.max()


def test_interpolated_bounce_back_sees_the_true_walls(oracle_mod):
    err_curved = poiseuille_profile(oracle_mod, True)
    err_stair = poiseuille_profile(oracle_mod, False)
    assert err_curved < 0.01, err_curved
    assert err_stair > 3 * err_curved, (err_stair, err_curved)


def conduction(oracle_mod, curved, a=2.3, ny=20, steps=10000):
    """Isothermal wall (T_solid = 300 K) along y = a, isothermal domain face
    at y = ny (600 K), no flow: steady (1/rho) d/dy(rho alpha dT/dy) = 0 with
    rho ~ 1/T, i.e. ln T linear between the true wall positions."""
    nx = 4
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny, A=0.0, u_in=0.0, T_solid=300.0, solid_isothermal=True,
                             bc=["periodic", "periodic", "wall_isothermal", "wall_isothermal", "periodic", "periodic"],
                             T_wall=[300.0, 300.0, 300.0, 600.0, 300.0, 300.0])
    yc = np.arange(ny) + 0.5
    solid = np.zeros((ny, nx), np.uint8)
    solid[yc < a, :] = 1
    sim = oracle_mod.Sim(cfg, solid)
    if curved:
        sim.set_geometry([(1, 0.0, -1.0, 0.0, -a)])
        assert sim.num_ghosts > 0
    T0 = np.full(nx * ny, 300.0)
    Y = np.tile(np.array(cfg["Y_in"])[:, None], (1, nx * ny))
    sim.set_state(T0, Y)
    sim.step(steps)
    T, _, _ = sim.get_state()
    Tc = T.reshape(ny, nx)[:, 0]
    fluid = yc > a
    lnT = np.log(300.0) + (np.log(600.0) - np.log(300.0)) * (yc - a) / (ny - a)
    return np.abs(np.log(Tc[fluid]) - lnT[fluid]).max() / np.log(2.0)


def test_image_point_ghosts_put_the_wall_temperature_on_the_true_wall(oracle_mod):
    """Two solid rows, so that both ghost layers of the FD stencils get image
    points.  Shepard's reconstruction is first order and its bias depends on
    where the image point falls, so the wall is placed at three offsets."""
    cur, st = [], []
    for a in (2.1, 2.3, 2.45):
        cur.append(conduction(oracle_mod, True, a=a, ny=20, steps=10000))
        st.append(conduction(oracle_mod, False, a=a, ny=20, steps=10000))
    assert max(cur) < 1.1e-2, cur
    assert np.mean(cur) < 0.5 * np.mean(st), (cur, st)
    assert all(c < s for c, s in zip(cur, st)), (cur, st)


def test_uniform_state_is_kept_by_curved_walls(oracle_mod):
    """A circle inside a periodic box at rest and uniform temperature equal
    to the solid's: nothing may move (Shepard weights sum to one, Eq. 37)."""
    nx = ny = 24
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny, A=0.0, u_in=0.0, bc=["periodic"] * 6, T_solid=300.0)
    yy, xx = np.mgrid[0:ny, 0:nx] + 0.5
    solid = (((xx - 11.7) ** 2 + (yy - 12.2) ** 2) < 5.3 ** 2).astype(np.uint8)
    sim = oracle_mod.Sim(cfg, solid)
    sim.set_geometry([(0, 11.7, 12.2, 0.0, 5.3)])
    T = np.full(nx * ny, 300.0)
    Y = np.tile(np.array(cfg["Y_in"])[:, None], (1, nx * ny))
    sim.set_state(T, Y)
    sim.step(30)
    T2, Y2, g2 = sim.get_state()
    assert np.abs(T2 - 300.0).max() < 1e-10 and np.abs(g2).max() < 1e-14
