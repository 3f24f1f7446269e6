"""Pins of the whole oracle step against physics and exact analysis:
  - the FD diffusion terms of T and Y_k (Eq. 1, 2, 7) and Lambda (Eq. 6)
    against the exact operators of smooth fields (sympy), converging at 4th
    order;
  - convection (Eq. 26) converging to u.grad(phi), with the correction
    summing to zero over species;
  - rest state, homogeneous reactor (scalar explicit Euler recurrence),
    exact conservation of sum(g) and momentum in closed/periodic boxes,
    sum_k Y_k = 1, mirror symmetry, Poiseuille flow (analytic parabola and
    pressure gradient), adiabatic flame temperature of a 1-D flame."""
import numpy as np
import pytest
import sympy as sp

from paper_2304_05657_gb300 import inputs

CS2 = 1.0 / 3.0
LE = [0.97, 1.11, 1.39, 0.83, 1.0]


def exact_fd_terms(cfg, kx, ky):
    """Exact (1/rho) div(rho alpha grad T), -(1/rho) div(rho Y_k V_k) with the
    mixture-averaged flux of Eq. 2, and Lambda (Eq. 6, no reaction) for
    smooth periodic fields."""
    x, y = sp.symbols("x y", real=True)
    Wk = [sp.nsimplify(w) for w in cfg["W"]]
    T = 1200 + 500 * sp.sin(kx * x + 0.3) * sp.cos(ky * y + 0.1)
    Yb = [0.04, 0.18, 0.05, 0.04]
    amp = [0.02, 0.05, 0.03, 0.02]
    Ys = [Yb[k] + amp[k] * sp.sin(kx * x + k) * sp.cos(ky * y + 2 * k) for k in range(4)]
    Ys.append(1 - sum(Ys))
    invW = sum(Ys[k] / Wk[k] for k in range(5))
    invW_in = sum(cfg["Y_in"][k] / cfg["W"][k] for k in range(5))
    rho = (cfg["T_in"] / T) * (invW_in / invW)
    alpha = cfg["nu"] / cfg["Pr"]
    D = [alpha / cfg["Le"][k] for k in range(5)]
    X = [Ys[k] / (Wk[k] * invW) for k in range(5)]
    grad = lambda f: (sp.diff(f, x), sp.diff(f, y))
    div = lambda v: sp.diff(v[0], x) + sp.diff(v[1], y)
    gT = grad(T)
    diff_T = div((rho * alpha * gT[0], rho * alpha * gT[1])) / rho
    gX = [grad(X[k]) for k in range(5)]
    Vc = [sum(D[k] * Wk[k] * invW * gX[k][a] for k in range(5)) for a in range(2)]
    diff_Y = []
    for k in range(5):
        flux = [-D[k] * Wk[k] * invW * gX[k][a] + Ys[k] * Vc[a] for a in range(2)]  # Y_k V_k
        diff_Y.append(-div((rho * flux[0], rho * flux[1])) / rho)
    lam = diff_T / T + sum(diff_Y[k] / (Wk[k] * invW) for k in range(5))
    fT = sp.lambdify((x, y), T, "numpy")
    fY = [sp.lambdify((x, y), Ys[k], "numpy") for k in range(5)]
    fdT = sp.lambdify((x, y), diff_T, "numpy")
    fdY = [sp.lambdify((x, y), diff_Y[k], "numpy") for k in range(5)]
    flam = sp.lambdify((x, y), lam, "numpy")
    return fT, fY, fdT, fdY, flam


@pytest.fixture(scope="module")
def analytic_cases():
    cfg = inputs.base_config(dim=2, nx=64, ny=48, bc=["periodic"] * 6, A=0.0, Le=LE)
    out = {}
    for m in (1, 2):
        kx = 2 * np.pi * (2 / m) / cfg["nx"]
        ky = 2 * np.pi * (1 / m) / cfg["ny"] * (2 if m == 1 else 1)
        out[m] = exact_fd_terms(cfg, kx, ky) + (kx, ky)
    return cfg, out


def diffusion_errors(oracle_mod, cfg, fns, samples):
    fT, fY, fdT, fdY, flam, kx, ky = fns
    nx, ny = cfg["nx"], cfg["ny"]
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    # one period must fit: the fields are periodic on the grid only for m=1
    T = fT(xx, yy).ravel()
    Y = np.stack([np.broadcast_to(fY[k](xx, yy), xx.shape).ravel() for k in range(5)])
    sim = oracle_mod.Sim(cfg, np.zeros(nx * ny, np.uint8))
    sim.set_state(T, Y)
    eT, eY, eL = [], [], []
    for (x, y) in samples:
        t = sim.cell_terms(x, y)
        sT = abs(fdT(x, y))
        eT.append(abs(t["diff_T"] - fdT(x, y)))
        eY.append(max(abs(t["diff_Y"][k] - fdY[k](x, y)) for k in range(5)))
        eL.append(abs(t["Lambda"] - flam(x, y)))
        assert abs(t["diff_Y"].sum()) < 1e-15  # the correction velocity closes the sum
        assert t["conv_T"] == 0.0 and np.all(t["conv_Y"] == 0.0)  # g = 0: u = 0
    return max(eT), max(eY), max(eL), sT


def test_diffusion_and_lambda_converge_at_fourth_order(oracle_mod):
    """Halving the wave numbers must cut the discrete-operator error ~16x."""
    errs = []
    for m in (1, 2):
        nx, ny = 64 * m, 48 * m
        cfg = inputs.base_config(dim=2, nx=nx, ny=ny, bc=["periodic"] * 6, A=0.0, Le=LE)
        kx, ky = 2 * np.pi * 2 / nx, 2 * np.pi * 2 / ny
        fns = exact_fd_terms(cfg, kx, ky) + (kx, ky)
        samples = [(int(nx * a), int(ny * b)) for a, b in [(0.1, 0.2), (0.37, 0.6), (0.8, 0.9), (0.55, 0.15)]]
        errs.append(diffusion_errors(oracle_mod, cfg, fns, samples))
    (eT1, eY1, eL1, _), (eT2, eY2, eL2, _) = errs
    for a, b, name in [(eT1, eT2, "T"), (eY1, eY2, "Y"), (eL1, eL2, "Lambda")]:
        assert a / b > 12.0, (name, a, b, a / b)
    # and the errors are small in absolute terms on the coarse grid
    assert eY1 < 1e-6 and eL1 < 1e-5


def test_convection_converges_and_correction_sums_to_zero(oracle_mod):
    """Populations g_i = w_i rho c_i.u0 carry the velocity u0 (Eq. 13b);
    the convective terms approach u0.grad(phi) at 3rd order (WENO3 on smooth
    data) and the species correction makes sum_k conv_Y = 0."""
    u0 = np.array([0.013, -0.007, 0.0])
    c = np.array([[cx, cy, 0] for cy in (-1, 0, 1) for cx in (-1, 0, 1)], dtype=np.float64)
    w = np.array([(1 / 6 if a else 2 / 3) * (1 / 6 if b else 2 / 3) for a, b, _ in c])
    errs = []
    for m in (1, 2):
        nx, ny = 64 * m, 48 * m
        cfg = inputs.base_config(dim=2, nx=nx, ny=ny, bc=["periodic"] * 6, A=0.0)
        yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
        kx, ky = 2 * np.pi * 2 / nx, 2 * np.pi * 2 / ny
        T = (1000 + 400 * np.sin(kx * xx) * np.cos(ky * yy)).ravel()
        dTx = (400 * kx * np.cos(kx * xx) * np.cos(ky * yy)).ravel()
        dTy = (-400 * ky * np.sin(kx * xx) * np.sin(ky * yy)).ravel()
        Y = np.empty((5, nx * ny))
        Y[0] = (0.03 + 0.01 * np.cos(kx * xx + 1) * np.sin(ky * yy)).ravel()
        Y[1] = 0.2
        Y[2] = (0.05 + 0.02 * np.sin(kx * xx) * np.sin(ky * yy + 0.5)).ravel()
        Y[3] = 0.04
        Y[4] = 1 - Y[:4].sum(axis=0)
        invW = (Y / np.array(cfg["W"])[:, None]).sum(axis=0)
        invW_in = sum(cfg["Y_in"][k] / cfg["W"][k] for k in range(5))
        rho = (cfg["T_in"] / T) * (invW_in / invW)
        g = w[:, None] * rho[None, :] * (c @ u0)[:, None]
        sim = oracle_mod.Sim(cfg, np.zeros(nx * ny, np.uint8))
        sim.set_state(T, Y, g)
        # the pulled populations are the neighbours' values: evaluate where
        # they equal g at the cell to rounding (u from the pulled values)
        err = 0.0
        for (a, b) in [(0.13, 0.31), (0.52, 0.77), (0.9, 0.5)]:
            x, y = int(nx * a), int(ny * b)
            t = sim.cell_terms(x, y)
            i = x + nx * y
            exact = t["u"][0] * dTx[i] + t["u"][1] * dTy[i]
            err = max(err, abs(t["conv_T"] - exact) / (400 * kx * np.abs(u0).max()))
            assert abs(t["conv_Y"].sum()) < 1e-17
        errs.append(err)
    assert errs[0] / errs[1] > 4.0, errs  # at least 2nd order (3rd away from extrema)
    assert errs[0] < 0.15  # 16 points per wavelength on the coarse grid


def periodic_box(oracle_mod, nx=20, ny=12, seed=0, A=0.0, walls=False, T_uniform=True):
    bc = ["wall_adiabatic"] * 4 + ["periodic"] * 2 if walls else ["periodic"] * 6
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny, bc=bc, A=A)
    solid = np.zeros((ny, nx), np.uint8)
    T = np.full(nx * ny, 900.0)
    Y = np.tile(np.array(cfg["Y_in"])[:, None], (1, nx * ny))
    rng = np.random.default_rng(seed)
    g = rng.uniform(-1e-3, 1e-3, size=(9, nx * ny))
    sim = oracle_mod.Sim(cfg, solid)
    return cfg, sim, T, Y, g


def test_rest_state_stays_at_rest(oracle_mod):
    cfg, sim, T, Y, g = periodic_box(oracle_mod)
    sim.set_state(T, Y, None)
    sim.step(50)
    T2, Y2, g2 = sim.get_state()
    assert np.array_equal(T2, T) and np.array_equal(Y2, Y)
    assert np.abs(g2).max() < 1e-15


@pytest.mark.parametrize("walls", [False, True])
def test_inert_isothermal_box_conserves_mass_exactly(oracle_mod, walls):
    """Uniform T and Y without reaction: Xi = 0, so collision and streaming
    (periodic wrap or bounce-back) conserve sum_cells sum_i g_i; a periodic
    box also conserves momentum."""
    cfg, sim, T, Y, g = periodic_box(oracle_mod, walls=walls)
    sim.set_state(T, Y, g)
    c = np.array([[cx, cy] for cy in (-1, 0, 1) for cx in (-1, 0, 1)], dtype=np.float64)
    m0, p0 = g.sum(), (c.T @ g).sum(axis=1)
    sim.step(60)
    _, _, g2 = sim.get_state()
    assert abs(g2.sum() - m0) < 1e-14
    if not walls:
        assert np.abs((c.T @ g2).sum(axis=1) - p0).max() < 1e-14
    else:  # the walls take momentum: it must have changed
        assert np.abs((c.T @ g2).sum(axis=1) - p0).max() > 1e-6


def test_homogeneous_reactor_follows_scalar_euler(oracle_mod):
    """A uniform reacting mixture in a periodic box: no gradients, so each
    cell obeys the explicit Euler recurrence of the single-step ODE,
    velocities stay zero and the pressure sum grows by rho cs^2 Lambda per
    cell and step."""
    nx, ny = 6, 5
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny, bc=["periodic"] * 6)
    sim = oracle_mod.Sim(cfg, np.zeros(nx * ny, np.uint8))
    T0 = 1500.0
    Y0 = np.array(cfg["Y_in"])
    sim.set_state(np.full(nx * ny, T0), np.tile(Y0[:, None], (1, nx * ny)))
    A_lat = cfg["A"] * cfg["dt"]
    W = np.array(cfg["W"])
    nu = np.array(cfg["nu_stoich"])
    yields = nu * W / (-nu[0] * W[0])
    T, Y = T0, Y0.copy()
    invW_in = (Y0 / W).sum()
    for n in range(40):
        psum0 = sim.get_state()[2].sum()
        q = A_lat * max(Y[0], 0) * max(Y[1], 0) * np.exp(-cfg["Ta"] / T)
        dT = cfg["Q"] / cfg["cp"] * q
        dY = yields * q
        invW = (Y / W).sum()
        rho = (cfg["T_in"] / T) * (invW_in / invW)
        lam = dT / T + (dY / W).sum() / invW
        sim.step(1)
        T, Y = T + dT, Y + dY
        T2, Y2, g2 = sim.get_state()
        assert np.allclose(T2, T, rtol=1e-13, atol=0)
        assert np.allclose(Y2, Y[:, None], rtol=1e-12, atol=1e-17)
        assert abs(g2.sum() - psum0 - nx * ny * rho * CS2 * lam) < 1e-12 * max(1.0, abs(g2.sum()))
    c = np.array([[cx, cy] for cy in (-1, 0, 1) for cx in (-1, 0, 1)], dtype=np.float64)
    assert np.abs(c.T @ g2).max() < 1e-13
    assert T > 1600.0  # the mixture did react


def channel_flame(oracle_mod, steps, nx=60, ny=16, walls="isothermal", burnt=True):
    cfg, solid, T, Y = inputs.channel(nx=nx, ny=ny, walls=walls, ignite=(10, 25))
    T, Y = inputs.ignition_fields(cfg, solid, 10, 25, burnt=burnt)
    sim = oracle_mod.Sim(cfg, solid)
    sim.set_state(T, Y)
    sim.step(steps)
    return cfg, sim


def test_mass_fractions_sum_to_one(oracle_mod):
    """The species correction of Eq. 26 and the correction velocity of Eq. 2
    keep sum_k Y_k = 1 to rounding in a strongly reacting flow."""
    cfg, sim = channel_flame(oracle_mod, 150, walls="adiabatic", burnt=False)
    T, Y, g = sim.get_state()
    assert np.abs(Y.sum(axis=0) - 1.0).max() < 1e-13
    assert T.max() > 2500.0  # the hot unburnt band has ignited


def test_mirror_symmetry_in_y(oracle_mod):
    """A channel with symmetric walls and a y-symmetric initial state keeps
    every field mirror-symmetric (populations map c_y -> -c_y)."""
    cfg, sim = channel_flame(oracle_mod, 120, ny=15)
    nx, ny = cfg["nx"], cfg["ny"]
    T, Y, g = sim.get_state()
    Tm = T.reshape(ny, nx)
    assert np.abs(Tm - Tm[::-1]).max() < 1e-9 * Tm.max()
    gm = g.reshape(9, ny, nx)
    for i in range(9):
        cx, cy = i % 3 - 1, i // 3 - 1
        j = (cx + 1) + 3 * (-cy + 1)
        assert np.abs(gm[i] - gm[j][::-1]).max() < 1e-12


def test_poiseuille_channel(oracle_mod):
    """Inert isothermal channel, parabolic inlet of mean ubar, convective
    outlet: the developed profile is u(y) = 6 ubar s (H - s)/H^2 with
    s = y + 1/2 (half-way walls) and dP_h/dx = -12 nu ubar / H^2."""
    nx, ny, ubar = 72, 12, 0.01
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny, A=0.0, poiseuille_inlet=True, u_in=ubar,
                             bc=["inlet", "outlet_pressure", "wall_adiabatic", "wall_adiabatic", "periodic", "periodic"])
    solid = np.zeros((ny, nx), np.uint8)
    T = np.full(nx * ny, 300.0)
    Y = np.tile(np.array(cfg["Y_in"])[:, None], (1, nx * ny))
    sim = oracle_mod.Sim(cfg, solid)
    sim.set_state(T, Y)
    sim.step(4000)
    _, _, g = sim.get_state()
    gm = g.reshape(9, ny, nx)
    cx = np.array([i % 3 - 1 for i in range(9)], dtype=np.float64)
    ux = np.tensordot(cx, gm, axes=1) / CS2  # rho = 1
    s = np.arange(ny) + 0.5
    exact = 6 * ubar * s * (ny - s) / ny ** 2
    prof = ux[:, nx // 2]
    assert np.abs(prof - exact).max() < 0.02 * exact.max()
    P = gm.sum(axis=0).mean(axis=0)
    slope = np.polyfit(np.arange(20, 50), P[20:50], 1)[0]
    assert abs(slope / (-12 * cfg["nu"] * ubar / ny ** 2) - 1.0) < 0.05


def test_adiabatic_flame_temperature(oracle_mod):
    """1-D planar flame, unit Lewis numbers, equal cp, adiabatic walls: the
    Shvab-Zeldovich variable T + (Q/cp) Y_F obeys a source-free linear
    equation, so started uniform (burnt gas at T_ad next to fresh gas) it
    stays uniform while the flame burns through, and the burnt gas behind
    the front approaches T_b = T_in + Q Y_F,in / cp."""
    nx = 240
    cfg = inputs.base_config(dim=2, nx=nx, ny=1, u_in=0.0,
                             bc=["wall_adiabatic", "outlet", "periodic", "periodic", "periodic", "periodic"])
    T_ad = cfg["T_in"] + cfg["Q"] * cfg["Y_in"][0] / cfg["cp"]
    solid = np.zeros((1, nx), np.uint8)
    T, Y = inputs.ignition_fields(cfg, solid, 0, 40, T_hot=T_ad, burnt=True)
    sim = oracle_mod.Sim(cfg, solid)
    sim.set_state(T, Y)
    sim.step(6000)
    T2, Y2, _ = sim.get_state()
    front = int(np.argmax(T2 < 0.5 * (T_ad + cfg["T_in"])))
    assert front > 60  # the flame has travelled into the fresh gas
    h = T2 + cfg["Q"] / cfg["cp"] * Y2[0]
    # uniform to the level the nonlinear WENO weights allow (T and Y_F get
    # slightly different weights); the flame itself moves T by ~2000 K
    assert np.abs(h / T_ad - 1.0).max() < 2e-4, (h.min(), h.max(), T_ad)
    burnt = T2[45:front - 40]
    assert burnt.size > 5
    assert np.abs(burnt / T_ad - 1.0).max() < 5e-3, (burnt.min(), burnt.max(), T_ad)


def test_packed_channels_are_independent_problems(oracle_mod):
    """Channels stacked along y with one isothermal solid row between them
    evolve exactly as the same channels run alone with isothermal walls:
    no stencil or population crosses a solid row."""
    widths = [4, 7, 10]
    cfg, solid, T, Y, seg = inputs.batched_channels(widths=widths, length=30, ignite=(5, 15), closed_end=False,
                                                     u_in=0.01)
    nx = cfg["nx"]
    o = oracle_mod.Sim(cfg, solid)
    rng = np.random.default_rng(5)
    g = rng.uniform(-1e-3, 1e-3, size=(9, solid.size))
    g[:, solid.ravel() == 1] = 0.0
    o.set_state(T, Y, g)
    o.step(25)
    Tb, Yb, gb = o.get_state()
    for (y0, y1), w in zip(seg, widths):
        c1, s1, _, _ = inputs.channel(nx=nx, ny=w, walls="isothermal", T_wall=cfg["T_wall"][2])
        sl = slice(y0 * nx, y1 * nx)
        o1 = oracle_mod.Sim(c1, s1)
        o1.set_state(T[sl], Y[:, sl], g[:, sl])
        o1.step(25)
        T1, Y1, g1 = o1.get_state()
        assert np.array_equal(T1, Tb[sl]) and np.array_equal(Y1, Yb[:, sl]) and np.array_equal(g1, gb[:, sl])
