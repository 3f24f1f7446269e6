"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds configuration data, geometry masks and initial fields
only; it contains none of the method's arithmetic.  Every random draw is
seeded (numpy PCG64).  The workloads are synthetic stand-ins for the
paper's cases (Sec. IV): the channel flames of Sec. IV.A, the staggered
cylinder burner of Sec. IV.B and the random sphere packing of Sec. IV.C,
with a single-step mechanism in place of the Cantera/BFER-2 chemistry.
"""
from __future__ import annotations

import numpy as np

# Species order: CH4, O2, CO2, H2O, N2.  Molar masses in g/mol.
SPECIES = ("CH4", "O2", "CO2", "H2O", "N2")
W = (16.04, 32.00, 44.01, 18.015, 28.014)
NU_STOICH = (-1.0, -2.0, 1.0, 2.0, 0.0)  # CH4 + 2 O2 -> CO2 + 2 H2O
FUEL, OXIDISER = 0, 1


def premixed_Y(phi: float = 1.0) -> list[float]:
    """Mass fractions of a methane/air mixture at equivalence ratio phi
    (air = O2 + 3.76 N2)."""
    moles = np.array([phi, 2.0, 0.0, 0.0, 2.0 * 3.76])
    mass = moles * np.array(W)
    return (mass / mass.sum()).tolist()


def base_config(**over) -> dict:
    """Defaults: single-step CH4/air (A = 1e9 1/s, Ta = 15000 K), nu = 0.05,
    Pr = 0.7, unit Lewis numbers, dx = 20 um (the channel resolution of
    Sec. IV.A) and a lattice step dt = 7.5e-7 s, so that A*dt = 750 per step:
    with these constant lattice transport coefficients the 1-D flame then has
    a thermal thickness of about 13 cells (the paper resolves 328 um with
    20 um cells, about 16), whereas dt = 7.5e-8 s (A*dt = 75) does not
    sustain a flame at all."""
    cfg = dict(
        dim=2, nx=64, ny=16, nz=1,
        bc=["inlet", "outlet_pressure", "wall_adiabatic", "wall_adiabatic", "periodic", "periodic"],
        T_wall=[300.0] * 6,
        W=list(W), nu_stoich=list(NU_STOICH), Le=[1.0] * 5,
        fuel=FUEL, oxidiser=OXIDISER,
        A=1.0e9, Ta=15000.0, Q=5.0e7, cp=1400.0, dt=7.5e-7, dx=20e-6,
        nu=0.05, Pr=0.7, omega_bulk=0.0, omega_hi=1.0,
        u_in=0.01, T_in=300.0, Y_in=premixed_Y(1.0),
        T_solid=300.0, solid_isothermal=True, poiseuille_inlet=False,
        weno_eps=1e-6, T_fp64=1000.0, precision="fp64",
    )
    cfg.update(over)
    if cfg["dim"] == 2:
        cfg["nz"] = 1
    return cfg


def ncells(cfg: dict) -> int:
    return cfg["nx"] * cfg["ny"] * (cfg["nz"] if cfg["dim"] == 3 else 1)


def burnt_Y(Y_unburnt) -> list[float]:
    """Composition after complete combustion of the fuel (or of the
    oxidiser, whichever runs out first) by CH4 + 2 O2 -> CO2 + 2 H2O,
    from a mole balance."""
    n = np.array(Y_unburnt) / np.array(W)          # moles per unit mass
    ext = min(n[FUEL] / -NU_STOICH[FUEL], n[OXIDISER] / -NU_STOICH[OXIDISER])
    n = n + ext * np.array(NU_STOICH)
    n[FUEL] = max(n[FUEL], 0.0)
    n[OXIDISER] = max(n[OXIDISER], 0.0)
    m = n * np.array(W)
    return (m / m.sum()).tolist()


def _isothermal_distance(cfg: dict, solid: np.ndarray, reach: int) -> np.ndarray:
    """Distance (cells, centre to wall plane) from each cell to the nearest
    isothermal boundary: an isothermal solid cell (when solids are
    isothermal) or an isothermal domain face; capped at `reach`."""
    from scipy import ndimage

    dim = cfg["dim"]
    shape = solid.shape  # (ny, nx) or (nz, ny, nx)
    wall = solid.astype(bool) if cfg["solid_isothermal"] else np.zeros(shape, dtype=bool)
    pads, modes = [], []
    for ax in range(dim):
        a = dim - 1 - ax  # array axis of grid axis `ax`
        lo, hi = cfg["bc"][2 * ax], cfg["bc"][2 * ax + 1]
        pads.append((a, lo, hi))
    m = reach + 1
    arr = wall
    for a, lo, hi in pads:
        if lo == "periodic":
            width = [(0, 0)] * arr.ndim
            width[a] = (m, m)
            arr = np.pad(arr, width, mode="wrap")
        else:
            sh = list(arr.shape)
            sh[a] = m
            blo = np.full(sh, lo == "wall_isothermal")
            bhi = np.full(sh, hi == "wall_isothermal")
            arr = np.concatenate([blo, arr, bhi], axis=a)
    if not arr.any():
        return np.full(shape, float(reach))
    d = ndimage.distance_transform_edt(~arr)
    sl = tuple(slice(m, m + n) for n in shape)
    return np.minimum(d[sl] - 0.5, float(reach))


def ignition_fields(cfg: dict, solid: np.ndarray, x0: int = 0, x1: int = 20, T_hot: float = 2000.0,
                    burnt: bool = True, edge: float = 1.5, wall_taper: float = 4.0):
    """Unburnt mixture at T_in with a hot band x in [x0, x1) at T_hot; the
    band holds burnt products (burnt=True) or the unburnt mixture.  The
    band has tanh edges of width `edge` cells along x (no edge where it
    starts at the inlet) and fades linearly to the cold state within
    `wall_taper` cells of isothermal walls and solids, so that the initial
    state is smooth on the grid (the paper starts from smooth flame
    profiles)."""
    N = ncells(cfg)
    shape = (cfg["nz"], cfg["ny"], cfg["nx"]) if cfg["dim"] == 3 else (cfg["ny"], cfg["nx"])
    xc = np.arange(cfg["nx"]) + 0.5
    left = np.ones_like(xc) if x0 <= 0 else 0.5 * (1.0 + np.tanh((xc - x0) / edge))
    right = 0.5 * (1.0 - np.tanh((xc - x1) / edge))
    prof = np.broadcast_to(left * right, shape)
    if wall_taper > 0:
        d = _isothermal_distance(cfg, solid, int(np.ceil(wall_taper)))
        prof = prof * np.clip(d / wall_taper, 0.0, 1.0)
    prof = prof.ravel()
    T = cfg["T_in"] + (T_hot - cfg["T_in"]) * prof
    Yb = burnt_Y(cfg["Y_in"]) if burnt else cfg["Y_in"]
    Y = np.empty((5, N), dtype=np.float64)
    for k in range(5):
        Y[k] = cfg["Y_in"][k] + (Yb[k] - cfg["Y_in"][k]) * prof
    s = solid.ravel().astype(bool)
    T[s] = cfg["T_solid"]
    return T, Y


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def channel(nx=256, ny=32, walls="adiabatic", T_wall=300.0, u_in=0.01, ignite=(0, 20), **over):
    """2-D channel: inlet at -x, outlet at +x, walls at +-y; hot band in
    columns ignite[0]..ignite[1]-1 (256x32 adiabatic = the plain FP64 case)."""
    wt = "wall_adiabatic" if walls == "adiabatic" else "wall_isothermal"
    cfg = base_config(dim=2, nx=nx, ny=ny, bc=["inlet", "outlet_pressure", wt, wt, "periodic", "periodic"],
                      T_wall=[T_wall] * 6, u_in=u_in, **over)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    T, Y = ignition_fields(cfg, solid, *ignite)
    return cfg, solid, T, Y


def batched_channels(widths=None, length=1024, T_wall=300.0, u_in=0.0, ignite=(0, 20), closed_end=True, **over):
    """Channels of uneven width stacked along y in one 2-D domain, separated
    by one solid row (isothermal at T_wall) so that no stencil couples them;
    domain faces at +-y are isothermal walls.  Default: 16 channels of widths
    16, 28, ..., 196 and length 1024, closed at the ignition end (-x) by an
    adiabatic wall and open at +x (constant pressure): a flame started in
    the hot band propagates toward the open end in the wide channels and
    quenches in the narrow ones.  closed_end=False puts a velocity inlet at
    -x instead.  Returns (cfg, solid, T, Y, segments) with segments =
    [(y0, y1), ...] the fluid rows of each channel."""
    if widths is None:
        widths = [16 + 12 * j for j in range(16)]
    ny = sum(widths) + len(widths) - 1
    left = "wall_adiabatic" if closed_end else "inlet"
    cfg = base_config(dim=2, nx=length, ny=ny,
                      bc=[left, "outlet_pressure", "wall_isothermal", "wall_isothermal", "periodic", "periodic"],
                      T_wall=[T_wall] * 6, T_solid=T_wall, solid_isothermal=True, u_in=u_in, **over)
    solid = np.zeros((ny, length), dtype=np.uint8)
    segments = []
    y = 0
    for j, w in enumerate(widths):
        segments.append((y, y + w))
        y += w
        if j < len(widths) - 1:
            solid[y, :] = 1
            y += 1
    T, Y = ignition_fields(cfg, solid, *ignite)
    return cfg, solid, T, Y, segments


def cylinder_burner(nx=2048, ny=512, d=40, pitch=64, x_range=(512, 1536), T_wall=373.0, phi=0.8,
                    u_in=0.02, ignite_width=20, **over):
    """Pseudo-2-D burner: staggered cylinders (diameter d, pitch `pitch`,
    alternate rows offset by pitch/2) filling x_range, isothermal at T_wall,
    periodic in y, premixed inlet at equivalence ratio phi; a hot band of
    ignite_width columns just downstream of the array."""
    cfg = base_config(dim=2, nx=nx, ny=ny, bc=["inlet", "outlet_pressure", "periodic", "periodic", "periodic", "periodic"],
                      T_solid=T_wall, solid_isothermal=True, u_in=u_in, Y_in=premixed_Y(phi), **over)
    yy, xx = np.mgrid[0:ny, 0:nx]
    solid = np.zeros((ny, nx), dtype=bool)
    r = d / 2.0
    col = 0
    for xc in np.arange(x_range[0] + pitch / 2.0, x_range[1], pitch):
        off = (pitch / 2.0) * (col % 2)
        for yc in np.arange(off, ny + pitch, pitch):
            solid |= (xx + 0.5 - xc) ** 2 + (yy + 0.5 - yc) ** 2 <= r * r
        col += 1
    solid = solid.astype(np.uint8)
    T, Y = ignition_fields(cfg, solid, x_range[1], x_range[1] + ignite_width)
    return cfg, solid, T, Y


def sphere_packing(nx=512, ny=256, nz=256, x_range=(64, 448), r_range=(8.0, 16.0), porosity=0.80,
                   seed=20230411, T_wall=300.0, u_in=0.01, ignite_width=20, T_hot=None, **over):
    """3-D random porous medium: overlapping spheres with radius uniform in
    r_range placed (numpy PCG64, given seed) inside x_range until the
    porosity of that slab drops to `porosity`; periodic in y and z,
    isothermal solid; inlet at -x; a hot band of burnt gas right after the
    packing, by default at the adiabatic flame temperature of the inlet
    mixture (T_in + Q Y_F,in / c_p): burnt gas at 2000 K there loses its
    heat to the cold packing and the flame dies out within about 1000 steps
    (measured on the 512x256x256 packing), at T_ad it burns on and enters
    the packing."""
    cfg = base_config(dim=3, nx=nx, ny=ny, nz=nz,
                      bc=["inlet", "outlet_pressure", "periodic", "periodic", "periodic", "periodic"],
                      T_solid=T_wall, solid_isothermal=True, u_in=u_in, **over)
    rng = np.random.Generator(np.random.PCG64(seed))
    solid = np.zeros((nz, ny, nx), dtype=bool)
    x0, x1 = x_range
    slab = (x1 - x0) * ny * nz
    filled = 0
    while 1.0 - filled / slab > porosity:
        r = rng.uniform(*r_range)
        c = np.array([rng.uniform(x0 + r, x1 - r), rng.uniform(0, ny), rng.uniform(0, nz)])
        ri = int(np.ceil(r))
        xs = np.arange(int(c[0]) - ri, int(c[0]) + ri + 2)
        ys = np.arange(int(c[1]) - ri, int(c[1]) + ri + 2)
        zs = np.arange(int(c[2]) - ri, int(c[2]) + ri + 2)
        xs = xs[(xs >= x0) & (xs < x1)]
        Z, Yg, X = np.meshgrid(zs, ys, xs, indexing="ij")
        dz = np.minimum(np.abs(Z + 0.5 - c[2]), nz - np.abs(Z + 0.5 - c[2]))
        dy = np.minimum(np.abs(Yg + 0.5 - c[1]), ny - np.abs(Yg + 0.5 - c[1]))
        inside = (X + 0.5 - c[0]) ** 2 + dy ** 2 + dz ** 2 <= r * r
        zi, yi, xi = Z[inside] % nz, Yg[inside] % ny, X[inside]
        before = solid[zi, yi, xi].sum()
        solid[zi, yi, xi] = True
        filled += inside.sum() - before
    solid = solid.astype(np.uint8)
    if T_hot is None:
        T_hot = cfg["T_in"] + cfg["Q"] * cfg["Y_in"][FUEL] / cfg["cp"]
    T, Y = ignition_fields(cfg, solid, x1, x1 + ignite_width, T_hot=T_hot)
    return cfg, solid, T, Y


def perturbed_state(cfg: dict, solid: np.ndarray, T: np.ndarray, Y: np.ndarray, seed: int,
                    g_amp: float = 1e-3, T_amp: float = 50.0, Y_amp: float = 0.01):
    """A seeded, non-trivial state for parity tests: random populations of
    size g_amp, and T and Y perturbed by uniform noise (Y renormalised to
    sum 1, kept positive).  Solid cells keep T and Y unperturbed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = ncells(cfg)
    Q = 9 if cfg["dim"] == 2 else 27
    g = rng.uniform(-g_amp, g_amp, size=(Q, N))
    s = solid.ravel().astype(bool)
    T2 = T.copy()
    T2[~s] += rng.uniform(-T_amp, T_amp, size=(~s).sum())
    Y2 = Y.copy()
    Y2[:, ~s] += rng.uniform(0.0, Y_amp, size=(5, (~s).sum()))
    Y2 /= Y2.sum(axis=0, keepdims=True)
    g[:, s] = 0.0
    return g, T2, Y2
