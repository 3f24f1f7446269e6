"""Parity at the benchmark's full sizes, in the launch configuration that
bench.py times: the workloads of bench.py (16 batched channels 1024 long;
the 512x256x256 D3Q27 sphere packing; the 2048x512 cylinder burner), a
pre-run with graph launches, the autotuned kernel variant, then one
`lbfd_step`.

The oracle cannot step these grids whole in a test, so it checks sampled
cells one by one: a cell's update reads only cells within two steps of it
along each axis (FD lines) and its 26 (or 8) lattice neighbours, so the
oracle steps a window of at most 5 cells per axis around the sample, taken
from the GPU's state before the step (read through `lbfd_read_cells`),
with the domain's boundary condition on every side where the window meets
a domain face and a periodic closure elsewhere (never reached from the
window's centre).  The centre of the window is compared with the GPU's
value after the step.  Samples: interior cells, cells next to in-domain
solids, and cells near domain faces, drawn with a fixed seed.

Tolerances for one step from the same inputs: FP64 1e-12 of the field's
scale (rounding order only); mixed FP32 with FP64 Arrhenius above 1000 K:
T within 2e-6 relative, Y_k within 1e-6, populations within 2e-7 absolute.
The stored populations are small (~1e-3) but the collision works on
pre-conditioned values and moments of size rho c_s^2 <= 1/3, so their FP32
error is absolute, about a few units of 2^-24 / 3 ~ 2e-8; 2e-7 is ten of
those.
"""
import numpy as np
import pytest

import bench

pytestmark = pytest.mark.gpu

AXES_BC = ((0, 1), (2, 3), (4, 5))


def classify_cells(cfg, solid):
    """interior / wall / face masks of the fluid cells (the tile kernels'
    criteria: +-2 along every axis and the lattice neighbours)."""
    dim = cfg["dim"]
    sol = solid if dim == 3 else solid[None]
    nz, ny, nx = sol.shape
    periodic = [cfg["bc"][2 * a] == "periodic" for a in range(3)]
    pad = np.full((nz + 4, ny + 4, nx + 4), 2, dtype=np.uint8)
    pad[2:-2, 2:-2, 2:-2] = sol
    for a, axis in ((0, 2), (1, 1), (2, 0)):
        if periodic[a] and (a < dim):
            # wrap the halo of a periodic axis
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            n = sol.shape[axis]
            dst[axis], src[axis] = slice(0, 2), slice(n, n + 2)
            pad[tuple(dst)] = pad[tuple(src)]
            dst[axis], src[axis] = slice(n + 2, n + 4), slice(2, 4)
            pad[tuple(dst)] = pad[tuple(src)]
    if dim == 2:  # no z neighbours in 2-D
        pad[:2], pad[-2:] = pad[2:3], pad[2:3]

    def sh(dx, dy, dz):
        return pad[2 + dz:2 + dz + nz, 2 + dy:2 + dy + ny, 2 + dx:2 + dx + nx]

    offs = []
    for a in range(dim):
        for j in (-2, -1, 1, 2):
            o = [0, 0, 0]
            o[a] = j
            offs.append(tuple(o))
    rng = (-1, 0, 1)
    for dz in (rng if dim == 3 else (0,)):
        for dy in rng:
            for dx in rng:
                if (dx, dy, dz) != (0, 0, 0):
                    offs.append((dx, dy, dz))
    fluid = sol == 0
    interior = fluid.copy()
    face = np.zeros_like(fluid)
    for o in offs:
        v = sh(*o)
        interior &= v == 0
        face |= v == 2
    rest = fluid & ~interior
    return interior.ravel(), (rest & ~face).ravel(), (rest & face).ravel()


def window(cfg, shape, cell):
    """Cell indices of the window around `cell`, the window's shape, its
    centre index and its boundary conditions."""
    dim = cfg["dim"]
    nz, ny, nx = shape
    z, r = divmod(cell, nx * ny)
    y, x = divmod(r, nx)
    coords, ext, cen, bc = [], [], [], list(cfg["bc"])
    for a, (c, n) in enumerate(((x, nx), (y, ny), (z, nz))):
        if a >= dim:
            coords.append([0])
            ext.append(1)
            cen.append(0)
            continue
        lo_f, hi_f = AXES_BC[a]
        if cfg["bc"][lo_f] == "periodic":
            idx = [(c + d) % n for d in range(-2, 3)]
            cen.append(2)
        else:
            lo, hi = max(0, c - 2), min(n - 1, c + 2)
            idx = list(range(lo, hi + 1))
            cen.append(c - lo)
            bc[lo_f] = cfg["bc"][lo_f] if lo == 0 else "periodic"
            bc[hi_f] = cfg["bc"][hi_f] if hi == n - 1 else "periodic"
        coords.append(idx)
        ext.append(len(idx))
    X, Y, Z = np.meshgrid(coords[0], coords[1], coords[2], indexing="ij")
    cells = (X + nx * (Y + ny * Z)).transpose(2, 1, 0).ravel()  # x fastest
    centre = cen[0] + ext[0] * (cen[1] + ext[1] * cen[2])
    return cells, ext, centre, bc


def pick(mask, n, rng):
    idx = np.flatnonzero(mask)
    if idx.size == 0:
        return idx
    return rng.choice(idx, size=min(n, idx.size), replace=False)


def check_workload(lbfd_lib, oracle_mod, name, precision, prerun, n_per_class, seed):
    cfg, solid, T, Y, _ = bench.workload(name, precision)
    dim = cfg["dim"]
    shape = solid.shape if dim == 3 else (1,) + solid.shape
    s = lbfd_lib.Solver(cfg, solid)
    s.init_fields(T, Y)
    if prerun:
        s.step_graph(prerun)
    s.autotune(reps=3)
    interior, wall, face = classify_cells(cfg, solid)
    rng = np.random.Generator(np.random.PCG64(seed))
    samples = np.concatenate([pick(interior, n_per_class, rng), pick(wall, n_per_class, rng),
                              pick(face, n_per_class, rng)])
    wins = [window(cfg, shape, int(c)) for c in samples]
    need = np.unique(np.concatenate([w[0] for w in wins]))
    before = s.read_cells(need)
    pos = {int(c): i for i, c in enumerate(need)}
    s.step(1)
    after = s.read_cells(samples)
    assert s.diagnostics()["n_nonfinite"] == 0
    Q = s.Q
    flat_solid = solid.ravel()
    got, want = [], []
    for (cells, ext, centre, bc), c in zip(wins, samples):
        rows = before[[pos[int(k)] for k in cells]]
        wcfg = dict(cfg, nx=ext[0], ny=ext[1], bc=bc)
        if dim == 3:
            wcfg["nz"] = ext[2]
        wsolid = flat_solid[cells].reshape(ext[2], ext[1], ext[0]) if dim == 3 else \
            flat_solid[cells].reshape(ext[1], ext[0])
        o = oracle_mod.Sim(dict(wcfg, precision="fp64"), wsolid)
        o.set_state(rows[:, Q], rows[:, Q + 1:].T.copy(), rows[:, :Q].T.copy())
        o.step(1)
        To, Yo, go = o.get_state()
        want.append(np.concatenate([go[:, centre], [To[centre]], Yo[:, centre]]))
        got.append(after[len(got)])
    got, want = np.array(got), np.array(want)
    return got, want, Q, samples.size


def assert_close(got, want, Q, precision, label):
    dg = float(np.abs(got[:, :Q] - want[:, :Q]).max())
    gscale = float(np.abs(want[:, :Q]).max())
    dT = float((np.abs(got[:, Q] - want[:, Q]) / np.abs(want[:, Q])).max())
    dY = float(np.abs(got[:, Q + 1:] - want[:, Q + 1:]).max())
    errs = {"g_abs": dg, "g_scale": gscale, "T_rel": dT, "Y_abs": dY}
    if precision == "fp64":
        ok = dg <= 1e-12 * max(gscale, 1e-300) and dT <= 1e-12 and dY <= 1e-12
    else:
        ok = dg <= 2e-7 and dT <= 2e-6 and dY <= 1e-6
    assert ok, (label, errs)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batched_channels_full_size_sampled_cells(lbfd_lib, oracle_mod, precision):
    got, want, Q, n = check_workload(lbfd_lib, oracle_mod, "batched16x1024", precision, prerun=2000,
                                     n_per_class=40, seed=31)
    assert n == 120
    assert_close(got, want, Q, precision, f"batched16x1024 {precision}")


def test_burner_full_size_sampled_cells(lbfd_lib, oracle_mod):
    got, want, Q, n = check_workload(lbfd_lib, oracle_mod, "burner2048x512", "mixed", prerun=200,
                                     n_per_class=30, seed=32)
    assert_close(got, want, Q, "mixed", "burner2048x512")


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_sphere_packing_full_size_sampled_cells(lbfd_lib, oracle_mod, precision):
    got, want, Q, n = check_workload(lbfd_lib, oracle_mod, "porous512x256x256", precision, prerun=20,
                                     n_per_class=30, seed=33)
    assert n == 90
    assert_close(got, want, Q, precision, f"porous512x256x256 {precision}")


def test_channel_256x32_fp64_100_steps(lbfd_lib, oracle_mod):
    """The plain FP64 form on the 256x32 adiabatic channel (ignition band of
    20 columns at 2000 K) against the oracle after 100 steps, every cell:
    relative L2 <= 1e-10 per field."""
    cfg, solid, T, Y, _ = bench.workload("channel256x32", "fp64")
    s = lbfd_lib.Solver(cfg, solid)
    s.init_fields(T, Y)
    s.autotune(reps=3)
    s.step(100)
    Tg, Yg, gg = s.get_state()
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y)
    o.step(100)
    To, Yo, go = o.get_state()
    rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    assert rel(Tg, To) <= 1e-10
    for k in range(Yo.shape[0]):
        if np.linalg.norm(Yo[k]) > 0:
            assert rel(Yg[k], Yo[k]) <= 1e-10, k
    for i in range(go.shape[0]):
        assert rel(gg[i], go[i]) <= 1e-10, i
