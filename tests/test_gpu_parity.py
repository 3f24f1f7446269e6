"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 per field, i.e. per scalar field and per population
plane, over all cells):
  - FP64 kernels: 1e-10 after the stated number of steps; the two codes
    differ only in rounding order (axis-wise moment transforms on the GPU vs
    a dense linear solve in the oracle, a rearranged WENO weight formula).
  - mixed FP32 kernels: 1e-5 on T and Y after 1000 steps of the 256x32
    channel; the populations are compared in absolute terms against their
    own scale (their mean is ~0, so a relative norm is meaningless).
"""
import numpy as np
import pytest

from paper_2304_05657_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    den = np.linalg.norm(b)
    if den == 0.0:
        return float(np.linalg.norm(a - b))
    return float(np.linalg.norm(a - b) / den)


def compare_states(gpu_state, orc_state, tol, label):
    Tg, Yg, gg = gpu_state
    To, Yo, go = orc_state
    errs = {"T": rel_l2(Tg, To)}
    for k in range(Yo.shape[0]):
        errs[f"Y{k}"] = rel_l2(Yg[k], Yo[k])
    for i in range(go.shape[0]):
        errs[f"g{i}"] = rel_l2(gg[i], go[i])
    bad = {k: v for k, v in errs.items() if not (v <= tol)}
    assert not bad, f"{label}: fields above {tol:g}: {bad}"
    return errs


def run_pair(lbfd, oracle, cfg, solid, T, Y, g, steps):
    s = lbfd.Solver(cfg, solid)
    s.set_state(T, Y, g)
    s.step(steps)
    gpu = s.get_state()
    o = oracle.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(steps)
    return s, o, gpu, o.get_state()


# ---------------------------------------------------------------------------
# cases: several tiles and a ragged tail, every boundary type
# ---------------------------------------------------------------------------

def case_channel_adiabatic():
    cfg, solid, T, Y = inputs.channel(nx=83, ny=21, ignite=(0, 20))
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=1)
    return cfg, solid, T, Y, g


def case_channel_isothermal_poiseuille():
    cfg, solid, T, Y = inputs.channel(nx=70, ny=19, walls="isothermal", T_wall=350.0, ignite=(30, 50),
                                      poiseuille_inlet=True, u_in=0.02)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=2)
    return cfg, solid, T, Y, g


def case_periodic_obstacles(nx=67, ny=29, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny, bc=["periodic"] * 6, u_in=0.0)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    for _ in range(6):  # blocks of 1..4 cells, incl. one-cell-thin walls
        x, y = rng.integers(0, nx), rng.integers(0, ny)
        solid[y:y + rng.integers(1, 5), x:x + rng.integers(1, 5)] = 1
    solid[10, 5:40] = 1  # a thin wall with fluid on both sides
    T, Y = inputs.ignition_fields(cfg, solid, 20, 35)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=seed + 1)
    return cfg, solid, T, Y, g


def case_periodic_obstacles_even():
    """Even nx: the packed-pair kernels stage and store two cells at a
    time, and their halo wraps across both periodic faces."""
    return case_periodic_obstacles(nx=66, ny=28, seed=13)


def case_obstacles_adiabatic_solid():
    cfg, solid, T, Y = inputs.channel(nx=61, ny=23, ignite=(35, 50), solid_isothermal=False)
    yy, xx = np.mgrid[0:23, 0:61]
    solid = (((xx + 0.5 - 20) ** 2 + (yy + 0.5 - 11.5) ** 2) <= 36).astype(np.uint8)
    T, Y = inputs.ignition_fields(cfg, solid, 35, 50)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=5)
    return cfg, solid, T, Y, g


def case_batched():
    cfg, solid, T, Y, seg = inputs.batched_channels(widths=[5, 8, 13], length=45, ignite=(10, 25))
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=6)
    return cfg, solid, T, Y, g


def case_d3q27():
    cfg, solid, T, Y = inputs.sphere_packing(nx=19, ny=10, nz=9, x_range=(3, 13), r_range=(2.0, 3.5),
                                             porosity=0.8, seed=7, ignite_width=4)
    cfg["bc"][2] = cfg["bc"][3] = "wall_isothermal"
    cfg["T_wall"] = [320.0] * 6
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=8)
    return cfg, solid, T, Y, g


CASES_2D = {
    "channel_adiabatic": case_channel_adiabatic,
    "channel_isothermal_poiseuille": case_channel_isothermal_poiseuille,
    "periodic_obstacles": case_periodic_obstacles,
    "periodic_obstacles_even": case_periodic_obstacles_even,
    "obstacles_adiabatic_solid": case_obstacles_adiabatic_solid,
    "batched": case_batched,
}


@pytest.mark.parametrize("name", sorted(CASES_2D))
def test_fp64_parity_2d(lbfd_lib, oracle_mod, name):
    cfg, solid, T, Y, g = CASES_2D[name]()
    _, _, gpu, orc = run_pair(lbfd_lib, oracle_mod, cfg, solid, T, Y, g, steps=100)
    compare_states(gpu, orc, 1e-10, name)


def test_fp64_parity_d3q27(lbfd_lib, oracle_mod):
    """D3Q27 (general kernel): walls, solid spheres, inlet and pressure outlet."""
    cfg, solid, T, Y, g = case_d3q27()
    _, _, gpu, orc = run_pair(lbfd_lib, oracle_mod, cfg, solid, T, Y, g, steps=20)
    compare_states(gpu, orc, 1e-10, "d3q27")


def test_fp64_parity_one_step_exact_inputs(lbfd_lib, oracle_mod):
    """After one step every cell must agree to ~1e-13 relative (no growth)."""
    cfg, solid, T, Y, g = case_periodic_obstacles()
    _, _, gpu, orc = run_pair(lbfd_lib, oracle_mod, cfg, solid, T, Y, g, steps=1)
    compare_states(gpu, orc, 1e-12, "one step")


def test_fp64_diagnostics_match(lbfd_lib, oracle_mod):
    cfg, solid, T, Y, g = case_channel_adiabatic()
    s, o, _, _ = run_pair(lbfd_lib, oracle_mod, cfg, solid, T, Y, g, steps=30)
    dg, do = s.diagnostics(), o.diagnostics()
    for key in ("x_f", "mass", "heat_release", "fuel_consumption", "T_max"):
        assert abs(dg[key] - do[key]) <= 1e-11 * max(1.0, abs(do[key])), (key, dg[key], do[key])
    for key in ("x_hrr_max", "n_nonfinite", "n_fluid"):
        assert dg[key] == do[key], (key, dg[key], do[key])


def test_fp64_empty_and_degenerate(lbfd_lib, oracle_mod):
    """A domain that is all solid does nothing; a one-cell-wide periodic
    column and a one-row channel match the oracle."""
    cfg = inputs.base_config(dim=2, nx=9, ny=4, bc=["periodic"] * 6)
    solid = np.ones((4, 9), dtype=np.uint8)
    T, Y = inputs.ignition_fields(cfg, solid, 0, 3)
    s = lbfd_lib.Solver(cfg, solid)
    s.set_state(T, Y)
    s.step(5)
    Tg, Yg, gg = s.get_state()
    assert np.array_equal(Tg, T) and np.array_equal(Yg, Y) and not gg.any()
    assert s.diagnostics()["n_fluid"] == 0
    for (nx, ny, bc) in [(1, 7, ["periodic"] * 6),
                         (33, 1, ["inlet", "outlet", "periodic", "periodic", "periodic", "periodic"])]:
        cfg = inputs.base_config(dim=2, nx=nx, ny=ny, bc=bc)
        solid = np.zeros((ny, nx), dtype=np.uint8)
        T, Y = inputs.ignition_fields(cfg, solid, 0, min(nx, 10))
        g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=9)
        _, _, gpu, orc = run_pair(lbfd_lib, oracle_mod, cfg, solid, T, Y, g, steps=20)
        compare_states(gpu, orc, 1e-10, f"{nx}x{ny}")


def test_mixed_precision_channel_1000_steps(lbfd_lib, oracle_mod):
    """FP32 storage/arithmetic (FP64 Arrhenius above 1000 K) vs the FP64
    oracle on the 256x32 adiabatic channel after 1000 steps."""
    cfg, solid, T, Y = inputs.channel(nx=256, ny=32)
    T, Y = inputs.ignition_fields(cfg, solid, 0, 20, burnt=False)
    cfg_m = dict(cfg, precision="mixed")
    s = lbfd_lib.Solver(cfg_m, solid)
    s.set_state(T, Y)
    s.step(1000)
    Tg, Yg, gg = s.get_state()
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y)
    o.step(1000)
    To, Yo, go = o.get_state()
    assert rel_l2(Tg, To) <= 1e-5
    for k in range(5):
        if np.linalg.norm(Yo[k]) > 0:
            assert rel_l2(Yg[k], Yo[k]) <= 1e-5, k
    scale = np.abs(go).max()
    assert np.abs(gg - go).max() <= 1e-4 * scale


def mixed_vs_oracle_after(lbfd_lib, oracle_mod, cfg, solid, T, Y, steps, variant=None):
    import os

    s = lbfd_lib.Solver(dict(cfg, precision="mixed"), solid)
    if variant is not None:
        s.variant = variant
    s.set_state(T, Y)
    s.step_graph(steps)
    Tg, Yg, gg = s.get_state()
    s.close()
    oracle_mod.set_threads(os.cpu_count() or 1)
    try:
        o = oracle_mod.Sim(cfg, solid)
        o.set_state(T, Y)
        o.step(steps)
        To, Yo, go = o.get_state()
    finally:
        oracle_mod.set_threads(1)
    fl = solid.ravel() == 0
    errs = {"T": rel_l2(Tg[fl], To[fl])}
    for k in range(5):
        if np.linalg.norm(Yo[k][fl]) > 0:
            errs[f"Y{k}"] = rel_l2(Yg[k][fl], Yo[k][fl])
    errs["g"] = np.abs(gg[:, fl] - go[:, fl]).max() / np.abs(go[:, fl]).max()
    return errs


def test_mixed_precision_packing_crop_1000_steps(lbfd_lib, oracle_mod):
    """The precision bar (fields within 1e-5 relative L2 of the FP64 oracle
    after 1000 steps) on the 3-D workload's recipe at a size the oracle
    runs in seconds: a 64x24x24 sphere packing (r in [3, 6]) with its band
    of burning gas behind it, the autotuner's 3-D variant (2)."""
    cfg, solid, T, Y = inputs.sphere_packing(nx=64, ny=24, nz=24, x_range=(6, 34), r_range=(3.0, 6.0))
    assert 0.05 < solid.mean() < 0.2 and (T > 1000.0).any()
    errs = mixed_vs_oracle_after(lbfd_lib, oracle_mod, cfg, solid, T, Y, 1000, variant=2)
    assert all(v <= 1e-5 for k, v in errs.items() if k != "g"), errs
    assert errs["g"] <= 1e-4, errs


def test_mixed_precision_batched_channels_1000_steps(lbfd_lib, oracle_mod):
    """The same bar on packed channels (isothermal walls and separators,
    closed ignition end), the packed-pair variant 11."""
    cfg, solid, T, Y, seg = inputs.batched_channels(widths=[16, 40, 64], length=128)
    errs = mixed_vs_oracle_after(lbfd_lib, oracle_mod, cfg, solid, T, Y, 1000, variant=11)
    assert all(v <= 1e-5 for k, v in errs.items() if k != "g"), errs
    assert errs["g"] <= 1e-4, errs


# ---------------------------------------------------------------------------
# kernel variants, graph launches, autotuner
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["channel_adiabatic", "periodic_obstacles", "batched"])
def test_every_kernel_variant_matches_oracle(lbfd_lib, oracle_mod, name):
    cfg, solid, T, Y, g = CASES_2D[name]()
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(60)
    orc = o.get_state()
    s = lbfd_lib.Solver(cfg, solid)
    for v in range(s.num_variants):
        s.variant = v
        s.set_state(T, Y, g)
        s.step(60)
        compare_states(s.get_state(), orc, 1e-10, f"{name} variant {v}")


def test_mixed_variants_agree_with_each_other(lbfd_lib):
    """FP32 variants differ only in rounding order."""
    cfg, solid, T, Y, g = case_channel_adiabatic()
    cfg = dict(cfg, precision="mixed")
    s = lbfd_lib.Solver(cfg, solid)
    ref = None
    for v in range(s.num_variants):
        s.variant = v
        s.set_state(T, Y, g)
        s.step(50)
        st = s.get_state()
        if ref is None:
            ref = st
        else:
            compare_states(st, ref, 1e-5, f"mixed variant {v}")


@pytest.mark.parametrize("name", sorted(CASES_2D))
def test_mixed_variants_match_oracle(lbfd_lib, oracle_mod, name):
    """Every FP32 variant (one cell per thread, and two cells per thread in
    packed FP32 arithmetic) against the FP64 oracle after 60 steps, with the
    mixed-precision bar of the 1000-step channel test: T and Y within 1e-5
    relative L2, populations within 1e-4 of their own scale.  The cases
    have odd nx (a pair tile whose second cell is missing), periodic wrap,
    in-domain solids, walls, inlet and outlet."""
    cfg, solid, T, Y, g = CASES_2D[name]()
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(60)
    To, Yo, go = o.get_state()
    s = lbfd_lib.Solver(dict(cfg, precision="mixed"), solid)
    scale = np.abs(go).max()
    for v in range(s.num_variants):
        s.variant = v
        s.set_state(T, Y, g)
        s.step(60)
        Tg, Yg, gg = s.get_state()
        assert rel_l2(Tg, To) <= 1e-5, (name, v, rel_l2(Tg, To))
        for k in range(5):
            if np.linalg.norm(Yo[k]) > 0:
                assert rel_l2(Yg[k], Yo[k]) <= 1e-5, (name, v, k, rel_l2(Yg[k], Yo[k]))
        assert np.abs(gg - go).max() <= 1e-4 * scale, (name, v, np.abs(gg - go).max() / scale)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "tangent", "tangent_mixed"])
def test_read_cells_equals_read_field(lbfd_lib, precision):
    """lbfd_read_cells returns, per listed cell, g_0..g_{Q-1}, T, Y_k as
    lbfd_read_field does; invalid indices are rejected without a copy."""
    cfg, solid, T, Y, g = case_batched()
    s = lbfd_lib.Solver(dict(cfg, precision=precision), solid)
    s.set_state(T, Y, g)
    s.step(3)
    Tg, Yg, gg = s.get_state()
    rng = np.random.Generator(np.random.PCG64(5))
    cells = rng.integers(0, solid.size, size=57)
    rows = s.read_cells(cells)
    assert rows.shape == (57, s.Q + 6)
    assert np.array_equal(rows[:, :s.Q], gg[:, cells].T)
    assert np.array_equal(rows[:, s.Q], Tg[cells])
    assert np.array_equal(rows[:, s.Q + 1:], Yg[:, cells].T)
    assert s.read_cells([]).shape == (0, s.Q + 6)
    with pytest.raises(lbfd_lib.LbfdError):
        s.read_cells([0, solid.size])


def test_graph_launch_equals_single_launches(lbfd_lib):
    cfg, solid, T, Y, g = case_batched()
    a = lbfd_lib.Solver(cfg, solid)
    a.set_state(T, Y, g)
    a.step(7)
    b = lbfd_lib.Solver(cfg, solid)
    b.set_state(T, Y, g)
    b.step_graph(3)
    b.step_graph(4)  # re-capture for a new n and the other parity
    b.step_graph(4)
    a.step(4)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert b.steps_done == 11


def test_autotune_keeps_state_and_picks_a_variant(lbfd_lib):
    cfg, solid, T, Y, g = case_periodic_obstacles()
    s = lbfd_lib.Solver(cfg, solid)
    s.set_state(T, Y, g)
    before = s.get_state()
    best, ms = s.autotune(reps=3)
    assert 0 <= best < s.num_variants and s.variant == best
    assert np.all(ms > 0)
    for x, y in zip(before, s.get_state()):
        assert np.array_equal(x, y)


def test_d3q27_tile_variants_match_oracle(lbfd_lib, oracle_mod):
    """A 3-D domain large enough for interior cells: every D3Q27 variant
    (general form, 2.5-D tiles with the boundary list) against the oracle."""
    cfg, solid, T, Y = inputs.sphere_packing(nx=40, ny=14, nz=13, x_range=(8, 30), r_range=(2.0, 3.5),
                                             porosity=0.85, seed=12, ignite_width=5)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=13)
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(8)
    orc = o.get_state()
    s = lbfd_lib.Solver(cfg, solid)
    assert s.num_variants == 8
    for v in range(s.num_variants):
        s.variant = v
        s.set_state(T, Y, g)
        s.step(8)
        compare_states(s.get_state(), orc, 1e-10, f"d3q27 variant {v}")
    for v in range(s.num_variants):  # mixed precision, same cases
        sm = lbfd_lib.Solver(dict(cfg, precision="mixed"), solid)
        sm.variant = v
        sm.set_state(T, Y, g)
        sm.step(8)
        Tg = sm.read_field(lbfd_lib.FIELD_T)
        assert rel_l2(Tg, orc[0]) <= 1e-6


def test_d3q27_split_variants_equal_fused(lbfd_lib):
    """The split 3-D variants (FD tile kernel, then a collision kernel fed
    Lambda and grad rho through a scratch buffer) do the fused variants'
    arithmetic in the same order; only the compiler's choice of fused
    multiply-adds may differ between the two programs, so the FP64 states
    agree to a few ulp: 1e-12 relative L2.  In FP32 with omega_hi = 1 the
    fused kernels form only the central moments of orders 0-2 while the
    collision kernel of the split ones forms all of them (the results are
    the same up to rounding): 1e-5, the FP32 population bar of the other
    tests (measured 5e-6)."""
    cfg, solid, T, Y = inputs.sphere_packing(nx=40, ny=14, nz=13, x_range=(8, 30), r_range=(2.0, 3.5),
                                             porosity=0.85, seed=12, ignite_width=5)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=13)
    for prec in ("fp64", "mixed"):
        s = lbfd_lib.Solver(dict(cfg, precision=prec), solid)
        for fused, split in ((1, 4), (2, 5)):
            st = []
            for v in (fused, split):
                s.variant = v
                s.set_state(T, Y, g)
                s.step(6)
                st.append(s.get_state())
            tol = 1e-12 if prec == "fp64" else 1e-5
            compare_states(st[1], st[0], tol, f"{prec} split {split} vs fused {fused}")


@pytest.mark.parametrize("iso", [True, False])
def test_d3q27_wall_aware_tiles_equal_the_wall_list(lbfd_lib, oracle_mod, iso):
    """Variants 6, 7 update the cells next to the spheres in the tile kernel
    (mirror-rule ghosts from the staged mask, bounce-back pulls) instead of
    the general form over the wall list (variants 1, 2): the same arithmetic
    up to rounding order, 1e-12 relative L2 in FP64 (1e-5 in FP32, as for
    the other FP32 variants: the populations are small deviations, measured
    5e-6), and the oracle to 1e-10; isothermal and adiabatic solids.  One
    launch fewer per step."""
    cfg, solid, T, Y = inputs.sphere_packing(nx=44, ny=16, nz=14, x_range=(8, 34), r_range=(2.0, 4.0),
                                             porosity=0.75, seed=17, ignite_width=5)
    cfg["solid_isothermal"] = iso
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=18)
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(7)
    orc = o.get_state()
    for prec in ("fp64", "mixed"):
        s = lbfd_lib.Solver(dict(cfg, precision=prec), solid)
        for lst, walls in ((1, 6), (2, 7)):
            st = []
            for v in (lst, walls):
                s.variant = v
                s.set_state(T, Y, g)
                s.step(7)
                st.append(s.get_state())
            assert s.launches_per_step == 2
            tol = 1e-12 if prec == "fp64" else 1e-5
            compare_states(st[1], st[0], tol, f"{prec} walls {walls} vs list {lst}")
            if prec == "fp64":
                compare_states(st[1], orc, 1e-10, f"walls variant {walls} vs oracle")
        s.close()


@pytest.mark.parametrize("outlet", ["outlet_pressure", "outlet"])
def test_d3q27_face_codes_match_oracle(lbfd_lib, oracle_mod, outlet):
    """The cells near the inlet and outlet faces take the coded form (the
    velocity inlet of Eq. 31, the constant-pressure outlet or the convective
    outlet of Eq. 32 applied per population, inlet Dirichlet and outlet
    zero-gradient ghosts on the x lines) instead of the general form, in
    every 3-D tile variant: FP64 against the oracle to 1e-10, mixed T to
    1e-6.  Solid cells next to both faces leave some cells to the general
    form (an Eq. 32 inner cell that is solid) and give others bounce-back
    bits beside the face rules.  Solid cells in the face planes at the
    periodic y/z seams make the boundary column of a face-crossing population
    a wrapped cell (the general form bounces such a population back)."""
    cfg, solid, T, Y = inputs.sphere_packing(nx=36, ny=12, nz=11, x_range=(8, 28), r_range=(2.0, 3.0),
                                             porosity=0.85, seed=21, ignite_width=4)
    cfg["bc"][1] = outlet
    solid[4, 5, 1] = solid[6, 3, 34] = solid[7, 8, 33] = True
    solid[0, 11, 0] = solid[10, 0, 35] = solid[5, 11, 0] = True
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=22)
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(8)
    orc = o.get_state()
    s = lbfd_lib.Solver(cfg, solid)
    for v in range(1, s.num_variants):
        s.variant = v
        s.set_state(T, Y, g)
        s.step(8)
        compare_states(s.get_state(), orc, 1e-10, f"{outlet} variant {v}")
    sm = lbfd_lib.Solver(dict(cfg, precision="mixed"), solid)
    for v in (2, 6):
        sm.variant = v
        sm.set_state(T, Y, g)
        sm.step(8)
        assert rel_l2(sm.read_field(lbfd_lib.FIELD_T), orc[0]) <= 1e-6


@pytest.mark.parametrize("omega_hi", [1.0, 1.3])
def test_d3q27_mixed_higher_order_rate(lbfd_lib, oracle_mod, omega_hi):
    """The FP32 3-D tile and coded kernels with omega_hi = 1 form only the
    central moments of orders 0-2 (the relaxation sets every higher cumulant
    to its equilibrium); with any other rate they form all of them.  Both
    against the oracle after 10 steps: T and Y to 1e-6, each population
    plane to 1e-5 (relative L2, as for the other FP32 variants)."""
    cfg, solid, T, Y = inputs.sphere_packing(nx=40, ny=14, nz=13, x_range=(8, 30), r_range=(2.0, 3.5),
                                             porosity=0.85, seed=12, ignite_width=5)
    cfg["omega_hi"] = omega_hi
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=14)
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(10)
    To, Yo, go = o.get_state()
    s = lbfd_lib.Solver(dict(cfg, precision="mixed"), solid)
    for v in (1, 2):
        s.variant = v
        s.set_state(T, Y, g)
        s.step(10)
        Tg, Yg, gg = s.get_state()
        assert rel_l2(Tg, To) <= 1e-6, v
        for k in range(Yo.shape[0]):
            if np.linalg.norm(Yo[k]) > 0:
                assert rel_l2(Yg[k], Yo[k]) <= 1e-6, (v, k)
        for i in range(go.shape[0]):
            assert rel_l2(gg[i], go[i]) <= 1e-5, (v, i)


def test_d3q27_packing_cut_by_the_faces(lbfd_lib, oracle_mod):
    """Spheres that reach the inlet and outlet planes (the packing fills the
    whole length, periodic in y and z), as in the crops of the large packing
    that the benchmark compares with the oracle: every 3-D variant in FP64
    against the oracle to 1e-10, and the FP32 tile variants 1, 2 with every
    population plane to 1e-5 and T to 1e-6 (relative L2)."""
    cfg, _, T, Y = inputs.sphere_packing(nx=30, ny=14, nz=13, x_range=(0, 30), r_range=(2.0, 4.0),
                                         porosity=0.8, seed=31, ignite_width=4)
    # the middle of a longer packing: spheres cut by both planes
    solid = inputs.sphere_packing(nx=60, ny=14, nz=13, x_range=(0, 60), r_range=(2.0, 4.0), porosity=0.8,
                                  seed=34)[1][:, :, 15:45].copy()
    assert solid[:, :, 0].sum() > 20 and solid[:, :, -1].sum() > 10
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=32)
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(8)
    orc = o.get_state()
    s = lbfd_lib.Solver(cfg, solid)
    for v in range(s.num_variants):
        s.variant = v
        s.set_state(T, Y, g)
        s.step(8)
        compare_states(s.get_state(), orc, 1e-10, f"faces cut, variant {v}")
    sm = lbfd_lib.Solver(dict(cfg, precision="mixed"), solid)
    for v in (1, 2):
        sm.variant = v
        sm.set_state(T, Y, g)
        sm.step(8)
        Tg, Yg, gg = sm.get_state()
        assert rel_l2(Tg, orc[0]) <= 1e-6, v
        for i in range(gg.shape[0]):
            assert rel_l2(gg[i], orc[2][i]) <= 1e-5, (v, i)
