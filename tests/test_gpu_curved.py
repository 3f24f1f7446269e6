"""Curved walls on the GPU (interpolated bounce-back, image-point ghosts)
against the oracle with the same primitives."""
import numpy as np
import pytest

from paper_2304_05657_gb300 import inputs

from test_gpu_parity import compare_states

pytestmark = pytest.mark.gpu


def cylinders_case():
    nx, ny = 70, 33
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny, u_in=0.02, T_solid=380.0, solid_isothermal=True,
                             bc=["inlet", "outlet_pressure", "periodic", "periodic", "periodic", "periodic"])
    prims = [(0, 20.3, 9.7, 0.0, 5.4), (0, 36.8, 24.1, 0.0, 6.2), (1, 0.0, -1.0, 0.0, -1.35)]
    yy, xx = np.mgrid[0:ny, 0:nx] + 0.5
    solid = ((xx - 20.3) ** 2 + (yy - 9.7) ** 2 < 5.4 ** 2) | ((xx - 36.8) ** 2 + (yy - 24.1) ** 2 < 6.2 ** 2)
    solid |= yy < 1.35
    solid = solid.astype(np.uint8)
    T, Y = inputs.ignition_fields(cfg, solid, 45, 60)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=31)
    return cfg, solid, prims, T, Y, g


@pytest.mark.parametrize("variant", [0, 1, 5])
def test_curved_walls_fp64_match_oracle(lbfd_lib, oracle_mod, variant):
    cfg, solid, prims, T, Y, g = cylinders_case()
    o = oracle_mod.Sim(cfg, solid)
    o.set_geometry(prims)
    o.set_state(T, Y, g)
    o.step(60)
    s = lbfd_lib.Solver(cfg, solid)
    s.variant = variant
    s.set_curved_walls(prims)
    s.set_state(T, Y, g)
    s.step(60)
    compare_states(s.get_state(), o.get_state(), 1e-10, f"curved variant {variant}")
    assert s.launches_per_step == (3 if variant else 2)


def test_curved_walls_sphere_d3q27_and_mixed(lbfd_lib, oracle_mod):
    nx, ny, nz = 22, 12, 12
    cfg = inputs.base_config(dim=3, nx=nx, ny=ny, nz=nz, u_in=0.02, T_solid=350.0, solid_isothermal=True,
                             bc=["inlet", "outlet_pressure", "periodic", "periodic", "periodic", "periodic"])
    prims = [(0, 10.6, 6.3, 5.8, 3.7)]
    zz, yy, xx = np.mgrid[0:nz, 0:ny, 0:nx] + 0.5
    solid = ((xx - 10.6) ** 2 + (yy - 6.3) ** 2 + (zz - 5.8) ** 2 < 3.7 ** 2).astype(np.uint8)
    T, Y = inputs.ignition_fields(cfg, solid, 14, 19)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=32)
    o = oracle_mod.Sim(cfg, solid)
    o.set_geometry(prims)
    o.set_state(T, Y, g)
    o.step(10)
    orc = o.get_state()
    for v in (0, 1, 6):  # variant 6 leaves the curved-wall cells to the wall list
        s = lbfd_lib.Solver(cfg, solid)
        s.variant = v
        s.set_curved_walls(prims)
        s.set_state(T, Y, g)
        s.step(10)
        compare_states(s.get_state(), orc, 1e-10, f"curved d3q27 variant {v}")
    sm = lbfd_lib.Solver(dict(cfg, precision="mixed"), solid)
    sm.set_curved_walls(prims)
    sm.set_state(T, Y, g)
    sm.step(10)
    Tm = sm.read_field(lbfd_lib.FIELD_T)
    assert np.linalg.norm(Tm - orc[0]) <= 1e-6 * np.linalg.norm(orc[0])


def test_curved_walls_reset_to_staircase(lbfd_lib, oracle_mod):
    cfg, solid, prims, T, Y, g = cylinders_case()
    s = lbfd_lib.Solver(cfg, solid)
    s.set_curved_walls(prims)
    s.set_curved_walls([])
    s.set_state(T, Y, g)
    s.step(20)
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(20)
    compare_states(s.get_state(), o.get_state(), 1e-10, "staircase again")
