"""The persistent step (lbfd_step_persistent): n steps in one cooperative
launch with a grid-wide barrier between steps.  It runs the per-cell
arithmetic of kernel variant 6, so it must match lbfd_step with that
variant (FP64: 1e-13 relative per field; the same code compiled into
another kernel may contract a multiply-add differently) and the FP64
oracle (1e-10); its bounded barrier must report LBFD_ETIMEOUT, without a
fault, when the wait limit is zero, and leave the handle usable."""
import numpy as np
import pytest

from paper_2304_05657_gb300 import inputs, lbfd

pytestmark = pytest.mark.gpu


def batch_case():
    cfg, solid, T, Y, seg = inputs.batched_channels(widths=[5, 8, 13, 20], length=70, ignite=(10, 25),
                                                     closed_end=False, u_in=0.01)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=21)
    return cfg, solid, T, Y, g


def periodic_blocks_case():
    cfg = inputs.base_config(dim=2, nx=67, ny=30, bc=["periodic"] * 6)
    rng = np.random.default_rng(8)
    solid = np.zeros((30, 67), np.uint8)
    for _ in range(6):
        x, y = rng.integers(0, 60), rng.integers(0, 25)
        solid[y:y + 4, x:x + 5] = 1
    T, Y = inputs.ignition_fields(cfg, solid, 20, 40)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=22)
    return cfg, solid, T, Y, g


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("make", [batch_case, periodic_blocks_case])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_matches_variant6_and_the_oracle(lbfd_lib, oracle_mod, make, precision):
    cfg, solid, T, Y, g = make()
    cfg = dict(cfg, precision=precision)
    steps = 41
    a = lbfd.Solver(cfg, solid)
    a.set_state(T, Y, g)
    a.step_persistent(steps)
    b = lbfd.Solver(cfg, solid)
    b.variant = 6
    b.set_state(T, Y, g)
    b.step(steps)
    assert a.steps_done == b.steps_done == steps
    Ta, Ya, ga = a.get_state()
    Tb, Yb, gb = b.get_state()
    bar = 1e-13 if precision == "fp64" else 1e-6
    fields = [(Ta, Tb)] + [(Ya[k], Yb[k]) for k in range(5)] + [(ga[i], gb[i]) for i in range(9)]
    assert max(rel(x, y) for x, y in fields) <= bar
    if precision == "fp64":
        o = oracle_mod.Sim(cfg, solid)
        o.set_state(T, Y, g)
        o.step(steps)
        To, Yo, go = o.get_state()
        fl = solid.ravel() == 0
        assert rel(Ta[fl], To[fl]) <= 1e-10
        assert max(rel(Ya[k][fl], Yo[k][fl]) for k in range(5)) <= 1e-10
        assert max(rel(ga[i][fl], go[i][fl]) for i in range(9)) <= 1e-10
    # an odd count leaves the state in the other buffer: ordinary steps continue from it
    a.step(3)
    b.step(3)
    assert rel(a.read_field(lbfd.FIELD_T), b.read_field(lbfd.FIELD_T)) <= bar
    a.close()
    b.close()


def test_persistent_wait_limit_reports_timeout_and_recovers(lbfd_lib):
    cfg, solid, T, Y, g = batch_case()
    s = lbfd.Solver(cfg, solid)
    s.set_state(T, Y, g)
    s.set_wait_limit(0)  # no block waits: the first barrier cannot be met
    with pytest.raises(lbfd.LbfdError) as err:
        s.step_persistent(5)
    assert err.value.status == lbfd.ETIMEOUT
    assert "step 1 of 5" in str(err.value)
    assert s.steps_done == 0
    # the handle is still usable: a new state, the default limit, the same result as variant 6
    s.set_wait_limit(2_000_000_000)
    s.set_state(T, Y, g)
    s.step_persistent(7)
    r = lbfd.Solver(cfg, solid)
    r.variant = 6
    r.set_state(T, Y, g)
    r.step(7)
    assert rel(s.read_field(lbfd.FIELD_T), r.read_field(lbfd.FIELD_T)) <= 1e-13
    s.step_persistent(0)
    s.close()
    r.close()


def test_persistent_not_supported_cases(lbfd_lib):
    cfg, solid, T, Y = inputs.sphere_packing(nx=24, ny=12, nz=12, x_range=(4, 20), r_range=(2.0, 3.0))
    s = lbfd.Solver(cfg, solid)
    with pytest.raises(lbfd.LbfdError) as err:
        s.step_persistent(2)
    assert err.value.status == lbfd.ENOTSUP
    s.close()
    cfg2, solid2, T2, Y2 = inputs.channel(nx=30, ny=8)
    t = lbfd.Solver(dict(cfg2, precision="tangent"), solid2)
    with pytest.raises(lbfd.LbfdError) as err:
        t.step_persistent(2)
    assert err.value.status == lbfd.ENOTSUP
    t.close()
