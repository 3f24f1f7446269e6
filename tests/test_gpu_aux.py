"""Auxiliary entry points on the GPU: checkpoint save/load (resume),
non-finite detection, batch creation, through the C ABI."""
import ctypes

import numpy as np
import pytest

from paper_2304_05657_gb300 import inputs, lbfd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_save_load_resumes_bit_exactly(lbfd_lib, tmp_path, precision):
    cfg, solid, T, Y = inputs.channel(nx=60, ny=14, walls="isothermal", ignite=(10, 25))
    cfg = dict(cfg, precision=precision)
    a = lbfd.Solver(cfg, solid)
    a.init_fields(T, Y)
    a.step(17)
    path = str(tmp_path / "state.lbfd")
    a.save(path)
    a.step(13)
    b = lbfd.Solver(cfg, solid)
    b.load(path)
    assert b.steps_done == 17
    b.step(13)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    # a file of another precision or grid is refused
    c = lbfd.Solver(dict(cfg, precision="mixed" if precision == "fp64" else "fp64"), solid)
    with pytest.raises(lbfd.LbfdError) as err:
        c.load(path)
    assert err.value.status == lbfd.EINVAL and "not a checkpoint" in str(err.value)
    cfg2, solid2, _, _ = inputs.channel(nx=61, ny=14)
    d = lbfd.Solver(dict(cfg2, precision=precision), solid2)
    with pytest.raises(lbfd.LbfdError):
        d.load(path)
    for s in (a, b, c, d):
        s.close()


def test_nonfinite_value_is_reported(lbfd_lib):
    """A NaN injected on the host into one fluid cell: the diagnostics
    return LBFD_ENONFINITE with a count of one cell (the sums leave it out),
    and after a step the value has spread to its neighbours."""
    cfg, solid, T, Y = inputs.channel(nx=40, ny=10, ignite=(10, 20))
    s = lbfd.Solver(cfg, solid)
    T2 = T.copy()
    T2[5 * 40 + 30] = np.nan
    s.set_state(T2, Y)
    out = np.empty(lbfd.NDIAG)
    st = s.lib.lbfd_diagnostics(s.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert st == lbfd.ENONFINITE
    assert out[6] == 1 and np.isfinite(out[1])
    s.step(1)
    assert s.diagnostics()["n_nonfinite"] > 1
    s.close()


def test_batch_create_packs_channels_like_the_host_recipe(lbfd_lib, oracle_mod):
    """lbfd_batch_create builds the packed mask itself: same rows as the
    seeded host recipe, and the same step as a handle made from that mask."""
    widths = [6, 9, 11]
    cfg, solid, T, Y, seg = inputs.batched_channels(widths=widths, length=50, ignite=(10, 20), closed_end=False,
                                                     u_in=0.01)
    s, rows = lbfd.batch_create(widths, 50, cfg)
    assert rows == seg
    r = lbfd.Solver(cfg, solid)
    for h in (s, r):
        h.init_fields(T, Y)
        h.step(20)
    for x, y in zip(s.get_state(), r.get_state()):
        assert np.array_equal(x, y)
    s.close()
    r.close()
