"""The allocation-free diagnostics entry point, for callers that cannot call
cudaMalloc (their device memory belongs to a host framework or a fixed
budget, or they may not synchronise the device or fail on memory pressure
after start-up).  It must return what lbfd_diagnostics returns, on two calls
in a row (its scratch is a static device array shared by every call).

This file is collected last on purpose; it runs the same alone in a fresh
process and after the other tests (the scratch address is looked up once per
device and cached)."""
import ctypes

import numpy as np
import pytest

from paper_2304_05657_gb300 import inputs

pytestmark = pytest.mark.gpu

EXACT = ("x_hrr_max", "n_nonfinite", "n_fluid")


def device_state(torch, s, solid):
    """Copy a solver's state into caller-owned device buffers (dense planes)."""
    nbytes = s.state_bytes()
    host = np.empty(nbytes, dtype=np.uint8)
    s.get_state_raw(host.ctypes.data, nbytes)
    dev = torch.from_numpy(host).cuda()
    mask = torch.from_numpy(np.ascontiguousarray(solid, dtype=np.uint8).ravel()).cuda()
    return dev, mask


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_diagnostics_match_the_allocating_entry_point(lbfd_lib, precision):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    cfg, solid, T, Y = inputs.channel(nx=150, ny=37, ignite=(0, 20))
    T, Y = inputs.ignition_fields(cfg, solid, 40, 60, burnt=False)
    cfg = dict(cfg, precision=precision)
    s = lbfd_lib.Solver(cfg, solid)
    s.set_state(T, Y)
    s.step(40)
    ref = s.diagnostics()
    assert ref["heat_release"] > 0.0
    dev, mask = device_state(torch, s, solid)
    esz = 8 if precision == "fp64" else 4
    N = s.N
    g_ptr = dev.data_ptr()
    T_ptr = g_ptr + s.Q * N * esz
    Y_ptr = T_ptr + N * esz
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    for call in range(2):
        got = lbfd_lib.diagnostics_noalloc(cfg, g_ptr, T_ptr, Y_ptr, N, mask.data_ptr(), stream)
        for key, val in ref.items():
            if key in EXACT:
                assert got[key] == val, (call, key, got[key], val)
            else:
                assert abs(got[key] - val) <= 1e-11 * max(1.0, abs(val)), (call, key, got[key], val)


def test_noalloc_rejects_bad_arguments(lbfd_lib):
    torch = pytest.importorskip("torch")
    cfg, solid, T, Y = inputs.channel(nx=40, ny=10)
    N = solid.size
    buf = torch.zeros(15 * N, dtype=torch.float64, device="cuda")
    mask = torch.zeros(N, dtype=torch.uint8, device="cuda")
    lib = lbfd_lib.load()
    g, m, p = lbfd_lib.make_structs(cfg)
    out = np.empty(lbfd_lib.NDIAG)
    outp = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ptr = buf.data_ptr()
    # plane stride smaller than the grid
    st = lib.lbfd_diagnostics_noalloc(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p), ctypes.c_void_p(ptr),
                                      ctypes.c_void_p(ptr), ctypes.c_void_p(ptr), N - 1,
                                      ctypes.c_void_p(mask.data_ptr()), None, outp)
    assert st == lbfd_lib.EINVAL and b"plane_stride" in lib.lbfd_last_error()
    # a host pointer where a device pointer is required
    host = np.zeros(15 * N)
    st = lib.lbfd_diagnostics_noalloc(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p),
                                      ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(ptr),
                                      ctypes.c_void_p(ptr), N, ctypes.c_void_p(mask.data_ptr()), None, outp)
    assert st == lbfd_lib.EINVAL and b"device pointers" in lib.lbfd_last_error()
