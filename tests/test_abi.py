"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/lbfd.h declares (no compute call is made here)."""
import ctypes
import os
import re

from paper_2304_05657_gb300 import build, lbfd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbfd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbfd_[a-z_0-9]+)\s*\(", text)))


def test_header_matches_binding_list():
    assert declared_functions() == sorted(lbfd.SYMBOLS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [name for name in declared_functions() if not hasattr(lib, name)]
    assert not missing, missing


def test_strerror_and_no_device_path():
    lib = lbfd.load(build.build())
    assert lib.lbfd_strerror(0) == b"ok"
    assert lib.lbfd_strerror(6).startswith(b"parameters")
    # null arguments are rejected before any CUDA call
    assert lib.lbfd_create(None, None, None, None, None) == lbfd.EINVAL
    assert lib.lbfd_step(None, 1) == lbfd.EINVAL
    assert lib.lbfd_destroy(None) == lbfd.OK


def test_create_rejects_unstable_and_invalid_parameters_without_a_gpu():
    """Validation runs before any CUDA call, so it is testable on the CPU."""
    import ctypes

    from paper_2304_05657_gb300 import inputs

    lib = lbfd.load(build.build())

    def create(**over):
        cfg = inputs.base_config(**over)
        g, m, p = lbfd.make_structs(cfg)
        h = ctypes.c_void_p()
        mask = (ctypes.c_uint8 * (cfg["nx"] * cfg["ny"]))()
        return lib.lbfd_create(ctypes.byref(g), mask, ctypes.byref(m), ctypes.byref(p), ctypes.byref(h))

    assert create(u_in=0.7) == lbfd.EUNSTABLE          # |u_in| >= cs
    assert create(nu=0.2) == lbfd.EUNSTABLE            # explicit-Euler Fourier limit
    assert create(omega_hi=2.5) == lbfd.EUNSTABLE
    assert create(Y_in=[0.5, 0.2, 0.0, 0.0, 0.2]) == lbfd.EINVAL  # sum != 1
    assert create(bc=["periodic", "outlet", "periodic", "periodic", "periodic", "periodic"]) == lbfd.EINVAL
    assert create(nx=0) == lbfd.EINVAL


def test_noalloc_entry_point_names_no_allocation():
    """The allocation-free diagnostics must not allocate: neither its body
    nor the helpers it calls in its translation unit name an allocating
    CUDA call."""
    src = open(os.path.join(ROOT, "paper_2304_05657_gb300", "csrc", "lbfd_api.cu")).read()
    start = src.index("static __device__ __align__(256) double lbfd_noalloc_scratch")
    body = src[start:]
    for name in ("cudaMalloc", "cudaFree", "cudaMallocAsync", "cudaMallocHost", "malloc(", "new "):
        assert name not in body, name
    # the reduction it launches clears its own words in the kernel launcher
    red = open(os.path.join(ROOT, "paper_2304_05657_gb300", "csrc", "lbfd_reduce.cu")).read()
    for fn in ("static cudaError_t diag_launch(", "cudaError_t launch_diagnostics("):
        body = red[red.index(fn):]
        body = body[:body.index("\n}\n")]
        assert "cudaMalloc" not in body and "cudaFree" not in body, fn
