"""Plain FP64 CPU oracle for the coupled LB/FD step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The CUDA library and its Python binding
never do.  The C source (``orc.c``) shares no code with the CUDA path; this
wrapper only marshals arguments through ctypes.

Parity pins of every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

MAXSP = 8
BC = {"periodic": 0, "wall_adiabatic": 1, "wall_isothermal": 2, "inlet": 3, "outlet": 4,
      "outlet_pressure": 5}


def build(force: bool = False) -> str:
    """Compile ``orc.c`` into ``liborc.so`` (plain gcc, FP contraction off)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP only threads orc_step over grid rows (for timing on all host
        # cores); without it the oracle is the same single-threaded code
        r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True)
        if r.returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class Setup(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 6), ("T_wall", ctypes.c_double * 6),
        ("n_species", ctypes.c_int),
        ("W", ctypes.c_double * MAXSP), ("nu_stoich", ctypes.c_double * MAXSP),
        ("Le", ctypes.c_double * MAXSP),
        ("fuel", ctypes.c_int), ("oxid", ctypes.c_int),
        ("A", ctypes.c_double), ("Ta", ctypes.c_double), ("Q", ctypes.c_double),
        ("cp", ctypes.c_double), ("dt", ctypes.c_double),
        ("nu", ctypes.c_double), ("Pr", ctypes.c_double),
        ("omega_bulk", ctypes.c_double), ("omega_hi", ctypes.c_double),
        ("u_in", ctypes.c_double), ("T_in", ctypes.c_double), ("Y_in", ctypes.c_double * MAXSP),
        ("T_solid", ctypes.c_double), ("solid_isothermal", ctypes.c_int),
        ("poiseuille_inlet", ctypes.c_int), ("weno_eps", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        lib.orc_new.restype = P
        lib.orc_new.argtypes = [ctypes.POINTER(Setup), ctypes.c_void_p]
        lib.orc_free.argtypes = [P]
        lib.orc_ncells.restype = ctypes.c_long
        lib.orc_ncells.argtypes = [P]
        lib.orc_q.restype = ctypes.c_int
        lib.orc_q.argtypes = [P]
        lib.orc_omega_s.restype = ctypes.c_double
        lib.orc_omega_s.argtypes = [P]
        lib.orc_set_state.argtypes = [P, D, D, ctypes.c_void_p]
        lib.orc_get_state.argtypes = [P, D, D, D]
        lib.orc_step.argtypes = [P, ctypes.c_int]
        lib.orc_step_slab.argtypes = [P, ctypes.c_int, ctypes.c_int]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_openmp.restype = ctypes.c_int
        lib.orc_set_geometry.argtypes = [P, ctypes.c_int, D]
        lib.orc_num_ghosts.restype = ctypes.c_long
        lib.orc_num_ghosts.argtypes = [P]
        lib.orc_cell_terms.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, D]
        lib.orc_collide_cell.argtypes = [P, D, ctypes.c_double, D, D, ctypes.c_double, D, D, D]
        lib.orc_central_moments.argtypes = [P, D, D, D]
        lib.orc_central_moments_inverse.argtypes = [P, D, D, D]
        lib.orc_diagnostics.argtypes = [P, D]
        lib.orc_column_peaks.argtypes = [P, ctypes.c_int, ctypes.c_int, D, D]
        lib.orc_cumulants.argtypes = [ctypes.c_int, D, D]
        lib.orc_cumulants_inverse.argtypes = [ctypes.c_int, D, D]
        lib.orc_weno3.restype = ctypes.c_double
        lib.orc_weno3.argtypes = [D, ctypes.c_double, ctypes.c_double]
        for name in ("orc_d1", "orc_d2", "orc_c2"):
            getattr(lib, name).restype = ctypes.c_double
            getattr(lib, name).argtypes = [D]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_setup(cfg: dict) -> Setup:
    """Fill the oracle's setup struct from a plain configuration dict
    (the dict produced by ``paper_2304_05657_gb300.inputs``)."""
    s = Setup()
    s.dim = cfg["dim"]
    s.nx, s.ny = cfg["nx"], cfg["ny"]
    s.nz = cfg.get("nz", 1) if cfg["dim"] == 3 else 1
    for f in range(6):
        s.bc[f] = BC[cfg["bc"][f]]
        s.T_wall[f] = cfg["T_wall"][f]
    nsp = len(cfg["W"])
    s.n_species = nsp
    for k in range(nsp):
        s.W[k] = cfg["W"][k]
        s.nu_stoich[k] = cfg["nu_stoich"][k]
        s.Le[k] = cfg["Le"][k]
        s.Y_in[k] = cfg["Y_in"][k]
    s.fuel, s.oxid = cfg["fuel"], cfg["oxidiser"]
    s.A, s.Ta, s.Q, s.cp, s.dt = cfg["A"], cfg["Ta"], cfg["Q"], cfg["cp"], cfg["dt"]
    s.nu, s.Pr = cfg["nu"], cfg["Pr"]
    s.omega_bulk, s.omega_hi = cfg["omega_bulk"], cfg["omega_hi"]
    s.u_in, s.T_in = cfg["u_in"], cfg["T_in"]
    s.T_solid = cfg["T_solid"]
    s.solid_isothermal = int(cfg["solid_isothermal"])
    s.poiseuille_inlet = int(cfg["poiseuille_inlet"])
    s.weno_eps = cfg["weno_eps"]
    return s


class Sim:
    """One oracle simulation: FP64 state on the host, advanced cell by cell."""

    def __init__(self, cfg: dict, solid: np.ndarray):
        self.lib = _load()
        self.cfg = dict(cfg)
        self.setup = make_setup(cfg)
        self.nsp = len(cfg["W"])
        solid = np.ascontiguousarray(solid, dtype=np.uint8).ravel()
        self._solid = solid
        self.h = self.lib.orc_new(ctypes.byref(self.setup), solid.ctypes.data_as(ctypes.c_void_p))
        if not self.h:
            raise MemoryError("oracle allocation failed")
        self.N = int(self.lib.orc_ncells(self.h))
        self.Q = int(self.lib.orc_q(self.h))
        assert solid.size == self.N

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_free(h)
            self.h = None

    @property
    def omega_s(self) -> float:
        return float(self.lib.orc_omega_s(self.h))

    def set_state(self, T, Y, g=None):
        T = np.ascontiguousarray(T, dtype=np.float64).ravel()
        Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(self.nsp, self.N)
        gp = None
        if g is not None:
            g = np.ascontiguousarray(g, dtype=np.float64).reshape(self.Q, self.N)
            gp = g.ctypes.data_as(ctypes.c_void_p)
        self.lib.orc_set_state(self.h, _dp(T), _dp(Y), gp)

    def get_state(self):
        T = np.empty(self.N)
        Y = np.empty((self.nsp, self.N))
        g = np.empty((self.Q, self.N))
        self.lib.orc_get_state(self.h, _dp(T), _dp(Y), _dp(g))
        return T, Y, g

    def step(self, n: int = 1):
        self.lib.orc_step(self.h, int(n))

    def set_geometry(self, prims):
        """Curved walls: prims is a list of (type, p0, p1, p2, p3) with
        type 0 = sphere/circle (centre, radius), 1 = half-space (unit normal
        into the solid, offset); cell centres at (x+.5, y+.5, z+.5)."""
        arr = np.ascontiguousarray(np.asarray(prims, dtype=np.float64).reshape(-1, 5))
        self._prims = arr
        self.lib.orc_set_geometry(self.h, int(arr.shape[0]), _dp(arr))

    @property
    def num_ghosts(self) -> int:
        return int(self.lib.orc_num_ghosts(self.h))

    def step_slab(self, x0: int, x1: int):
        """One step of the cells x0 <= x < x1 only."""
        self.lib.orc_step_slab(self.h, int(x0), int(x1))

    def cell_terms(self, x: int, y: int, z: int = 0) -> dict:
        nsp, Q = self.nsp, self.Q
        out = np.zeros(12 + 3 * nsp + 2 * Q + 1 + nsp)
        self.lib.orc_cell_terms(self.h, x, y, z, _dp(out))
        o = 0
        r = {}
        r["rho"] = out[o]; o += 1
        r["u"] = out[o:o + 3].copy(); o += 3
        r["grad_rho"] = out[o:o + 3].copy(); o += 3
        for key in ("conv_T", "diff_T", "reac_T", "Lambda", "P_h"):
            r[key] = out[o]; o += 1
        for key in ("conv_Y", "diff_Y", "reac_Y"):
            r[key] = out[o:o + nsp].copy(); o += nsp
        r["g_in"] = out[o:o + Q].copy(); o += Q
        r["g_star"] = out[o:o + Q].copy(); o += Q
        r["T_new"] = out[o]; o += 1
        r["Y_new"] = out[o:o + nsp].copy(); o += nsp
        return r

    def collide_cell(self, g, rho, u, grad_rho, Lam):
        g = np.ascontiguousarray(g, dtype=np.float64)
        u = np.ascontiguousarray(np.resize(np.asarray(u, np.float64), 3))
        gr = np.ascontiguousarray(np.resize(np.asarray(grad_rho, np.float64), 3))
        gs = np.zeros(self.Q)
        xi = np.zeros(self.Q)
        ph = ctypes.c_double()
        self.lib.orc_collide_cell(self.h, _dp(g), float(rho), _dp(u), _dp(gr), float(Lam),
                                  _dp(gs), _dp(xi), ctypes.byref(ph))
        return gs, xi, ph.value

    def central_moments(self, f, u):
        f = np.ascontiguousarray(f, dtype=np.float64)
        u = np.ascontiguousarray(np.resize(np.asarray(u, np.float64), 3))
        Pi = np.zeros(self.Q)
        self.lib.orc_central_moments(self.h, _dp(f), _dp(u), _dp(Pi))
        return Pi

    def central_moments_inverse(self, Pi, u):
        Pi = np.ascontiguousarray(Pi, dtype=np.float64)
        u = np.ascontiguousarray(np.resize(np.asarray(u, np.float64), 3))
        f = np.zeros(self.Q)
        self.lib.orc_central_moments_inverse(self.h, _dp(Pi), _dp(u), _dp(f))
        return f

    def column_peaks(self, rows=None):
        """Per column: the peak heat release over rows y0 <= y < y1 and its
        distance to the nearer edge of the band (2-D)."""
        y0, y1 = rows if rows is not None else (0, self.cfg["ny"])
        peak = np.zeros(self.cfg["nx"])
        dist = np.zeros(self.cfg["nx"])
        self.lib.orc_column_peaks(self.h, int(y0), int(y1), _dp(peak), _dp(dist))
        return peak, dist

    def diagnostics(self) -> dict:
        out = np.zeros(8)
        self.lib.orc_diagnostics(self.h, _dp(out))
        keys = ("x_f", "mass", "heat_release", "fuel_consumption", "T_max", "x_hrr_max",
                "n_nonfinite", "n_fluid")
        return dict(zip(keys, out.tolist()))


def set_threads(n: int) -> int:
    """Threads of every later step (1 unless changed; the result does not
    depend on it).  Returns the count in effect: 1 when the library was
    built without OpenMP."""
    lib = _load()
    if not lib.orc_openmp():
        n = 1
    lib.orc_set_threads(int(n))
    return max(1, int(n))


def cumulants(dim: int, Pi):
    Pi = np.ascontiguousarray(Pi, dtype=np.float64)
    K = np.zeros_like(Pi)
    _load().orc_cumulants(dim, _dp(Pi), _dp(K))
    return K


def cumulants_inverse(dim: int, K):
    K = np.ascontiguousarray(K, dtype=np.float64)
    Pi = np.zeros_like(K)
    _load().orc_cumulants_inverse(dim, _dp(K), _dp(Pi))
    return Pi


def weno3(v, u: float, eps: float) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(_load().orc_weno3(_dp(v), float(u), float(eps)))


def d1(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(_load().orc_d1(_dp(v)))


def d2(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(_load().orc_d2(_dp(v)))


def c2(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(_load().orc_c2(_dp(v)))
