"""Thin ctypes binding of the C ABI in ``include/lbfd.h``.

Function names match the C entry points; this module only marshals
arguments.  Every step of the method runs in the CUDA kernels of
``liblbfd.so``.  There is no CPU fallback: if the library or a CUDA device
is missing, creation fails with an exception.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbfd.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, EUNSTABLE, ENOTSUP = range(8)
BC = {"periodic": 0, "wall_adiabatic": 1, "wall_isothermal": 2, "inlet": 3, "outlet": 4, "outlet_pressure": 5}
FP64, MIXED, TANGENT, TANGENT_MIXED = 0, 1, 2, 3
PRECISION = {"fp64": FP64, "mixed": MIXED, "tangent": TANGENT, "tangent_mixed": TANGENT_MIXED}
OBJ_FLAME_POSITION, OBJ_HEAT_RELEASE, OBJ_QUENCH_DISTANCE = 0, 1, 2
THETA = ("ln_A", "Ta", "T_wall", "u_in")
NSP = 5
FIELD_T, FIELD_Y0, FIELD_UX, FIELD_UY, FIELD_UZ, FIELD_PH, FIELD_RHO, FIELD_HRR, FIELD_G0 = 0, 1, 6, 7, 8, 9, 10, 11, 16
NDIAG = 8
DIAG_KEYS = ("x_f", "mass", "heat_release", "fuel_consumption", "T_max", "x_hrr_max", "n_nonfinite", "n_fluid")

# exported symbols: every entry point declared in include/lbfd.h
SYMBOLS = (
    "lbfd_create", "lbfd_destroy", "lbfd_set_stream", "lbfd_init_fields", "lbfd_set_state", "lbfd_step",
    "lbfd_read_field", "lbfd_diagnostics", "lbfd_flame_position", "lbfd_state_bytes", "lbfd_get_state_raw",
    "lbfd_set_state_raw", "lbfd_steps_done", "lbfd_num_cells", "lbfd_num_populations", "lbfd_strerror",
    "lbfd_last_error", "lbfd_step_graph", "lbfd_num_variants", "lbfd_get_variant", "lbfd_set_variant",
    "lbfd_autotune", "lbfd_diagnostics_noalloc", "lbfd_launches_per_step", "lbfd_read_tangent", "lbfd_gradient",
    "lbfd_diagnostics_rows", "lbfd_set_inlet_velocity", "lbfd_set_curved_walls", "lbfd_read_cells",
    "lbfd_adjoint_gradient", "lbfd_step_persistent", "lbfd_set_wait_limit", "lbfd_adjoint_setup",
    "lbfd_adjoint_record", "lbfd_adjoint_backward", "lbfd_adjoint_run", "lbfd_column_peaks", "lbfd_save",
    "lbfd_load", "lbfd_batch_create",
)


class LbfdError(RuntimeError):
    def __init__(self, status: int, where: str, lib=None):
        msg = f"{where}: status {status}"
        if lib is not None:
            msg += f" ({lib.lbfd_strerror(status).decode()})"
            last = lib.lbfd_last_error().decode()
            if last:
                msg += f" [{last}]"
        super().__init__(msg)
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("bc", ctypes.c_int * 6), ("T_wall", ctypes.c_double * 6)]


class Mechanism(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int), ("W", ctypes.c_double * 8), ("nu_stoich", ctypes.c_double * 8),
                ("fuel", ctypes.c_int), ("oxidiser", ctypes.c_int), ("A", ctypes.c_double),
                ("Ta", ctypes.c_double), ("Q", ctypes.c_double), ("cp", ctypes.c_double),
                ("Le", ctypes.c_double * 8)]


class Params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("Pr", ctypes.c_double), ("omega_bulk", ctypes.c_double),
                ("omega_hi", ctypes.c_double), ("u_in", ctypes.c_double), ("T_in", ctypes.c_double),
                ("Y_in", ctypes.c_double * 8), ("T_solid", ctypes.c_double), ("solid_isothermal", ctypes.c_int),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("T_fp64", ctypes.c_double),
                ("weno_eps", ctypes.c_double), ("precision", ctypes.c_int), ("poiseuille_inlet", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load liblbfd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2304_05657_gb300.build.build()")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    lib.lbfd_create.argtypes = [ctypes.POINTER(Grid), ctypes.c_void_p, ctypes.POINTER(Mechanism),
                                ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]
    lib.lbfd_destroy.argtypes = [H]
    lib.lbfd_set_stream.argtypes = [H, ctypes.c_void_p]
    lib.lbfd_init_fields.argtypes = [H, D, D]
    lib.lbfd_set_state.argtypes = [H, D, D, ctypes.c_void_p]
    lib.lbfd_step.argtypes = [H, ctypes.c_int]
    lib.lbfd_read_field.argtypes = [H, ctypes.c_int, D]
    lib.lbfd_read_cells.argtypes = [H, ctypes.POINTER(ctypes.c_longlong), ctypes.c_longlong, D]
    lib.lbfd_diagnostics.argtypes = [H, D]
    lib.lbfd_flame_position.argtypes = [H, D, D, D]
    lib.lbfd_state_bytes.restype = ctypes.c_size_t
    lib.lbfd_state_bytes.argtypes = [H]
    lib.lbfd_get_state_raw.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t]
    lib.lbfd_set_state_raw.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t]
    lib.lbfd_steps_done.restype = ctypes.c_longlong
    lib.lbfd_steps_done.argtypes = [H]
    lib.lbfd_num_cells.restype = ctypes.c_longlong
    lib.lbfd_num_cells.argtypes = [H]
    lib.lbfd_num_populations.restype = ctypes.c_int
    lib.lbfd_num_populations.argtypes = [H]
    lib.lbfd_step_graph.argtypes = [H, ctypes.c_int]
    lib.lbfd_step_persistent.argtypes = [H, ctypes.c_int]
    lib.lbfd_set_wait_limit.argtypes = [H, ctypes.c_longlong]
    lib.lbfd_num_variants.argtypes = [H]
    lib.lbfd_get_variant.argtypes = [H]
    lib.lbfd_set_variant.argtypes = [H, ctypes.c_int]
    lib.lbfd_launches_per_step.argtypes = [H]
    lib.lbfd_read_tangent.argtypes = [H, ctypes.c_int, ctypes.c_int, D]
    lib.lbfd_diagnostics_rows.argtypes = [H, ctypes.c_int, ctypes.c_int, D]
    lib.lbfd_column_peaks.argtypes = [H, ctypes.c_int, ctypes.c_int, D, D]
    lib.lbfd_save.argtypes = [H, ctypes.c_char_p]
    lib.lbfd_load.argtypes = [H, ctypes.c_char_p]
    lib.lbfd_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                      ctypes.POINTER(Grid), ctypes.POINTER(Mechanism), ctypes.POINTER(Params),
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int)]
    lib.lbfd_set_inlet_velocity.argtypes = [H, ctypes.c_double]
    lib.lbfd_set_curved_walls.argtypes = [H, ctypes.c_int, D]
    lib.lbfd_gradient.argtypes = [H, ctypes.c_int, D, D]
    lib.lbfd_adjoint_gradient.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D]
    lib.lbfd_adjoint_setup.argtypes = [H, ctypes.c_int]
    lib.lbfd_adjoint_record.argtypes = [H, ctypes.c_int, ctypes.c_int, D]
    lib.lbfd_adjoint_backward.argtypes = [H, ctypes.c_double, D]
    lib.lbfd_adjoint_run.argtypes = [H, ctypes.c_int, ctypes.c_int, D, D]
    lib.lbfd_autotune.argtypes = [H, ctypes.c_int, D, ctypes.POINTER(ctypes.c_int)]
    lib.lbfd_diagnostics_noalloc.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Mechanism), ctypes.POINTER(Params),
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                             ctypes.c_void_p, ctypes.c_void_p, D]
    lib.lbfd_strerror.restype = ctypes.c_char_p
    lib.lbfd_strerror.argtypes = [ctypes.c_int]
    lib.lbfd_last_error.restype = ctypes.c_char_p
    lib.lbfd_last_error.argtypes = []
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_structs(cfg: dict):
    g = Grid()
    g.dim, g.nx, g.ny = cfg["dim"], cfg["nx"], cfg["ny"]
    g.nz = cfg["nz"] if cfg["dim"] == 3 else 1
    for f in range(6):
        g.bc[f] = BC[cfg["bc"][f]]
        g.T_wall[f] = cfg["T_wall"][f]
    m = Mechanism()
    m.n_species = len(cfg["W"])
    for k in range(m.n_species):
        m.W[k], m.nu_stoich[k], m.Le[k] = cfg["W"][k], cfg["nu_stoich"][k], cfg["Le"][k]
    m.fuel, m.oxidiser = cfg["fuel"], cfg["oxidiser"]
    m.A, m.Ta, m.Q, m.cp = cfg["A"], cfg["Ta"], cfg["Q"], cfg["cp"]
    p = Params()
    p.nu, p.Pr, p.omega_bulk, p.omega_hi = cfg["nu"], cfg["Pr"], cfg["omega_bulk"], cfg["omega_hi"]
    p.u_in, p.T_in = cfg["u_in"], cfg["T_in"]
    for k in range(len(cfg["Y_in"])):
        p.Y_in[k] = cfg["Y_in"][k]
    p.T_solid, p.solid_isothermal = cfg["T_solid"], int(cfg["solid_isothermal"])
    p.dx, p.dt, p.T_fp64, p.weno_eps = cfg["dx"], cfg["dt"], cfg["T_fp64"], cfg["weno_eps"]
    p.precision = PRECISION[cfg.get("precision", "fp64")]
    p.poiseuille_inlet = int(cfg["poiseuille_inlet"])
    return g, m, p


def _check(lib, st: int, where: str, allow=()):
    if st != OK and st not in allow:
        raise LbfdError(st, where, lib)
    return st


class Solver:
    """One lbfd handle: device-resident state on the current CUDA device."""

    def __init__(self, cfg: dict, solid: np.ndarray, stream=None):
        self.lib = load()
        self.cfg = dict(cfg)
        self._structs = make_structs(cfg)
        g, m, p = self._structs
        solid = np.ascontiguousarray(solid, dtype=np.uint8).ravel()
        if solid.size != inputs.ncells(cfg):
            raise ValueError("mask size does not match the grid")
        h = ctypes.c_void_p()
        st = self.lib.lbfd_create(ctypes.byref(g), solid.ctypes.data_as(ctypes.c_void_p), ctypes.byref(m),
                                  ctypes.byref(p), ctypes.byref(h))
        _check(self.lib, st, "lbfd_create")
        self.h = h
        self.N = int(self.lib.lbfd_num_cells(h))
        self.Q = int(self.lib.lbfd_num_populations(h))
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbfd_destroy(self.h)
            self.h = None

    __del__ = close

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        _check(self.lib, self.lib.lbfd_set_stream(self.h, ctypes.c_void_p(handle or 0)), "lbfd_set_stream")

    def init_fields(self, T, Y):
        T = np.ascontiguousarray(T, dtype=np.float64).ravel()
        Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(NSP, self.N)
        _check(self.lib, self.lib.lbfd_init_fields(self.h, _dp(T), _dp(Y)), "lbfd_init_fields")

    def set_state(self, T, Y, g=None):
        T = np.ascontiguousarray(T, dtype=np.float64).ravel()
        Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(NSP, self.N)
        gp = None
        if g is not None:
            g = np.ascontiguousarray(g, dtype=np.float64).reshape(self.Q, self.N)
            gp = g.ctypes.data_as(ctypes.c_void_p)
        _check(self.lib, self.lib.lbfd_set_state(self.h, _dp(T), _dp(Y), gp), "lbfd_set_state")

    def step(self, n: int = 1):
        _check(self.lib, self.lib.lbfd_step(self.h, int(n)), "lbfd_step")

    def step_graph(self, n: int):
        _check(self.lib, self.lib.lbfd_step_graph(self.h, int(n)), "lbfd_step_graph")

    def step_persistent(self, n: int):
        """n steps in one persistent launch (grid-wide barriers between
        steps); raises LbfdError with status ETIMEOUT when a barrier wait
        gave up."""
        _check(self.lib, self.lib.lbfd_step_persistent(self.h, int(n)), "lbfd_step_persistent")

    def set_wait_limit(self, ns: int):
        _check(self.lib, self.lib.lbfd_set_wait_limit(self.h, int(ns)), "lbfd_set_wait_limit")

    @property
    def num_variants(self) -> int:
        return int(self.lib.lbfd_num_variants(self.h))

    @property
    def variant(self) -> int:
        return int(self.lib.lbfd_get_variant(self.h))

    @variant.setter
    def variant(self, v: int):
        _check(self.lib, self.lib.lbfd_set_variant(self.h, int(v)), "lbfd_set_variant")

    def read_tangent(self, field: int, k: int) -> np.ndarray:
        """Derivative k (order of THETA) of a raw field; tangent precision."""
        out = np.empty(self.N)
        _check(self.lib, self.lib.lbfd_read_tangent(self.h, int(field), int(k), _dp(out)), "lbfd_read_tangent")
        return out

    def gradient(self, objective: int = OBJ_FLAME_POSITION):
        """(J, dJ/dtheta) of the current state; tangent precision."""
        val = np.zeros(1)
        grad = np.zeros(4)
        _check(self.lib, self.lib.lbfd_gradient(self.h, int(objective), _dp(val), _dp(grad)), "lbfd_gradient")
        return float(val[0]), grad

    def adjoint_gradient(self, steps: int, checkpoint_every: int = 200, objective: int = OBJ_FLAME_POSITION):
        """Advance `steps` steps and return (J, dJ/dtheta) by the discrete
        adjoint with checkpoints every `checkpoint_every` steps (FP64)."""
        val = np.zeros(1)
        grad = np.zeros(4)
        st = self.lib.lbfd_adjoint_gradient(self.h, int(steps), int(checkpoint_every), int(objective), _dp(val),
                                            _dp(grad))
        _check(self.lib, st, "lbfd_adjoint_gradient")
        return float(val[0]), grad

    def adjoint_setup(self, checkpoint_every: int):
        _check(self.lib, self.lib.lbfd_adjoint_setup(self.h, int(checkpoint_every)), "lbfd_adjoint_setup")

    def adjoint_record(self, steps: int, objective: int = OBJ_FLAME_POSITION) -> float:
        """Advance `steps` steps keeping checkpoints; J of the final state."""
        val = np.zeros(1)
        _check(self.lib, self.lib.lbfd_adjoint_record(self.h, int(steps), int(objective), _dp(val)),
               "lbfd_adjoint_record")
        return float(val[0])

    def adjoint_backward(self, seed: float = 1.0) -> np.ndarray:
        """seed * dJ/dtheta by the backward sweep over the recorded steps."""
        grad = np.zeros(4)
        _check(self.lib, self.lib.lbfd_adjoint_backward(self.h, float(seed), _dp(grad)), "lbfd_adjoint_backward")
        return grad

    def adjoint_run(self, steps: int, objective: int = OBJ_FLAME_POSITION):
        val = np.zeros(1)
        grad = np.zeros(4)
        _check(self.lib, self.lib.lbfd_adjoint_run(self.h, int(steps), int(objective), _dp(val), _dp(grad)),
               "lbfd_adjoint_run")
        return float(val[0]), grad

    @property
    def launches_per_step(self) -> int:
        return int(self.lib.lbfd_launches_per_step(self.h))

    def autotune(self, reps: int = 20):
        """Time every kernel variant on the current state and keep the
        fastest; returns (best, ms per variant)."""
        ms = np.zeros(self.num_variants)
        best = ctypes.c_int()
        _check(self.lib, self.lib.lbfd_autotune(self.h, int(reps), _dp(ms), ctypes.byref(best)), "lbfd_autotune")
        return best.value, ms

    def read_field(self, field: int) -> np.ndarray:
        out = np.empty(self.N)
        _check(self.lib, self.lib.lbfd_read_field(self.h, int(field), _dp(out)), "lbfd_read_field")
        return out

    def read_cells(self, cells) -> np.ndarray:
        """The state of the listed cells: float64 [n, Q + 1 + 5] with the
        columns g_0 .. g_{Q-1}, T, Y_0 .. Y_4."""
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).ravel())
        out = np.empty((cells.size, self.Q + 1 + NSP))
        st = self.lib.lbfd_read_cells(self.h, cells.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                      int(cells.size), _dp(out))
        _check(self.lib, st, "lbfd_read_cells")
        return out

    def get_state(self):
        """(T[N], Y[5,N], g[Q,N]) as float64 host arrays."""
        T = self.read_field(FIELD_T)
        Y = np.stack([self.read_field(FIELD_Y0 + k) for k in range(NSP)])
        g = np.stack([self.read_field(FIELD_G0 + i) for i in range(self.Q)])
        return T, Y, g

    def diagnostics(self, rows=None) -> dict:
        """Reductions over the fluid cells (all, or the rows y0 <= y < y1)."""
        out = np.empty(NDIAG)
        if rows is None:
            st = self.lib.lbfd_diagnostics(self.h, _dp(out))
        else:
            st = self.lib.lbfd_diagnostics_rows(self.h, int(rows[0]), int(rows[1]), _dp(out))
        _check(self.lib, st, "lbfd_diagnostics", allow=(ENONFINITE,))
        return dict(zip(DIAG_KEYS, out.tolist()))

    def column_peaks(self, rows=None):
        """(peak heat release per column, distance of the peak to the nearer
        edge of the rows y0 <= y < y1) over all x; 2-D."""
        y0, y1 = rows if rows is not None else (0, self.cfg["ny"])
        peak = np.empty(self.cfg["nx"])
        dist = np.empty(self.cfg["nx"])
        _check(self.lib, self.lib.lbfd_column_peaks(self.h, int(y0), int(y1), _dp(peak), _dp(dist)),
               "lbfd_column_peaks")
        return peak, dist

    def save(self, path: str):
        _check(self.lib, self.lib.lbfd_save(self.h, os.fsencode(path)), "lbfd_save")

    def load(self, path: str):
        _check(self.lib, self.lib.lbfd_load(self.h, os.fsencode(path)), "lbfd_load")

    def set_curved_walls(self, prims):
        """Curved walls from primitives (type, p0, p1, p2, p3); see lbfd.h."""
        arr = np.ascontiguousarray(np.asarray(prims, dtype=np.float64).reshape(-1, 5))
        _check(self.lib, self.lib.lbfd_set_curved_walls(self.h, int(arr.shape[0]), _dp(arr)), "lbfd_set_curved_walls")

    def set_inlet_velocity(self, u_in: float):
        _check(self.lib, self.lib.lbfd_set_inlet_velocity(self.h, float(u_in)), "lbfd_set_inlet_velocity")
        self.cfg["u_in"] = float(u_in)

    def flame_position(self):
        x, m, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self.lib, self.lib.lbfd_flame_position(self.h, ctypes.byref(x), ctypes.byref(m), ctypes.byref(q)),
               "lbfd_flame_position", allow=(ENONFINITE,))
        return x.value, m.value, q.value

    def state_bytes(self) -> int:
        return int(self.lib.lbfd_state_bytes(self.h))

    def get_state_raw(self, ptr: int, nbytes: int):
        _check(self.lib, self.lib.lbfd_get_state_raw(self.h, ctypes.c_void_p(ptr), nbytes), "lbfd_get_state_raw")

    def set_state_raw(self, ptr: int, nbytes: int):
        _check(self.lib, self.lib.lbfd_set_state_raw(self.h, ctypes.c_void_p(ptr), nbytes), "lbfd_set_state_raw")

    @property
    def steps_done(self) -> int:
        return int(self.lib.lbfd_steps_done(self.h))


def batch_create(widths, length: int, cfg: dict, stream=None):
    """lbfd_batch_create: one Solver for 2-D channels of the given widths
    stacked along y with a solid row between them; returns (solver, rows)
    with rows = [(y0, y1), ...] per channel.  cfg gives the face types,
    mechanism and parameters (its nx, ny are replaced)."""
    lib = load()
    widths = [int(w) for w in widths]
    g, m, p = make_structs(cfg)
    wa = (ctypes.c_int * len(widths))(*widths)
    rows = (ctypes.c_int * (2 * len(widths)))()
    h = ctypes.c_void_p()
    st = lib.lbfd_batch_create(len(widths), wa, int(length), ctypes.byref(g), ctypes.byref(m), ctypes.byref(p),
                               ctypes.byref(h), rows)
    _check(lib, st, "lbfd_batch_create")
    ny = sum(widths) + len(widths) - 1
    s = Solver.__new__(Solver)
    s.lib = lib
    s.cfg = dict(cfg, nx=int(length), ny=ny, nz=1)
    s._structs = make_structs(s.cfg)
    s.h = h
    s.N = int(lib.lbfd_num_cells(h))
    s.Q = int(lib.lbfd_num_populations(h))
    if stream is not None:
        s.set_stream(stream)
    return s, [(rows[2 * j], rows[2 * j + 1]) for j in range(len(widths))]


def diagnostics_noalloc(cfg: dict, g_ptr: int, T_ptr: int, Y_ptr: int, plane_stride: int, solid_ptr: int,
                        stream=None) -> dict:
    """lbfd_diagnostics_noalloc on caller-owned device buffers (integer
    device addresses, e.g. torch tensors' data_ptr()); the library
    allocates nothing for this call."""
    lib = load()
    g, m, p = make_structs(cfg)
    out = np.empty(NDIAG)
    handle = getattr(stream, "cuda_stream", stream) or 0
    st = lib.lbfd_diagnostics_noalloc(ctypes.byref(g), ctypes.byref(m), ctypes.byref(p), ctypes.c_void_p(g_ptr),
                                      ctypes.c_void_p(T_ptr), ctypes.c_void_p(Y_ptr), int(plane_stride),
                                      ctypes.c_void_p(solid_ptr), ctypes.c_void_p(handle), _dp(out))
    _check(lib, st, "lbfd_diagnostics_noalloc", allow=(ENONFINITE,))
    return dict(zip(DIAG_KEYS, out.tolist()))
