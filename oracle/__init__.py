"""FP64 CPU oracle of the coupled three-lattice CSF lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library: the C source ``lbe_oracle.c`` is compiled
here with gcc and loaded with ctypes.

Populations are numpy arrays of shape (27, ny, nx): planes f_0..f_8, g_0..g_8,
hbar_0..hbar_8 (Sec. II Eq. 12, Eq. 27; Sec. III Eq. aEq12), x fastest.

Parameters are plain dicts with the keys of ``PARAM_KEYS``.  ``sigmaT`` is the
positive coefficient of sigma = sigma0 - sigmaT (T - Tref), i.e. minus the
paper's d sigma/d T of Eq. aEq3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

PARAM_KEYS = ("rho", "cv", "eta1", "eta2", "lam1", "lam2", "sigma0", "sigmaT",
              "Tref", "eps", "beta", "tau_g", "mobility", "ax", "ay", "eta_n")


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("periodic_y", ctypes.c_int32), ("ablate", ctypes.c_int32)] + \
               [(k, ctypes.c_double) for k in PARAM_KEYS] + [("rho2", ctypes.c_double)] + \
               [("interp", ctypes.c_int32), ("wall_mid", ctypes.c_int32),
                ("cos_wet", ctypes.c_double), ("dissip", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            P = ctypes.POINTER(_Params)
            L.orc_init.argtypes = [P, dp, dp, dp, dp, dp]
            L.orc_init.restype = ctypes.c_int
            L.orc_run.argtypes = [P, dp, dp, dp, dp, ctypes.c_int64]
            L.orc_run.restype = ctypes.c_int
            L.orc_fields.argtypes = [P, dp, dp, dp, dp, dp, dp, dp, dp]
            L.orc_fields.restype = None
            L.orc_scalar_ops.argtypes = [P, dp, dp, dp, dp, dp] + [dp] * 11
            L.orc_scalar_ops.restype = None
            L.orc_cell_terms.argtypes = [P] + [ctypes.c_double] * 10 + [dp] * 6
            L.orc_cell_terms.restype = None
            ip = ctypes.POINTER(ctypes.c_int32)
            L.orc_lattice.argtypes = [ip, ip, dp, ip, dp]
            L.orc_lattice.restype = None
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_set_threads.restype = None
            _lib = L
    return _lib


def _p(params: dict, nx: int, ny: int) -> _Params:
    s = _Params()
    s.nx, s.ny = int(nx), int(ny)
    s.periodic_y = int(params.get("periodic_y", 0))
    for k in PARAM_KEYS:
        setattr(s, k, float(params[k]))
    # density of phase c = 1 (default: uniform density); ablate: test hook
    # planting a mistake in the density terms (see lbe_oracle.c)
    s.rho2 = float(params.get("rho2", params["rho"]))
    s.ablate = int(params.get("ablate", 0))
    # variants: property law (0 linear, 1 harmonic), wall temperature at the
    # link's crossing point, contact angle of phase 1 (cos; 0: neutral)
    s.interp = int(params.get("interp", 0))
    s.wall_mid = int(params.get("wall_mid", 0))
    s.cos_wet = float(params.get("cos_wet", 0.0))
    # the pressure-work / viscous-dissipation term of Eq. aEq7 (0: dropped)
    s.dissip = int(params.get("dissip", 0))
    return s


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.shape != shape:
        a = np.ascontiguousarray(np.broadcast_to(a, shape))
    return a


def lattice():
    """(ex, ey, w, opp, cs2) of the oracle's D2Q9 set."""
    ex = (ctypes.c_int32 * 9)()
    ey = (ctypes.c_int32 * 9)()
    w = (ctypes.c_double * 9)()
    op = (ctypes.c_int32 * 9)()
    cs2 = ctypes.c_double()
    lib().orc_lattice(ex, ey, w, op, ctypes.byref(cs2))
    return (np.array(ex[:]), np.array(ey[:]), np.array(w[:]), np.array(op[:]),
            cs2.value)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of the following calls (0: one per processor)."""
    lib().orc_set_threads(int(n))


def init(params: dict, c0, T0, Tbot, Ttop) -> np.ndarray:
    """Initial populations (u = 0, p = 0) for order parameter c0 and
    temperature T0 (both (ny, nx)); Tbot/Ttop are the wall temperatures (nx)."""
    c0 = np.asarray(c0)
    ny, nx = c0.shape
    c0 = _f64(c0, (ny, nx))
    T0 = _f64(T0, (ny, nx))
    Tb = _f64(Tbot, (nx,))
    Tt = _f64(Ttop, (nx,))
    pop = np.empty((27, ny, nx), dtype=np.float64)
    rc = lib().orc_init(ctypes.byref(_p(params, nx, ny)), _d(c0), _d(T0), _d(Tb),
                        _d(Tt), _d(pop))
    if rc != 0:
        raise ValueError("oracle init rejected the parameters (rc=%d)" % rc)
    return pop


def run(params: dict, pop, Tbot, Ttop, nsteps: int) -> np.ndarray:
    """Advance a population state by ``nsteps`` time steps."""
    pop = _f64(pop, np.shape(pop))
    _, ny, nx = pop.shape
    Tb = _f64(Tbot, (nx,))
    Tt = _f64(Ttop, (nx,))
    out = np.empty_like(pop)
    rc = lib().orc_run(ctypes.byref(_p(params, nx, ny)), _d(Tb), _d(Tt), _d(pop),
                       _d(out), int(nsteps))
    if rc != 0:
        raise ValueError("oracle run failed (rc=%d)" % rc)
    return out


def fields(params: dict, pop, Tbot, Ttop) -> dict:
    """Macroscopic c, p, ux, uy, T of a population state (each (ny, nx))."""
    pop = _f64(pop, np.shape(pop))
    _, ny, nx = pop.shape
    Tb = _f64(Tbot, (nx,))
    Tt = _f64(Ttop, (nx,))
    out = {k: np.empty((ny, nx)) for k in ("c", "p", "ux", "uy", "T")}
    lib().orc_fields(ctypes.byref(_p(params, nx, ny)), _d(Tb), _d(Tt), _d(pop),
                     _d(out["c"]), _d(out["p"]), _d(out["ux"]), _d(out["uy"]),
                     _d(out["T"]))
    return out


SCALAR_KEYS = ("gcx", "gcy", "lapc", "kappa", "gTx", "gTy", "gpx", "gpy", "mu",
               "Fx", "Fy")


def scalar_ops(params: dict, c, p, T, Tbot, Ttop) -> dict:
    """Stencil stage of the step from cell values of c, p and T: gradients,
    Laplacian, curvature, chemical potential and force at every cell."""
    c = np.asarray(c)
    ny, nx = c.shape
    c = _f64(c, (ny, nx))
    p = _f64(p, (ny, nx))
    T = _f64(T, (ny, nx))
    Tb = _f64(Tbot, (nx,))
    Tt = _f64(Ttop, (nx,))
    out = {k: np.empty((ny, nx)) for k in SCALAR_KEYS}
    lib().orc_scalar_ops(ctypes.byref(_p(params, nx, ny)), _d(Tb), _d(Tt), _d(c),
                         _d(p), _d(T), *[_d(out[k]) for k in SCALAR_KEYS])
    return out


def cell_terms(params: dict, c, p, T, mu, ux, uy, Fx, Fy, gpx, gpy) -> dict:
    """Equilibria and collision sources of one cell (9 values each)."""
    arrs = {k: np.zeros(9) for k in ("feq", "geq", "heq", "fsrc", "gsrc", "hsrc")}
    lib().orc_cell_terms(ctypes.byref(_p(params, 1, 2)), c, p, T, mu, ux, uy, Fx,
                         Fy, gpx, gpy, *[_d(arrs[k]) for k in
                                         ("feq", "geq", "heq", "fsrc", "gsrc", "hsrc")])
    return arrs


# ---------------------------------------------------------------- migration
def centroid_velocity(params: dict, pop, Tbot, Ttop) -> float:
    """Phase-1 centroid velocity of a state: sum c u_y / sum c over the cells
    (the migration velocity of the drop, Sec. IV.C; c is the drop's order
    parameter, u the velocity of Eq. 13 with the half-step force)."""
    F = fields(params, pop, Tbot, Ttop)
    return float((F["c"] * F["uy"]).sum() / F["c"].sum())


def migration_loss(params: dict, c0, T0, Tbot, Ttop, steps: int, window: int) -> float:
    """Mean centroid velocity over the states n = steps-window+1 .. steps of
    the run that starts from the rest state of (c0, T0)."""
    if not 1 <= window <= steps:
        raise ValueError("window must be in [1, steps]")
    pop = init(params, c0, T0, Tbot, Ttop)
    pop = run(params, pop, Tbot, Ttop, steps - window)
    total = 0.0
    for _ in range(window):
        pop = run(params, pop, Tbot, Ttop, 1)
        total += centroid_velocity(params, pop, Tbot, Ttop)
    return total / window


def migration_centroid(params: dict, pop, Tbot, Ttop) -> float:
    """Phase-1 centroid height sum c y / sum c (cell centres y = 0..ny-1)."""
    F = fields(params, pop, Tbot, Ttop)
    y = np.arange(F["c"].shape[0], dtype=np.float64)[:, None]
    return float((F["c"] * y).sum() / F["c"].sum())
