"""CDBM oracle: TEST INFRASTRUCTURE ONLY.

A plain double-precision CPU statement of the central-moment discrete Boltzmann
method (Sec. 2, Eqs. 1-20 of Lin, Su, Fei and Luo), used to check the CUDA
library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code, table or constant with the CUDA
library (``paper_2502_16818_gb300``), and neither imports the other.

The arithmetic lives in ``cdbm_oracle.c`` (compiled with gcc, OpenMP over cells);
this module only builds it and marshals numpy arrays through ctypes.

Every function is pinned by ``tests/test_oracle_pins.py`` against quantities the
paper or the mathematics fixes (Gauss-Hermite moments of Eq. 5, exact
conservation, the exact Riemann solution, the sound speed sqrt(gamma T), the
Taylor-Green decay rate, the Chapman-Enskog stress of Eq. 21, brute force on
hand-built cases).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (OpenMP when available). Returns the path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
            "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("rk", ctypes.c_int), ("threads", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dt", ctypes.c_double),
        ("tau", ctypes.c_double), ("I", ctypes.c_double),
        ("vg", ctypes.c_double * 4), ("eg", ctypes.c_double * 4),
    ]


def _configure(lib):
    P = ctypes.POINTER(_Params)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_velocity_set.argtypes = [dp, dp, dp, dp, dp]
    lib.orc_central_matrix.argtypes = [dp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
    lib.orc_central_moments_eq.argtypes = [ctypes.c_double] * 3 + [dp]
    lib.orc_solve.argtypes = [ctypes.c_int, dp, dp, dp]
    lib.orc_feq.argtypes = [P] + [ctypes.c_double] * 4 + [dp]
    lib.orc_cell_macros.argtypes = [P, dp, dp, dp, dp, dp]
    lib.orc_minmod.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.orc_minmod.restype = ctypes.c_double
    lib.orc_nnd_derivative.argtypes = [ctypes.c_double, dp, ctypes.c_double]
    lib.orc_nnd_derivative.restype = ctypes.c_double
    lib.orc_init.argtypes = [P, dp, dp, dp, dp, dp]
    lib.orc_step.argtypes = [P, dp, ctypes.c_int]
    lib.orc_macros.argtypes = [P, dp, dp, dp, dp, dp]
    lib.orc_tne.argtypes = [P, dp, dp]
    lib.orc_conserved_sums.argtypes = [P, dp, dp]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


class use_library:
    """Context manager that routes this module through another build of the oracle
    source (used by the tests that plant mistakes in a copy of it)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def compile_variant(source_text: str, out_path: str) -> str:
    """Compiles C source text with the oracle's flags into out_path (a .so)."""
    src = out_path[:-3] + ".c"
    with open(src, "w") as fh:
        fh.write(source_text)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
            src, "-o", out_path, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return out_path


def source() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(x, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = np.ascontiguousarray(np.broadcast_to(a, shape))
    return a


@dataclass
class Model:
    """Grid, velocity set and parameters of one CDBM run (Eqs. 1-3, Sec. 3)."""
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    tau: float
    I: float
    vg: tuple
    eg: tuple
    bc_x: int = 0          # 0 periodic, 1 zero-gradient
    bc_y: int = 0
    rk: int = 0            # 0 two-stage TVD Runge-Kutta, 1 midpoint
    threads: int = 0

    def c(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.bc_x, p.bc_y, p.rk, p.threads = self.nx, self.ny, self.bc_x, self.bc_y, self.rk, self.threads
        p.dx, p.dy, p.dt, p.tau, p.I = self.dx, self.dy, self.dt, self.tau, self.I
        p.vg[:] = list(self.vg)
        p.eg[:] = list(self.eg)
        return p


def velocity_set(vg, eg):
    """Returns (vx, vy, eta), each of length 16, per Eqs. (2)-(3)."""
    lib = _load()
    vg, eg = _arr(vg), _arr(eg)
    vx, vy, et = np.zeros(16), np.zeros(16), np.zeros(16)
    lib.orc_velocity_set(_ptr(vg), _ptr(eg), _ptr(vx), _ptr(vy), _ptr(et))
    return vx, vy, et


def central_matrix(vx, vy, eta, ux, uy) -> np.ndarray:
    """The 16x16 matrix M(u) of Eq. (6)."""
    lib = _load()
    vx, vy, eta = _arr(vx), _arr(vy), _arr(eta)
    M = np.zeros((16, 16))
    lib.orc_central_matrix(_ptr(vx), _ptr(vy), _ptr(eta), ux, uy, _ptr(M))
    return M


def central_moments_eq(I, rho, T) -> np.ndarray:
    """fbar_eq: central moments of the Maxwellian of Eq. (5) in the rows of Eq. (6)."""
    lib = _load()
    out = np.zeros(16)
    lib.orc_central_moments_eq(I, rho, T, _ptr(out))
    return out


def solve(A, b) -> np.ndarray:
    lib = _load()
    A, b = _arr(A), _arr(b)
    n = b.shape[0]
    x = np.zeros(n)
    if lib.orc_solve(n, _ptr(A), _ptr(b), _ptr(x)) != 0:
        raise np.linalg.LinAlgError("oracle solve: zero pivot")
    return x


def feq(m: Model, rho, ux, uy, T) -> np.ndarray:
    """f_eq = M(u)^-1 fbar_eq (Eq. 7) for one cell."""
    lib = _load()
    out = np.zeros(16)
    pc = m.c()
    if lib.orc_feq(ctypes.byref(pc), rho, ux, uy, T, _ptr(out)) != 0:
        raise np.linalg.LinAlgError("oracle feq: singular moment matrix")
    return out


def cell_macros(m: Model, f16):
    lib = _load()
    f16 = _arr(f16)
    r, u, v, T = (ctypes.c_double() for _ in range(4))
    pc = m.c()
    lib.orc_cell_macros(ctypes.byref(pc), _ptr(f16), ctypes.byref(r), ctypes.byref(u),
                        ctypes.byref(v), ctypes.byref(T))
    return r.value, u.value, v.value, T.value


def minmod(X, Y) -> float:
    return _load().orc_minmod(X, Y)


def nnd_derivative(v, fs5, dr) -> float:
    """v df/dr at the middle of five samples, Eqs. (12)-(20)."""
    fs5 = _arr(fs5)
    return _load().orc_nnd_derivative(v, _ptr(fs5), dr)


def init(m: Model, rho, ux, uy, T) -> np.ndarray:
    """f[16][ny][nx] = f_eq of the given fields (each broadcast to [ny][nx])."""
    lib = _load()
    shp = (m.ny, m.nx)
    rho, ux, uy, T = (_arr(a, shp) for a in (rho, ux, uy, T))
    f = np.zeros((16, m.ny, m.nx))
    pc = m.c()
    bad = lib.orc_init(ctypes.byref(pc), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T), _ptr(f))
    if bad:
        raise np.linalg.LinAlgError("oracle init: %d singular cells" % bad)
    return f


def step(m: Model, f: np.ndarray, nsteps: int) -> np.ndarray:
    """Returns f advanced by nsteps Runge-Kutta steps (the input is not modified)."""
    lib = _load()
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    assert g.shape == (16, m.ny, m.nx)
    pc = m.c()
    bad = lib.orc_step(ctypes.byref(pc), _ptr(g), int(nsteps))
    if bad:
        raise RuntimeError("oracle step failed (%d)" % bad)
    return g


def macros(m: Model, f: np.ndarray):
    """(rho, ux, uy, T), each [ny][nx]."""
    lib = _load()
    f = _arr(f)
    out = [np.zeros((m.ny, m.nx)) for _ in range(4)]
    pc = m.c()
    lib.orc_macros(ctypes.byref(pc), _ptr(f), *(_ptr(a) for a in out))
    return tuple(out)


def tne(m: Model, f: np.ndarray) -> np.ndarray:
    """Delta* (Eqs. 8-11) as [12][ny][nx] in the order of rows 5..16 of Eq. (6)."""
    lib = _load()
    f = _arr(f)
    out = np.zeros((12, m.ny, m.nx))
    pc = m.c()
    if lib.orc_tne(ctypes.byref(pc), _ptr(f), _ptr(out)):
        raise np.linalg.LinAlgError("oracle tne: singular cells")
    return out


def conserved_sums(m: Model, f: np.ndarray) -> np.ndarray:
    lib = _load()
    f = _arr(f)
    out = np.zeros(4)
    pc = m.c()
    lib.orc_conserved_sums(ctypes.byref(pc), _ptr(f), _ptr(out))
    return out
