"""ctypes binding of the C ABI in include/cdbm.h (argument marshalling only).

Every function here has the name of the C entry point it calls; all arithmetic
runs in the CUDA library ``_build/libcdbm.so``.  There is no CPU fallback:
loading fails loudly when the library has not been built.

``Solver`` wraps one context with PyTorch supplying device memory (through the
caching allocator, passed to ``cdbm_create`` as callbacks) and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

CDBM_OK, CDBM_EINVAL, CDBM_ESINGULAR, CDBM_ENOMEM, CDBM_ECUDA, CDBM_ENONPHYS, CDBM_ETIMEOUT = range(7)
STATUS_NAMES = {0: "CDBM_OK", 1: "CDBM_EINVAL", 2: "CDBM_ESINGULAR", 3: "CDBM_ENOMEM",
                4: "CDBM_ECUDA", 5: "CDBM_ENONPHYS", 6: "CDBM_ETIMEOUT"}
CDBM_BC_PERIODIC, CDBM_BC_ZEROGRAD = 0, 1
CDBM_FP64, CDBM_FP32_BULK, CDBM_FP32_DF64, CDBM_FP32_DEV = 0, 1, 2, 3
CDBM_ADJ_LIMITER_EXACT, CDBM_ADJ_LIMITER_FROZEN_RATIO, CDBM_ADJ_LIMITER_FROZEN = 0, 1, 2
CDBM_RK2_TVD, CDBM_RK2_MIDPOINT = 0, 1

#: every entry point declared in include/cdbm.h
EXPORTS = ("cdbm_create", "cdbm_set_rk", "cdbm_init", "cdbm_step", "cdbm_set_small_grid_path",
           "cdbm_set_row_marching", "cdbm_macros", "cdbm_tne", "cdbm_conserved_sums", "cdbm_get_state", "cdbm_set_state", "cdbm_state_ptr", "cdbm_time",
           "cdbm_sync", "cdbm_last_error", "cdbm_destroy", "cdbm_step_noalloc",
           "cdbm_batch_create", "cdbm_batch_init", "cdbm_batch_step", "cdbm_batch_autotune",
           "cdbm_batch_set_tile", "cdbm_batch_set_symmetric", "cdbm_batch_macros", "cdbm_batch_info", "cdbm_batch_sync",
           "cdbm_batch_last_error", "cdbm_batch_destroy", "cdbm_adjoint_forward",
           "cdbm_adjoint_backward", "cdbm_adjoint_set_limiter", "cdbm_macros_vjp",
           "cdbm_diag_rcp64", "cdbm_diag_fp64_fma")
CDBM_NOALLOC_MAX_CELLS = 32768


class cdbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int)]


class cdbm_vset(ctypes.Structure):
    _fields_ = [("v", ctypes.c_double * 4), ("eta", ctypes.c_double * 4)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class cdbm_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class CdbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Loads libcdbm.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing: build it with __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    ctx = ctypes.c_void_p
    sig = {
        "cdbm_create": ([ctypes.POINTER(cdbm_grid), ctypes.POINTER(cdbm_vset), ctypes.c_double,
                         ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp,
                         ctypes.POINTER(cdbm_allocator), ctypes.POINTER(ctx)], ctypes.c_int),
        "cdbm_set_rk": ([ctx, ctypes.c_int], ctypes.c_int),
        "cdbm_init": ([ctx, _vp, _vp, _vp, _vp], ctypes.c_int),
        "cdbm_step": ([ctx, ctypes.c_int], ctypes.c_int),
        "cdbm_set_small_grid_path": ([ctx, ctypes.c_int], ctypes.c_int),
        "cdbm_set_row_marching": ([ctx, ctypes.c_int], ctypes.c_int),
        "cdbm_macros": ([ctx, _vp, _vp, _vp, _vp], ctypes.c_int),
        "cdbm_tne": ([ctx, _vp], ctypes.c_int),
        "cdbm_conserved_sums": ([ctx, _dp], ctypes.c_int),
        "cdbm_get_state": ([ctx, _vp, _dp], ctypes.c_int),
        "cdbm_set_state": ([ctx, _vp, ctypes.c_double], ctypes.c_int),
        "cdbm_state_ptr": ([ctx, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "cdbm_time": ([ctx, _dp], ctypes.c_int),
        "cdbm_sync": ([ctx], ctypes.c_int),
        "cdbm_last_error": ([ctx], ctypes.c_char_p),
        "cdbm_destroy": ([ctx], None),
        "cdbm_step_noalloc": ([ctypes.POINTER(cdbm_grid), ctypes.POINTER(cdbm_vset), ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, _vp, ctypes.c_int, _vp], ctypes.c_int),
        "cdbm_batch_create": ([ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(cdbm_vset), ctypes.c_double,
                               ctypes.c_double, ctypes.c_int, _vp, ctypes.POINTER(cdbm_allocator),
                               ctypes.POINTER(ctx)], ctypes.c_int),
        "cdbm_batch_init": ([ctx, _vp, _vp, _vp, _vp], ctypes.c_int),
        "cdbm_batch_step": ([ctx, ctypes.c_int], ctypes.c_int),
        "cdbm_batch_autotune": ([ctx, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cdbm_batch_set_tile": ([ctx, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "cdbm_batch_set_symmetric": ([ctx, ctypes.c_int], ctypes.c_int),
        "cdbm_batch_macros": ([ctx, _vp, _vp, _vp, _vp], ctypes.c_int),
        "cdbm_batch_info": ([ctx, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cdbm_batch_sync": ([ctx], ctypes.c_int),
        "cdbm_batch_last_error": ([ctx], ctypes.c_char_p),
        "cdbm_batch_destroy": ([ctx], None),
        "cdbm_adjoint_forward": ([ctx, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "cdbm_adjoint_backward": ([ctx, _vp, _vp, _vp, _vp, _vp, _dp], ctypes.c_int),
        "cdbm_adjoint_set_limiter": ([ctx, ctypes.c_int], ctypes.c_int),
        "cdbm_macros_vjp": ([ctx, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "cdbm_diag_rcp64": ([_vp, _vp, ctypes.c_longlong, _vp], ctypes.c_int),
        "cdbm_diag_fp64_fma": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _dp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(lib, ctx, status):
    if status != CDBM_OK:
        raise CdbmError(status, lib.cdbm_last_error(ctx).decode())


# ---- thin wrappers with the C names (pointers are ints / ctypes values) ----

def cdbm_create(grid: cdbm_grid, vset: cdbm_vset, I, tau, dt, precision=CDBM_FP64, stream=0,
                allocator: cdbm_allocator | None = None):
    lib = load()
    out = ctypes.c_void_p()
    st = lib.cdbm_create(ctypes.byref(grid), ctypes.byref(vset), float(I), float(tau), float(dt),
                         int(precision), ctypes.c_void_p(stream),
                         ctypes.byref(allocator) if allocator is not None else None, ctypes.byref(out))
    _check(lib, None, st)
    return out


def cdbm_set_rk(ctx, rk):
    lib = load()
    _check(lib, ctx, lib.cdbm_set_rk(ctx, int(rk)))


def cdbm_init(ctx, rho, ux, uy, T):
    lib = load()
    _check(lib, ctx, lib.cdbm_init(ctx, rho, ux, uy, T))


def cdbm_step(ctx, nsteps):
    lib = load()
    _check(lib, ctx, lib.cdbm_step(ctx, int(nsteps)))


def cdbm_set_small_grid_path(ctx, enable):
    lib = load()
    _check(lib, ctx, lib.cdbm_set_small_grid_path(ctx, int(bool(enable))))


def cdbm_set_row_marching(ctx, enable):
    lib = load()
    _check(lib, ctx, lib.cdbm_set_row_marching(ctx, int(bool(enable))))


def cdbm_macros(ctx, rho, ux, uy, T):
    lib = load()
    _check(lib, ctx, lib.cdbm_macros(ctx, rho, ux, uy, T))


def cdbm_tne(ctx, out):
    lib = load()
    _check(lib, ctx, lib.cdbm_tne(ctx, out))


def cdbm_conserved_sums(ctx):
    lib = load()
    out = (ctypes.c_double * 4)()
    _check(lib, ctx, lib.cdbm_conserved_sums(ctx, out))
    return np.array(out[:])


def cdbm_get_state(ctx, f):
    lib = load()
    t = ctypes.c_double()
    _check(lib, ctx, lib.cdbm_get_state(ctx, f, ctypes.byref(t)))
    return t.value


def cdbm_set_state(ctx, f, t):
    lib = load()
    _check(lib, ctx, lib.cdbm_set_state(ctx, f, float(t)))


def cdbm_state_ptr(ctx) -> int:
    lib = load()
    p = ctypes.c_void_p()
    _check(lib, ctx, lib.cdbm_state_ptr(ctx, ctypes.byref(p)))
    return p.value


def cdbm_time(ctx) -> float:
    lib = load()
    t = ctypes.c_double()
    _check(lib, ctx, lib.cdbm_time(ctx, ctypes.byref(t)))
    return t.value


def cdbm_sync(ctx):
    lib = load()
    _check(lib, ctx, lib.cdbm_sync(ctx))


def cdbm_last_error(ctx) -> str:
    return load().cdbm_last_error(ctx).decode()


def cdbm_destroy(ctx):
    load().cdbm_destroy(ctx)


def cdbm_step_noalloc(grid: cdbm_grid, vset: cdbm_vset, I, tau, dt, f, nsteps, stream=0):
    """Advances the caller's device state f ([16][ny][nx], address as int) in place
    without any allocation; see include/cdbm.h."""
    lib = load()
    st = lib.cdbm_step_noalloc(ctypes.byref(grid), ctypes.byref(vset), float(I), float(tau),
                               float(dt), ctypes.c_void_p(f), int(nsteps), ctypes.c_void_p(stream))
    _check(lib, None, st)


def cdbm_adjoint_forward(ctx, nsteps, every):
    lib = load()
    _check(lib, ctx, lib.cdbm_adjoint_forward(ctx, int(nsteps), int(every)))


def cdbm_adjoint_backward(ctx, fbar, grad_rho=0, grad_ux=0, grad_uy=0, grad_T=0):
    """Device addresses in, dL/dtau out (float)."""
    lib = load()
    gt = ctypes.c_double()
    _check(lib, ctx, lib.cdbm_adjoint_backward(ctx, fbar, grad_rho or None, grad_ux or None, grad_uy or None,
                                               grad_T or None, ctypes.byref(gt)))
    return gt.value


def cdbm_adjoint_set_limiter(ctx, mode):
    lib = load()
    _check(lib, ctx, lib.cdbm_adjoint_set_limiter(ctx, int(mode)))


def cdbm_macros_vjp(ctx, rho_bar, ux_bar, uy_bar, T_bar, fbar):
    lib = load()
    _check(lib, ctx, lib.cdbm_macros_vjp(ctx, rho_bar or None, ux_bar or None, uy_bar or None, T_bar or None,
                                         fbar))


def cdbm_diag_rcp64(x, y, n, stream=0):
    """y = 1 / x (device addresses, n doubles) by the kernels' reciprocal."""
    lib = load()
    _check(lib, None, lib.cdbm_diag_rcp64(ctypes.c_void_p(x), ctypes.c_void_p(y), int(n),
                                          ctypes.c_void_p(stream)))


def cdbm_diag_fp64_fma(out, blocks, threads, iters, stream=0) -> float:
    """Launches the FP64 FMA probe (out: device address of blocks * threads doubles);
    returns its flop count."""
    lib = load()
    fl = ctypes.c_double()
    _check(lib, None, lib.cdbm_diag_fp64_fma(ctypes.c_void_p(out), int(blocks), int(threads), int(iters),
                                             ctypes.c_void_p(stream), ctypes.byref(fl)))
    return fl.value


def _bcheck(lib, b, status):
    if status != CDBM_OK:
        raise CdbmError(status, lib.cdbm_batch_last_error(b).decode())


def cdbm_batch_create(nx, dx, I, vset: cdbm_vset, tau, dt, precision=CDBM_FP64, stream=0,
                      allocator: cdbm_allocator | None = None):
    lib = load()
    n = len(nx)
    nx_a = np.ascontiguousarray(nx, dtype=np.int32)
    dx_a = np.ascontiguousarray(dx, dtype=np.float64)
    I_a = np.ascontiguousarray(I, dtype=np.float64)
    out = ctypes.c_void_p()
    st = lib.cdbm_batch_create(n, nx_a.ctypes.data, dx_a.ctypes.data, I_a.ctypes.data, ctypes.byref(vset),
                               float(tau), float(dt), int(precision), ctypes.c_void_p(stream),
                               ctypes.byref(allocator) if allocator is not None else None, ctypes.byref(out))
    _bcheck(lib, None, st)
    return out


def cdbm_batch_init(b, rho, ux, uy, T):
    lib = load()
    _bcheck(lib, b, lib.cdbm_batch_init(b, rho, ux, uy, T))


def cdbm_batch_step(b, nsteps):
    lib = load()
    _bcheck(lib, b, lib.cdbm_batch_step(b, int(nsteps)))


def cdbm_batch_autotune(b, trial_steps):
    lib = load()
    t, k = ctypes.c_int(), ctypes.c_int()
    _bcheck(lib, b, lib.cdbm_batch_autotune(b, int(trial_steps), ctypes.byref(t), ctypes.byref(k)))
    return t.value, k.value


def cdbm_batch_set_tile(b, threads, blocks_per_sm):
    lib = load()
    _bcheck(lib, b, lib.cdbm_batch_set_tile(b, int(threads), int(blocks_per_sm)))


def cdbm_batch_set_symmetric(b, enable):
    lib = load()
    _bcheck(lib, b, lib.cdbm_batch_set_symmetric(b, int(bool(enable))))


def cdbm_batch_macros(b, rho, ux, uy, T):
    lib = load()
    _bcheck(lib, b, lib.cdbm_batch_macros(b, rho, ux, uy, T))


def cdbm_batch_info(b):
    lib = load()
    n, t, k = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
    _bcheck(lib, b, lib.cdbm_batch_info(b, ctypes.byref(n), ctypes.byref(t), ctypes.byref(k)))
    return n.value, t.value, k.value


def cdbm_batch_sync(b):
    lib = load()
    _bcheck(lib, b, lib.cdbm_batch_sync(b))


def cdbm_batch_last_error(b) -> str:
    return load().cdbm_batch_last_error(b).decode()


def cdbm_batch_destroy(b):
    load().cdbm_batch_destroy(b)


# ------------------------------------------------------------------ Solver

def _ptr(x):
    """Device or host address of a torch tensor / numpy array (float64, contiguous)."""
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"], "need contiguous float64"
        return x.ctypes.data
    assert x.dtype.is_floating_point and x.element_size() == 8 and x.is_contiguous(), \
        "need a contiguous float64 tensor"
    return x.data_ptr()


class Solver:
    """One CDBM run on the current CUDA device.

    Parameters follow ``cdbm_create``: grid size and spacing, boundary kinds,
    relaxation time ``tau``, time step ``dt``, extra degrees of freedom ``I`` and
    the velocity set ``vg`` = (v_a..v_d), ``eg`` = (eta_a..eta_d) of Eqs. (2)-(3).
    Work runs on ``stream`` (a torch.cuda.Stream; default: the current stream).
    """

    def __init__(self, nx, ny, dx, dy, dt, tau, I, vg, eg, bc_x=CDBM_BC_PERIODIC,
                 bc_y=CDBM_BC_PERIODIC, precision=CDBM_FP64, rk=CDBM_RK2_TVD, stream=None):
        import torch
        self._torch = torch
        self.nx, self.ny = int(nx), int(ny)
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        dev = self.device

        def _alloc(nbytes, strm, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm or 0)
            except Exception:      # reported to the library as NULL -> CDBM_ENOMEM
                return None

        def _free(ptr, nbytes, strm, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        self._allocator = cdbm_allocator(self._alloc_cb, self._free_cb, None)
        grid = cdbm_grid(self.nx, self.ny, float(dx), float(dy), int(bc_x), int(bc_y))
        vset = cdbm_vset((ctypes.c_double * 4)(*vg), (ctypes.c_double * 4)(*eg))
        self.ctx = cdbm_create(grid, vset, I, tau, dt, precision, self.stream.cuda_stream,
                               self._allocator)
        if rk != CDBM_RK2_TVD:
            cdbm_set_rk(self.ctx, rk)

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.I, w.vg, w.eg, w.bc_x, w.bc_y, **kw)

    # -- fields -------------------------------------------------------------
    def _field(self, a):
        torch = self._torch
        if isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
            a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64),
                                                     (self.ny, self.nx)))
            return a, a.ctypes.data
        a = a.to(torch.float64).contiguous()
        return a, a.data_ptr()

    def init(self, rho, ux, uy, T):
        keep = [self._field(a) for a in (rho, ux, uy, T)]
        cdbm_init(self.ctx, *(p for _, p in keep))
        for a, _ in keep:
            if hasattr(a, "record_stream"):
                a.record_stream(self.stream)

    def step(self, nsteps=1):
        cdbm_step(self.ctx, nsteps)

    def macros(self):
        """(rho, ux, uy, T) as new [ny][nx] float64 CUDA tensors."""
        torch = self._torch
        out = [torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
               for _ in range(4)]
        cdbm_macros(self.ctx, *(t.data_ptr() for t in out))
        return tuple(out)

    def tne(self):
        torch = self._torch
        out = torch.empty((12, self.ny, self.nx), dtype=torch.float64, device=self.device)
        cdbm_tne(self.ctx, out.data_ptr())
        return out

    def conserved_sums(self):
        return cdbm_conserved_sums(self.ctx)

    def state(self):
        torch = self._torch
        out = torch.empty((16, self.ny, self.nx), dtype=torch.float64, device=self.device)
        cdbm_get_state(self.ctx, out.data_ptr())
        return out

    def set_state(self, f, t=0.0):
        a, p = (f, _ptr(f)) if isinstance(f, np.ndarray) else (f.contiguous(), None)
        cdbm_set_state(self.ctx, p if p is not None else a.data_ptr(), t)

    @property
    def time(self):
        return cdbm_time(self.ctx)

    def sync(self):
        cdbm_sync(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            cdbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """An ensemble of independent 1-D tubes advanced by one persistent kernel
    (cdbm_batch_*).  ``tubes`` is a list of workloads with ny == 1 sharing the
    velocity set, tau and dt (for example ``workloads.ensemble_tube``)."""

    def __init__(self, tubes, precision=CDBM_FP64, stream=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        w0 = tubes[0]
        for w in tubes:
            assert w.ny == 1 and w.vg == w0.vg and w.eg == w0.eg and w.dt == w0.dt and w.tau == w0.tau
        self.nx = [w.nx for w in tubes]
        self.offsets = np.concatenate([[0], np.cumsum(self.nx)])
        dev = self.device

        def _alloc(nbytes, strm, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm or 0)
            except Exception:
                return None

        def _free(ptr, nbytes, strm, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        self._allocator = cdbm_allocator(self._alloc_cb, self._free_cb, None)
        vset = cdbm_vset((ctypes.c_double * 4)(*w0.vg), (ctypes.c_double * 4)(*w0.eg))
        self.b = cdbm_batch_create(self.nx, [w.dx for w in tubes], [w.I for w in tubes], vset, w0.tau,
                                   w0.dt, precision, self.stream.cuda_stream, self._allocator)
        self.total = int(self.offsets[-1])

    def init(self, tubes):
        fields = [np.ascontiguousarray(np.concatenate([getattr(w, k).reshape(-1) for w in tubes]))
                  for k in ("rho", "ux", "uy", "T")]
        cdbm_batch_init(self.b, *(a.ctypes.data for a in fields))

    def step(self, nsteps=1):
        cdbm_batch_step(self.b, nsteps)

    def autotune(self, trial_steps=5):
        return cdbm_batch_autotune(self.b, trial_steps)

    def set_tile(self, threads, blocks_per_sm):
        cdbm_batch_set_tile(self.b, threads, blocks_per_sm)

    def set_symmetric(self, enable):
        cdbm_batch_set_symmetric(self.b, enable)

    def macros(self):
        """(rho, ux, uy, T) as concatenated float64 numpy arrays."""
        out = [np.zeros(self.total) for _ in range(4)]
        cdbm_batch_macros(self.b, *(a.ctypes.data for a in out))
        return tuple(out)

    def tube(self, arrays, t):
        lo, hi = self.offsets[t], self.offsets[t + 1]
        return tuple(a[lo:hi] for a in arrays)

    def info(self):
        return cdbm_batch_info(self.b)

    def sync(self):
        cdbm_batch_sync(self.b)

    def close(self):
        if getattr(self, "b", None):
            cdbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_run_function():
    """torch.autograd.Function over a whole CDBM run (built lazily so that importing
    this module does not import torch)."""
    import torch

    class CDBMRun(torch.autograd.Function):
        """(rho, u_x, u_y, T) at the end of `nsteps` steps from initial fields
        (rho0, ux0, uy0, T0) and relaxation time tau; `spec` holds the remaining run
        parameters (nx, ny, dx, dy, dt, I, vg, eg; periodic axes; optional
        limiter, a CDBM_ADJ_LIMITER_* mode of cdbm_adjoint_set_limiter).  The
        backward pass runs the adjoint kernels with a checkpoint every `every`
        steps."""

        @staticmethod
        def forward(ctx, rho0, ux0, uy0, T0, tau, spec, nsteps, every):
            s = Solver(spec["nx"], spec["ny"], spec["dx"], spec["dy"], spec["dt"], float(tau), spec["I"],
                       spec["vg"], spec["eg"])
            s.init(rho0.detach(), ux0.detach(), uy0.detach(), T0.detach())
            if spec.get("limiter", CDBM_ADJ_LIMITER_EXACT) != CDBM_ADJ_LIMITER_EXACT:
                cdbm_adjoint_set_limiter(s.ctx, spec["limiter"])
            cdbm_adjoint_forward(s.ctx, nsteps, every)
            out = s.macros()
            ctx.solver = s
            ctx.tau_like = tau
            return out

        @staticmethod
        def backward(ctx, grho, gux, guy, gT):
            s = ctx.solver
            dev = s.device
            ptr = lambda g: g.contiguous().data_ptr() if g is not None else 0
            keep = [g.contiguous() if g is not None else None for g in (grho, gux, guy, gT)]
            fbar = torch.empty((16, s.ny, s.nx), dtype=torch.float64, device=dev)
            cdbm_macros_vjp(s.ctx, *(ptr(g) for g in keep), fbar.data_ptr())
            grads = [torch.empty((s.ny, s.nx), dtype=torch.float64, device=dev) for _ in range(4)]
            gtau = cdbm_adjoint_backward(s.ctx, fbar.data_ptr(), *(g.data_ptr() for g in grads))
            s.close()
            tau = ctx.tau_like
            gtau_t = torch.tensor(gtau, dtype=tau.dtype, device=tau.device) if torch.is_tensor(tau) else None
            return grads[0], grads[1], grads[2], grads[3], gtau_t, None, None, None

    return CDBMRun
