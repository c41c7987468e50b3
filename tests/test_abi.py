"""C-ABI checks that need no GPU: the library builds, loads and exports every entry
point include/cdbm.h declares, and cdbm_create rejects bad runs (validation and the
moment-matrix check happen on the host before any CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_2502_16818_gb300 import _build, cdbm, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return cdbm.load()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "cdbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cdbm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_binding_exports():
    assert header_symbols() == sorted(cdbm.EXPORTS)


def test_library_exports_every_header_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    # cdbm_grid: int, int, double, double, int, int -> 8 + 16 + 8 = 32 bytes on LP64
    assert ctypes.sizeof(cdbm.cdbm_grid) == 32
    assert ctypes.sizeof(cdbm.cdbm_vset) == 64


def _create(vg=W.VSET_SOD[0], eg=W.VSET_SOD[1], nx=10, ny=1, dx=0.01, dy=0.01, dt=1e-4, tau=1e-4,
            I=0.0, bc=(1, 0), precision=0):
    grid = cdbm.cdbm_grid(nx, ny, dx, dy, bc[0], bc[1])
    vset = cdbm.cdbm_vset((ctypes.c_double * 4)(*vg), (ctypes.c_double * 4)(*eg))
    out = ctypes.c_void_p(123)
    lib = cdbm.load()
    st = lib.cdbm_create(ctypes.byref(grid), ctypes.byref(vset), I, tau, dt, precision, None, None,
                         ctypes.byref(out))
    return st, out.value, lib.cdbm_last_error(None).decode()


@pytest.mark.parametrize("kw,needle", [
    (dict(nx=0), "grid"),
    (dict(ny=-1), "grid"),
    (dict(dx=0.0), "dx"),
    (dict(dt=-1e-5), "dx"),
    (dict(tau=float("nan")), "dx"),
    (dict(I=-1.0), "I must"),
    (dict(dt=3e-4, tau=1e-4, dx=1.0), "dt/tau"),
    (dict(dt=5e-3, tau=1e-2, dx=0.01), "CFL"),
    (dict(bc=(2, 0)), "boundary"),
    (dict(precision=7), "precision"),
    (dict(vg=(2.5, -1.0, 1.2, 1.1)), "velocity set"),
])
def test_create_rejects_invalid(lib, kw, needle):
    st, out, msg = _create(**kw)
    assert st == cdbm.CDBM_EINVAL and out is None
    assert needle in msg


@pytest.mark.parametrize("vg,eg", [
    ((2.5, 2.5, 1.2, 1.1), (0.0, 0.0, 0.0, 0.0)),   # no eta: the vector block is singular
    ((1.0, 2.0, 1.5, 2.0), (0.5, 1.0, 0.2, 1.0)),   # 2 v_b^2 + eta_b^2 = 2 v_d^2 + eta_d^2
    ((1.0, 2.0, 1.0, 1.5), (0.7, 1.0, 0.7, 0.3)),   # v_a^2 + eta_a^2 = v_c^2 + eta_c^2
])
def test_create_rejects_singular_velocity_sets(lib, vg, eg):
    st, out, msg = _create(vg=vg, eg=eg)
    assert st == cdbm.CDBM_ESINGULAR and out is None
    assert "singular" in msg


def test_null_arguments(lib):
    lib_ = cdbm.load()
    assert lib_.cdbm_create(None, None, 0.0, 1.0, 1.0, 0, None, None, None) == cdbm.CDBM_EINVAL
    assert lib_.cdbm_step(None, 1) == cdbm.CDBM_EINVAL
    assert lib_.cdbm_sync(None) == cdbm.CDBM_EINVAL
    lib_.cdbm_destroy(None)
