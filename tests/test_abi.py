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


def test_diagnostic_and_batch_switch_argument_checks(lib):
    """Argument checks that return before any CUDA call."""
    lib_ = cdbm.load()
    assert lib_.cdbm_diag_rcp64(None, None, -1, None) == cdbm.CDBM_EINVAL
    assert "n < 0" in lib_.cdbm_last_error(None).decode()
    assert lib_.cdbm_diag_rcp64(None, None, 0, None) == cdbm.CDBM_OK          # nothing to do
    assert lib_.cdbm_diag_rcp64(None, None, 5, None) == cdbm.CDBM_EINVAL       # NULL with n > 0
    flops = ctypes.c_double()
    for blocks, threads, iters in ((0, 128, 1), (1, 100, 1), (1, 2048, 1), (1, 128, 0)):
        st = lib_.cdbm_diag_fp64_fma(ctypes.c_void_p(16), blocks, threads, iters, None, ctypes.byref(flops))
        assert st == cdbm.CDBM_EINVAL, (blocks, threads, iters)
    assert lib_.cdbm_diag_fp64_fma(None, 1, 128, 1, None, ctypes.byref(flops)) == cdbm.CDBM_EINVAL
    assert lib_.cdbm_batch_set_symmetric(None, 1) == cdbm.CDBM_EINVAL
    # the batch validates its precision before any CUDA call
    nx = (ctypes.c_int * 1)(10)
    dx = (ctypes.c_double * 1)(0.1)
    I = (ctypes.c_double * 1)(0.0)
    vset = cdbm.cdbm_vset((ctypes.c_double * 4)(*W.VSET_SOD[0]), (ctypes.c_double * 4)(*W.VSET_SOD[1]))
    out = ctypes.c_void_p(123)
    st = lib_.cdbm_batch_create(1, nx, dx, I, ctypes.byref(vset), 1e-4, 1e-5, 7, None, None, ctypes.byref(out))
    assert st == cdbm.CDBM_EINVAL and out.value is None
    assert "unsupported precision 7" in lib_.cdbm_last_error(None).decode()


def test_symmetric_velocity_maps(tmp_path):
    """The index maps of the y-symmetric kernels (cdbm_device.cuh, compiled here as
    host code) against the geometry of Eq. (2) as the oracle builds it: each
    velocity's direction signs, the image it holds on a y-symmetric state (same x
    component, opposite y component), the mirror plane a computed velocity also
    writes, and the 10 distinct velocities (v_y >= 0, the images of the others)."""
    import shutil
    import subprocess
    import oracle
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    exe = str(tmp_path / "velocity_maps")
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2502_16818_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "velocity_maps.cu"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [list(map(int, line.split())) for line in out[:16]]
    distinct = list(map(int, out[16].split()))
    vx, vy, _ = oracle.velocity_set((1.0, 1.0, 2.0, 2.0), (0.0, 0.0, 0.0, 1.0))
    image = {i: [k for k in range(16) if vx[k] == vx[i] and vy[k] == -vy[i]][0] for i in range(16)}
    for i, dx, dy, mirror, partner in rows:
        assert (dx, dy) == (int(round(vx[i] / abs(vx[i]))) if vx[i] else 0,
                            int(round(vy[i] / abs(vy[i]))) if vy[i] else 0), i
        if vy[i] < 0:
            assert mirror == image[i] and partner == -1, i      # held by its image
        else:
            assert mirror == i, i                               # computed
            assert partner == (image[i] if image[i] != i else -1), i
    assert distinct == [i for i in range(16) if vy[i] >= 0]
