"""cdbm_step_noalloc: the allocation-free time step.

Some callers cannot allocate device memory themselves -- a host code whose memory
pool owns every GPU byte and forbids allocations inside its time loop, or a plug-in
that receives device buffers but has no allocator.  For them the library offers a
step that keeps its scratch in a fixed device array of the library instead of
allocating it.  These tests call it through the C ABI and check that it reproduces
the context-based cdbm_step, twice in a row (the second call reuses the scratch the
first one left behind), and that it rejects grids above its fixed maximum.

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2502_16818_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12      # same bound as the short-run parity tests


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16818_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _c_args(w):
    from paper_2502_16818_gb300 import cdbm
    grid = cdbm.cdbm_grid(w.nx, w.ny, w.dx, w.dy, w.bc_x, w.bc_y)
    vset = cdbm.cdbm_vset((ctypes.c_double * 4)(*w.vg), (ctypes.c_double * 4)(*w.eg))
    return grid, vset


def _workload(name):
    if name == "blocks":
        return W.random_blocks(96, 40, seed=21, dt=1e-4, tau=2e-4)
    if name == "max_cells":
        # exactly CDBM_NOALLOC_MAX_CELLS cells: the stage buffer's last plane ends at
        # the flag slot of the fixed scratch
        w = W.random_blocks(256, 128, seed=22)
        w.dx, w.dy = 1.0 / 256, 1.0 / 128
        w.dt = 0.2 * w.dy / 2.2
        w.tau = 2 * w.dt
        return w
    return W.sod(nx=500, I=0.0)


@pytest.mark.parametrize("name", ["blocks", "max_cells", "sod"])
def test_step_noalloc_matches_cdbm_step(name):
    """Two calls in a row against a context stepped alongside.  On 2-D grids both
    paths launch the same stage kernels, so the states agree bit for bit; a short
    tube steps through the context's cluster kernel, which agrees to rounding."""
    from paper_2502_16818_gb300 import Solver, cdbm
    w = _workload(name)
    if name == "max_cells":
        assert w.nx * w.ny == cdbm.CDBM_NOALLOC_MAX_CELLS
    ref = Solver.from_workload(w)
    ref.init(w.rho, w.ux, w.uy, w.T)
    f = ref.state().clone()                    # caller-owned state, same initial value
    grid, vset = _c_args(w)
    stream = torch.cuda.current_stream().cuda_stream
    for nsteps in (7, 5):                      # two calls in a row on the same scratch
        ref.step(nsteps)
        expect = ref.state()
        cdbm.cdbm_step_noalloc(grid, vset, w.I, w.tau, w.dt, f.data_ptr(), nsteps, stream)
        if w.ny > 1:
            assert torch.equal(f, expect), (name, nsteps)
        err = (f - expect).abs().max().item() / expect.abs().max().item()
        assert err <= TOL, (name, nsteps, err)
    ref.sync()
    ref.close()


def test_step_noalloc_rejects_oversized_grid():
    from paper_2502_16818_gb300 import CdbmError, cdbm
    n = cdbm.CDBM_NOALLOC_MAX_CELLS + 1
    w = W.sod(nx=n, I=0.0, dt=1e-7, tau=1e-6)
    grid, vset = _c_args(w)
    f = torch.ones((16, 1, n), dtype=torch.float64, device="cuda")
    with pytest.raises(CdbmError) as e:
        cdbm.cdbm_step_noalloc(grid, vset, w.I, w.tau, w.dt, f.data_ptr(), 1, 0)
    assert e.value.status == cdbm.CDBM_EINVAL
    assert "exceeds its fixed scratch" in str(e.value)
    assert torch.all(f == 1.0)
