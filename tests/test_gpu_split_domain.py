"""A periodic grid split into two strips, each advanced by its own context on the same
GPU, equals the undivided run bit for bit (the split-domain symmetry: a strip
decomposition changes nothing but where the cells live).

Each strip context holds its own cells plus 4 ghost rows (or columns) on each side.
One time step has two Runge-Kutta stages with a stencil of radius 2 (Eqs. 12-20), so
a step corrupts at most the 4 outermost rows of a context, which are the ghosts;
refreshing the ghosts from the other strip after every step keeps every owned cell
exact.  The exchange copies the 4-row halos between device tensors (the states go
through cdbm_get_state / cdbm_set_state, FP64, exact copies).  The owned cells of the
strips then run the same per-cell operations as the whole grid, whatever launch
geometry each context picks, so the comparison is bitwise.
"""
import numpy as np
import pytest

from paper_2502_16818_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 4          # ghost width: 2 stages x stencil radius 2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16818_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _solver(w, nx, ny):
    from paper_2502_16818_gb300 import Solver
    return Solver(nx, ny, w.dx, w.dy, w.dt, w.tau, w.I, w.vg, w.eg, w.bc_x, w.bc_y)


@pytest.mark.parametrize("axis", ["y", "x"])
@pytest.mark.parametrize("shape", [(96, 64), (130, 2 * 40)])
def test_two_strips_equal_undivided_run(axis, shape):
    nx, ny = shape
    w = W.random_blocks(nx, ny, seed=nx + ny, bc=(W.PERIODIC, W.PERIODIC))
    w.dx, w.dy = 1.0 / nx, 1.0 / ny
    w.dt = 0.2 * min(w.dx, w.dy) / 2.2
    w.tau = 2 * w.dt
    steps = 12
    whole = _solver(w, nx, ny)
    whole.init(w.rho, w.ux, w.uy, w.T)
    f = whole.state()                                 # [16][ny][nx], the shared start
    whole.step(steps)
    expect = whole.state()
    whole.close()

    dim = 1 if axis == "y" else 2                     # tensor axis of the split
    n = f.shape[dim]
    half = n // 2
    owned = [(0, half), (half, n)]
    strips = []
    for lo, hi in owned:
        m = hi - lo + 2 * H
        strips.append(_solver(w, nx if axis == "y" else m, m if axis == "y" else ny))

    def with_ghosts(g, lo, hi):
        idx = torch.arange(lo - H, hi + H, device=g.device) % n
        return g.index_select(dim, idx).contiguous()

    g = f.clone()
    for _ in range(steps):
        for s, (lo, hi) in zip(strips, owned):
            s.set_state(with_ghosts(g, lo, hi), 0.0)
            s.step(1)
        parts = [s.state().narrow(dim, H, hi - lo) for s, (lo, hi) in zip(strips, owned)]
        g = torch.cat(parts, dim=dim)
    for s in strips:
        s.sync()
        s.close()
    assert torch.equal(g, expect), float((g - expect).abs().max())
