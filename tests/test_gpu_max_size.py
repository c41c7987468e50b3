"""Grids at the limits of the kernels' index arithmetic, against the CPU oracle.

- 11803 x 11500 cells (135.7 M): the 16 velocity planes of one state buffer hold
  2.17e9 values, more than 2^31, so the element offsets of the last plane's upper rows
  (rows >= 9444) and the byte offsets of every plane but the first need 64-bit
  arithmetic.  One run per precision (35 GB of state in FP64), 2 steps, checked at
  sampled cells against oracle patches: the block corners of the piecewise-constant
  fields (where the limiter works), rows on both sides of the 2^31 offset, the top row
  (whose periodic neighbours are the bottom rows) and the last cell.
- 3 x 70001 cells: more rows than a launch grid has in y (65535), so the one-cell-per-
  thread stage kernel loops over rows; with and without row marching, the whole grid
  against the oracle.

Bars: FP64 <= 1e-10 relative max-norm (rho, T by their maxima; u by max(|u|, c_s)),
the state planes <= 1e-11 of their maximum; the single-precision modes <= 1e-5, the
method's single-precision bar, applied per cell.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2502_16818_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("rho", "ux", "uy", "T")
PRECISIONS = [0, 1, 2, 3]
PREC_IDS = ["fp64", "fp32_bulk", "fp32_df64", "fp32_dev"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16818_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _cfl_safe(w):
    """Time step at a CFL number of 0.4 for the sound velocity set (|v| <= 1.4)."""
    w.dx, w.dy = 1.0 / w.nx, 1.0 / w.ny
    w.dt = 0.2 * min(w.dx if w.nx > 1 else 1.0, w.dy) / 1.4
    w.tau = 2 * w.dt
    return w


def _model(w, **kw):
    d = dict(nx=w.nx, ny=w.ny, dx=w.dx, dy=w.dy, dt=w.dt, tau=w.tau, I=w.I, vg=w.vg, eg=w.eg,
             bc_x=w.bc_x, bc_y=w.bc_y)
    d.update(kw)
    return oracle.Model(**d)


def _axis(c, r, n, bc):
    """Patch indices along one axis and the position of c in them (periodic axes wrap,
    zero-gradient axes stop at the edge, which is then the patch's own edge)."""
    if bc == W.PERIODIC:
        return np.arange(c - r, c + r + 1) % n, r
    lo, hi = max(0, c - r), min(n - 1, c + r)
    return np.arange(lo, hi + 1), c - lo


def _oracle_at(w, cy, cx, steps):
    """Oracle macros and state at (cy, cx) from a patch of radius 4 steps + 2 around
    it; the patch's zero-gradient edges cannot reach the centre in that many steps
    (stencil radius 2 per stage)."""
    r = 4 * steps + 2
    ys, py = _axis(cy, r, w.ny, w.bc_y)
    xs, px = _axis(cx, r, w.nx, w.bc_x)
    sub = [a[np.ix_(ys, xs)] for a in (w.rho, w.ux, w.uy, w.T)]
    m = _model(w, nx=len(xs), ny=len(ys), bc_x=W.ZERO_GRADIENT, bc_y=W.ZERO_GRADIENT)
    f = oracle.step(m, oracle.init(m, *sub), steps)
    ref = oracle.macros(m, f)
    return [ref[k][py, px] for k in range(4)], f[:, py, px]


@pytest.fixture(scope="module")
def huge():
    w = W.random_blocks(11803, 11500, seed=97, bc=(W.ZERO_GRADIENT, W.PERIODIC))
    return _cfl_safe(w)


@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
def test_state_beyond_2_31_values(huge, prec):
    from paper_2502_16818_gb300 import Solver
    w, steps = huge, 2
    P = w.nx * w.ny
    assert 16 * P > 2 ** 31
    first_row_past = (2 ** 31 - 15 * P) // w.nx + 1          # plane 15 offsets >= 2^31 from here
    s = Solver.from_workload(w, precision=prec)
    s.init(w.rho, w.ux, w.uy, w.T)
    s.step(steps)
    s.sync()
    got = [t.cpu().numpy() for t in s.macros()]
    f_gpu = s.state()
    s.close()
    bx, by = max(1, w.nx // 7), max(1, w.ny // 5)           # block sizes of random_blocks
    pts = [(by * k + d, bx * j + e) for k in (1, 4) for j in (1, 3, 6) for d in (-1, 0) for e in (-1, 0)]
    pts += [(first_row_past + d, x) for d in (-2, -1, 0, 1) for x in (0, 5000, w.nx - 1)]
    pts += [(w.ny - 1, 0), (w.ny - 1, w.nx - 1), (w.ny - 1, 7777), (0, 0), (0, w.nx - 1)]
    rng = np.random.default_rng(5)
    pts += [(int(rng.integers(w.ny)), int(rng.integers(w.nx))) for _ in range(8)]
    cs = math.sqrt(W.gamma_of(w.I) * float(np.mean(got[3])))
    us = max(np.abs(got[1]).max(), np.abs(got[2]).max(), cs)
    scale = [np.abs(got[0]).max(), us, us, np.abs(got[3]).max()]
    tol, tol_f = (1e-10, 1e-11) if prec == 0 else (1e-5, 1e-5)
    for (cy, cx) in pts:
        ref, fref = _oracle_at(w, cy, cx, steps)
        for k, name in enumerate(FIELDS):
            e = abs(got[k][cy, cx] - ref[k]) / scale[k]
            assert e <= tol, "%s at (%d,%d): %.3e" % (name, cy, cx, e)
        fcell = f_gpu[:, cy, cx].cpu().numpy()
        assert np.abs(fcell - fref).max() <= tol_f * np.abs(fref).max(), (cy, cx)
    del f_gpu
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", PRECISIONS, ids=PREC_IDS)
def test_more_rows_than_the_launch_grid(prec):
    from paper_2502_16818_gb300 import Solver, cdbm
    w = _cfl_safe(W.random_blocks(3, 70001, seed=71, bc=(W.ZERO_GRADIENT, W.PERIODIC)))
    steps = 3
    runs = []
    for enable in (0, 1):
        s = Solver.from_workload(w, precision=prec)
        cdbm.cdbm_set_row_marching(s.ctx, enable)
        s.init(w.rho, w.ux, w.uy, w.T)
        s.step(steps)
        s.sync()
        runs.append(([t.cpu().numpy() for t in s.macros()], s.state().cpu().numpy()))
        s.close()
    assert np.array_equal(runs[0][1], runs[1][1])                # the same operations per cell
    m = _model(w)
    f = oracle.step(m, oracle.init(m, w.rho, w.ux, w.uy, w.T), steps)
    ref = oracle.macros(m, f)
    got = runs[0][0]
    cs = math.sqrt(W.gamma_of(w.I) * float(np.mean(ref[3])))
    us = max(np.abs(ref[1]).max(), np.abs(ref[2]).max(), cs)
    tol = 1e-10 if prec == 0 else 1e-5
    assert np.abs(got[0] - ref[0]).max() / np.abs(ref[0]).max() <= tol
    assert max(np.abs(got[1] - ref[1]).max(), np.abs(got[2] - ref[2]).max()) / us <= tol
    assert np.abs(got[3] - ref[3]).max() / np.abs(ref[3]).max() <= tol
    if prec == 0:
        assert np.abs(runs[0][1] - f).max() <= 1e-11 * np.abs(f).max()
