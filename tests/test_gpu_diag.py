"""Diagnostic entry points (cdbm_diag_*), through the C ABI.

rcp64 is the reciprocal every stage kernel uses for 1 / rho: the hardware estimate
refined by one cubic Newton-Raphson step, r (1 + e + e^2) with e = 1 - a r.  The
end-to-end parity bar (1e-10) would hide a reciprocal that is a few ulp off, so it is
bounded here on its own against IEEE division (numpy's, correctly rounded) over the
densities the method meets and far beyond: 10^6 values over [1e-6, 1e6], half log
spaced, half log-uniform random.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16818_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def test_rcp64_within_one_ulp_of_division():
    from paper_2502_16818_gb300 import cdbm
    n = 1 << 20
    rng = np.random.default_rng(0)
    x = np.concatenate([np.logspace(-6, 6, n // 2), 10.0 ** rng.uniform(-6, 6, n // 2)])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    cdbm.cdbm_diag_rcp64(xd.data_ptr(), yd.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    y = yd.cpu().numpy()
    q = 1.0 / x                                   # correctly rounded
    ulps = np.abs(y - q) / np.spacing(q)
    assert ulps.max() <= 1.0, ulps.max()
    # a defect of the Newton step would show as a systematic offset, not as rare
    # last-bit differences
    assert np.mean(y == q) > 0.9, np.mean(y == q)
    # |y x - 1| from the exact product: y * x = p + err with err from the exact
    # splitting of y and x into 26-bit halves (Dekker), all in double
    def split(a):
        c = a * 134217729.0
        hi = c - (c - a)
        return hi, a - hi
    yh, yl = split(y)
    xh, xl = split(x)
    p = y * x
    err = ((yh * xh - p) + yh * xl + yl * xh) + yl * xl
    resid = np.abs((p - 1.0) + err)
    # within one ulp of the correctly rounded quotient, itself within half an ulp of
    # 1 / x: |y x - 1| <= 1.5 2^-52
    assert resid.max() <= 1.5 * 2.0 ** -52, resid.max()


def test_rcp64_edge_sizes():
    from paper_2502_16818_gb300 import CdbmError, cdbm
    cdbm.cdbm_diag_rcp64(0, 0, 0, 0)                      # nothing to do
    x = torch.tensor([1.0, 2.0, 0.125, 3.0], dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    cdbm.cdbm_diag_rcp64(x.data_ptr(), y.data_ptr(), 4, 0)
    torch.cuda.synchronize()
    assert y.tolist()[:3] == [1.0, 0.5, 8.0]
    with pytest.raises(CdbmError):
        cdbm.cdbm_diag_rcp64(x.data_ptr(), y.data_ptr(), -1, 0)


def test_fp64_fma_probe_runs():
    from paper_2502_16818_gb300 import CdbmError, cdbm
    out = torch.empty(4 * 128, dtype=torch.float64, device="cuda")
    flops = cdbm.cdbm_diag_fp64_fma(out.data_ptr(), 4, 128, 100, 0)
    torch.cuda.synchronize()
    assert flops == 2 * 8 * 100 * 4 * 128
    # the chains x <- 0.9999999 x + 1e-7 stay near their start (~1 + k 1e-3)
    assert torch.all(torch.isfinite(out)) and float(out.min()) > 7.9 and float(out.max()) < 8.1
    with pytest.raises(CdbmError):
        cdbm.cdbm_diag_fp64_fma(out.data_ptr(), 4, 100, 10, 0)
