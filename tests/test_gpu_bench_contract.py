"""The bench's JSON line on a small grid: one line on stdout with every key the
measurement contract names (metric, value, unit, timing, roofline, CPU baseline,
end-to-end, clocks, launch count), with consistent values."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16818_gb300 import _build
    _build.build()


def test_bench_line_has_the_contract_keys():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--n", "256", "--steps", "4", "--warmup", "3",
           "--full-steps", "0", "--adj-steps", "0", "--no-configs", "--no-ensemble"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "gpu_launches", "clocks", "roofline", "e2e",
                "cpu_baseline", "fp32_bulk", "fp32_df64", "fp32_dev"):
        assert key in d, key
    assert d["steps"] == 4 and d["warmup"] == 3 and d["n_gpus"] == 1
    cells = 256 * 256
    assert abs(d["value"] - cells * 4 / (d["ms_per_step"] * 4e-3)) <= 1e-6 * d["value"]
    assert d["gpu_launches"] == 2 * 4
    assert d["config"]["workload"] == "taylor_green_256x256_fp64"
    roof = d["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic", "peak_measured", "frac_of_measured_peak"):
        assert key in roof, key
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) <= 1e-12
    assert 0.8 < roof["peak_measured"] / roof["peak"] < 1.05      # the probe reaches the nominal FP64 rate
    assert roof["traffic"] is None                                 # the capture scales only above the L2
    e2e = d["e2e"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0 and e2e["value"] > 0
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] > 0
    for mode in ("fp32_bulk", "fp32_df64", "fp32_dev"):
        assert d[mode]["l2_density_error_vs_fp64"] <= 1e-5
    # the on-demand kernels, each with its time and HBM GB/s
    names = {"fp64": ("init_kernel", "macros_kernel", "tne_kernel", "sums_partial_kernel")}
    names["fp32_bulk"] = names["fp32_df64"] = names["fp32_dev"] = names["fp64"][1:]
    for mode, keys in names.items():
        aux = d["aux_kernels"] if mode == "fp64" else d[mode]["aux_kernels"]
        assert sorted(aux) == sorted(keys), (mode, sorted(aux))
        for k in keys:
            row = aux[k]
            assert row["ms"] > 0 and row["hbm_gbs"] > 0
            assert abs(row["hbm_gbs"] - row["bytes_per_cell"] * cells / (row["ms"] * 1e-3) / 1e9) <= 1e-9 * row["hbm_gbs"]
