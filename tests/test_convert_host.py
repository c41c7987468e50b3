"""Host check of the integer float <-> double conversions the single-precision
stage kernels use (paper_2502_16818_gb300/csrc/cdbm_convert.h): every float widened,
and 44 M doubles (random bit patterns, the float range, exact ties, the ends of the
range) narrowed, each compared bit for bit with the C conversion (IEEE round to
nearest, ties to even)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2502_16818_gb300", "csrc")


def test_integer_conversions_match_c_casts(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "convert_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "convert_check.cc"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.split() == ["widen", "0", "narrow_random", "0", "narrow_float_range", "0",
                                "narrow_ties", "0", "narrow_edges", "0"]
