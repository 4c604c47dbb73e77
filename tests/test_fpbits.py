"""The integer-pipe FP64 <-> FP32 conversions the kernels use in place of FP64
instructions (csrc/fpbits.cuh), compiled for the host and checked bit for bit
against the C library's conversions in each rounding mode, ldexp and the
ordering of doubles, on random bit patterns and inputs near rounding ties."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fpbits_match_ieee_conversions(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "fpbits_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-frounding-math", "-I",
                    os.path.join(ROOT, "paper_1604_03290_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "fpbits_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe, "3000000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails 0" in r.stdout
