"""The FP64 path's own reciprocal, quotient and inverse cube root (Newton-
Raphson from the hardware approximations, swe_kernels.cuh) against CUDA's
IEEE division and cbrt on the GPU: within 1, 2 and 4 units in the last
place. The FP64 step's parity with the oracle (1e-11) rests on these."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_newton_raphson_fp64_math_against_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "fp64_math_check")
    subprocess.run([nvcc, "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-o", exe, os.path.join(HERE, "fp64_math_check.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    err = {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}
    assert err["rcp"] <= 1.0, err
    assert err["div"] <= 2.0, err
    assert err["icbrt"] <= 4.0, err
