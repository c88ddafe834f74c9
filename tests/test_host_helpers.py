"""Header-only helpers of the GPU path checked on the CPU (compiled with nvcc as host code): the
tensor-core weight layout maps every (row, tap, channel) to its own slot, and the float32
form's operand scale puts a tensor's largest magnitude in [2^13, 2^14) (below 2^14 when
clamped)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_layout_bijection_and_operand_scales(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "check_helpers")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-o", exe,
                        os.path.join(HERE, "host", "check_helpers.cu")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "OK" in r.stdout
