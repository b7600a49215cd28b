"""Host-only layout consistency of the plan-time tables (tests/layout_check.cu,
compiled with nvcc and run on the CPU: no device call)."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fold_buffer_covers_the_table_layout():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "layout_check")
        subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                        os.path.join(HERE, "layout_check.cu")], check=True, cwd=tmp, timeout=600)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout
    assert r.stdout.strip().endswith("OK")
