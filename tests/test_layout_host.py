"""Host check of the state layouts: compiles tests/layout_check.cu (the
library's own layout header, host code only) with nvcc and runs it."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_field_map_is_a_bijection_and_rows_are_block_aligned(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "layout_check")
    src = os.path.join(ROOT, "tests", "layout_check.cu")
    inc = os.path.join(ROOT, "paper_2301_01622_gb300", "csrc")
    r = subprocess.run([nvcc, "-std=c++17", "-I", inc, src, "-o", exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "layout check ok" in r.stdout, r.stdout[-2000:]
