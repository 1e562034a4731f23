"""Index arithmetic of the windowed stage kernel, checked on the host.

Builds tests/window_index_check.cu (host code only runs) with nvcc and runs it:
every tile geometry the library launches keeps its global and shared-memory
indices in range and its tile-face mini-windows consistent. No GPU needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not on PATH")
def test_window_indices(tmp_path):
    exe = tmp_path / "window_index_check"
    subprocess.run(["nvcc", "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-o", str(exe), os.path.join(HERE, "window_index_check.cu")],
                   check=True, capture_output=True, timeout=600)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "all index checks passed" in out.stdout
