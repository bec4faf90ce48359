"""Host builds of index logic the GPU kernels use, run without a GPU: the
compact numbering of the Gram kernels' 4 x 4 tiles (gram_tile), compiled
from the library's own header by nvcc as host code."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not available")


def test_gram_tile_numbering_covers_every_tile_once(tmp_path):
    exe = tmp_path / "gram_tile_check"
    src = os.path.join(ROOT, "tests", "host", "gram_tile_check.cu")
    subprocess.run([_nvcc(), "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1408_0042_gb300", "csrc"), src, "-o", str(exe)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
