"""Host-only: the fused stage's row tiling (row_tile, row_tiles in
csrc/args.cuh) checked exhaustively by a small native program built with nvcc
for the host (tests/native/row_tiling_check.cu): partition of the rows, rows
written only by the tile that covers them, border rows only by border tiles,
tiles inside the image, at least 2R rows for the last interior tile with short
border rows.  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_row_tiling_exhaustive(tmp_path):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "row_tiling_check")
    src = os.path.join(ROOT, "tests", "native", "row_tiling_check.cu")
    inc = [os.path.join(ROOT, "paper_1702_07482_gb300", "csrc"), os.path.join(ROOT, "include")]
    cmd = [nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-gencode",
           "arch=compute_103a,code=sm_103a", *sum((["-I", d] for d in inc), []), src, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")
