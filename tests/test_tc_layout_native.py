"""Host-only: the shared-memory and TMEM layouts of the tensor-core kernels (TcCfg
in csrc/args.cuh, TcAdjCfg and TcDkCfg in csrc/tc_bwd_cfg.cuh) for every
instantiated configuration, checked by a small native
program built with nvcc for the host (tests/native/tc_layout_check.cu): every
byte range an MMA descriptor or a staging loop addresses lies inside its own
region, the regions are disjoint, and shared memory and TMEM fit.  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tensor_core_layouts(tmp_path):
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "tc_layout_check")
    src = os.path.join(ROOT, "tests", "native", "tc_layout_check.cu")
    inc = [os.path.join(ROOT, "paper_1702_07482_gb300", "csrc"), os.path.join(ROOT, "include")]
    cmd = [nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-gencode",
           "arch=compute_103a,code=sm_103a", *sum((["-I", d] for d in inc), []), src, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok 27")
