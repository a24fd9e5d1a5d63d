"""Batch scheduler of libetp (csrc/batch.cu) on the CPU: the real scheduler linked
against a stub etp_step (tests/native/batch_stub.cu) — admission, per-context
exclusivity, failure retirement, tick counts, shutdown."""
import os
import shutil
import subprocess

import pytest


def test_batch_scheduler_with_stub_step(tmp_path, root):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "batch_sched_test")
    src = [os.path.join(root, "tests", "native", "batch_stub.cu"),
           os.path.join(root, "paper_2405_05213_gb300", "csrc", "batch.cu")]
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr",
                        "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe, *src, "-lpthread"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("OK"), out.stdout + out.stderr
