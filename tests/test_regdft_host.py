"""Host-side check of the register-level DFTs used inside every transform kernel: the device code is also
compiled for the host (nvcc) and compared with the DFT sum in double precision for each size."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1301_1215_gb300", "csrc")


def test_register_dfts_match_direct_sum(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "regdft_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "host", "regdft_check.cu"),
                    "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    sizes = set()
    for line in out:
        if line.startswith("twiddle"):
            continue
        r, d, err = line.split()
        sizes.add(int(r))
        assert float(err) < 2e-7, line
    assert {4, 8, 12, 16, 20, 24, 32} <= sizes
