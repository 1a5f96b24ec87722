"""Integer binary64 <-> binary32 conversions of the mixed-precision kernels,
checked on the host against IEEE round-to-nearest conversions (every binary32
value, the rounding ties, subnormal, overflow and NaN inputs)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_integer_conversions_match_ieee(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "conv_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2508_16387_gb300", "csrc"),
                    os.path.join(HERE, "native", "conv_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
