"""Integer binary64 <-> binary32 conversions of the mixed-precision kernels,
checked on the host against IEEE round-to-nearest conversions (every binary32
value, the rounding ties, subnormal, overflow and NaN inputs); the FP64 division
helpers on the device; and, on the host, the bulk kernel's shared-memory budget
per tile shape."""
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
    subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu", "-Xcompiler", "-fopenmp", "-lgomp",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2508_16387_gb300", "csrc"),
                    os.path.join(HERE, "native", "conv_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout


@pytest.mark.gpu
def test_fp64_reciprocal_and_quotient_match_ieee(tmp_path):
    """The bulk kernels' FP64 quotient (Newton-Raphson reciprocal from a binary32 seed, then a
    residual correction) equals IEEE a / b on the device; the reciprocal alone is within an ulp,
    and the reciprocal square root within two ulps of 1/sqrt(x)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "div_check")
    subprocess.run([nvcc, "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2508_16387_gb300", "csrc"),
                    os.path.join(HERE, "native", "div_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "quotient mismatches 0" in r.stdout, r.stdout
    worst = float(r.stdout.split("reciprocal worst ulp")[1].split()[0])
    assert worst <= 1.0, r.stdout
    # the reciprocal square root of the MG isentrope integrand: within two ulps of 1/sqrt(x)
    worst_rsqrt = float(r.stdout.split("rsqrt worst ulp")[1].split()[0])
    assert worst_rsqrt <= 2.0, r.stdout


def test_bulk_kernel_tiles_fit_their_blocks_per_sm(tmp_path):
    """The bulk kernel's shared memory per tile shape (a compile-time size) leaves room for the
    resident blocks per SM the design counts on: two 16-row, four 8-row and six 4-row FP32
    blocks, one FP64 block (checked on the host, no GPU)."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "smem_check")
    subprocess.run([nvcc, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2508_16387_gb300", "csrc"),
                    os.path.join(HERE, "native", "smem_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "misfits 0" in r.stdout
