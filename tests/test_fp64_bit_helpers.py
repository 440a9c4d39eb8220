"""The FP64 helpers the kernels evaluate on the integer pipe (sign tests,
min / max, |a| < t, max(x, 0), exact doubling / halving, -4x, x/2, the
product by a sign factor +-1, the limited slope) give the IEEE results: a
host build of the kernels' own header, checked against the host compiler's
IEEE arithmetic on random and special doubles."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_fp64_integer_pipe_helpers_are_ieee_exact(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "fp64_bits_check")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off",
                           os.path.join(HERE, "fp64_bits_check.cu"), "-o", exe])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
