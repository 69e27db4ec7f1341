"""The library's 32-bit index arithmetic, checked on the host (no GPU):
division by invariant integers and the face topology, including the 11
implicit columns of the face operators in the stored ELL slot order.  The
check program (index_math_check.cu) includes the library's header, is
compiled here with nvcc for the host, and compares against definitions
written out with plain 64-bit arithmetic."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_index_arithmetic_on_the_host():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "index_math_check")
        r = subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr",
                            "-gencode", "arch=compute_103a,code=sm_103a",
                            os.path.join(HERE, "index_math_check.cu"), "-o", exe],
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout[-2000:] + r.stderr[-2000:]
