"""The integer-pipe IEEE double division and square root of the CUDA library
(csrc/svd2_softfp.cuh), compiled for the host with g++ and compared bit for bit
with the CPU's hardware division and square root.  The host build replaces
the GPU's approximate-reciprocal seeds by the exact value moved by up to
+-2 (and, as a margin check, +-4) units in the last place."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "softfp_host_check.cpp")
INC = os.path.join(ROOT, "paper_2005_07403_gb300", "csrc")


@pytest.mark.parametrize("ulps,count,seed", [(2, 400000, 1), (4, 200000, 2)])
def test_softfp_matches_hardware_on_host(tmp_path, ulps, count, seed):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    exe = str(tmp_path / "softfp_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                    f"-DSFP_HOST_PERTURB_ULPS={ulps}", f"-I{INC}", "-o", exe, SRC], check=True)
    r = subprocess.run([exe, str(count), str(seed)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
