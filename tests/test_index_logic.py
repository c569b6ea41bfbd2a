"""The kernels' index logic, compiled from dev.cuh for the host and run on the
CPU (tests/index_check.cu): the flux segments sweep every face of every
transverse line exactly once and read and write inside the block's arrays,
for all directions, segment lengths 1-16 and ragged shapes (along x all
items before the remainders sweep equal lengths); find_block maps every item
to its block on prefix sums with empty blocks; the integer-pipe compares
agree with the IEEE comparisons they replace."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_index_logic_on_the_host():
    from paper_2409_10384_gb300 import build as B
    nv = B._nvcc()
    if shutil.which(nv) is None and not os.path.exists(nv):
        pytest.skip("nvcc not available")
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    exe = os.path.join(out, "index_check")
    cmd = [nv, *B.ARCH, "-std=c++17", "-O1", "-I", B.CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "index_check.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
