"""The learned proposal's ray layout (air_internal.cuh: prop_rays, prop_ray,
prop_index), which the proposal kernels write and the march, the batched
kernel and the gather read back: a host program built from the library's
own header checks, for every combination of quadrant depths up to level 5,
that every ray round-trips through prop_index, that no pixel is traced
twice, and that pixels below the proposed depths are reported as missing."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1010_5534_gb300", "csrc")


def _nvcc():
    for c in ("/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def test_proposal_layout_round_trips():
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = os.path.join(HERE, "native", "prop_layout_check.cu")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "prop_layout_check")
        subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", CSRC, src, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
