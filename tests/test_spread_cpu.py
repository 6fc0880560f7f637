"""Query spreading of the tensor calls, checked on the host: tests/host/
spread_check.cu is compiled against csrc/common.cuh and checks that the row
and query maps are inverse bijections with the padding of real calls."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_spread_maps_are_inverse_bijections(tmp_path):
    from paper_1707_00516_gb300 import build as Bd
    nvcc = Bd._nvcc()
    if not (os.path.exists(nvcc) or shutil.which(nvcc)):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "spread_check")
    subprocess.run([nvcc, "-std=c++17", "-I", Bd.INCLUDE, "-I", Bd.CSRC, "-o", exe,
                    os.path.join(HERE, "host", "spread_check.cu")], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "bad 0" in r.stdout
