"""The tensor form's work schedule, checked on the host: tests/host/sched_check.cu
is compiled against csrc/sched.cu and run over 2560 shapes (group counts,
query tiles, reference tiles, paired and unpaired).  See that file for the
invariants."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_schedule_covers_every_unit_once(tmp_path):
    from paper_1707_00516_gb300 import build as Bd
    nvcc = Bd._nvcc()
    if not (os.path.exists(nvcc) or shutil.which(nvcc)):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "sched_check")
    subprocess.run([nvcc, "-std=c++17", "-I", Bd.INCLUDE, "-I", Bd.CSRC, "-o", exe,
                    os.path.join(HERE, "host", "sched_check.cu"), os.path.join(Bd.CSRC, "sched.cu")],
                   check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "bad 0" in r.stdout
