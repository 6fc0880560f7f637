"""The C-ABI library builds, loads and exports what include/fastid.h declares;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1707_00516_gb300 import binding as B
from paper_1707_00516_gb300.build import INCLUDE, LIB, build

HEADER = os.path.join(INCLUDE, "fastid.h")


@pytest.fixture(scope="module")
def lib():
    build()
    return B.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fastid_\w+)\s*\(", src)))


def exported_functions(path=LIB):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    return sorted({ln.split()[-1] for ln in out.splitlines() if " T fastid_" in ln})


def test_header_exports_match(lib):
    decl = declared_functions()
    assert decl, "no declarations parsed"
    assert decl == exported_functions()
    assert sorted(B.EXPORTS) == decl


def test_version_and_status_strings(lib):
    assert lib.fastid_version() == 100
    for code in range(8):
        assert lib.fastid_status_string(code).decode().startswith("FASTID_")


def test_create_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.fastid_create(ctypes.byref(h), 0)
    assert st in (B.ECUDA, B.EINVAL)
    assert not h.value
    assert lib.fastid_create(None, 0) == B.EINVAL


def test_null_context_is_einval(lib):
    P = None
    assert lib.fastid_destroy(P) == B.OK
    assert lib.fastid_set_form(P, 0) == B.EINVAL
    assert lib.fastid_sync_status(P, P) == B.EINVAL
    assert lib.fastid_profile(P, 1) == B.EINVAL
    assert lib.fastid_profile_read(P, None, None, None, 0) == B.EINVAL
    assert lib.fastid_pack(P, P, 1, 64, 64, P, 1, P, P) == B.EINVAL
    assert lib.fastid_mix(P, P, 1, 1, P, 1, P, 1, P, P) == B.EINVAL
    assert lib.fastid_load_refs(P, P, 1, 64, 1, 0, None, P) == B.EINVAL
    assert lib.fastid_free_refs(P, P) == B.OK
    assert lib.fastid_refs_view(P, P, 0, 1, None) == B.EINVAL
    assert lib.fastid_topk_fold(P, P, P, P, P, 0, 1, 16, P) == B.EINVAL
    assert lib.fastid_topk_accumulate(P, P, 0, P, 1, 1, P, 16, 0, P, P, P) == B.EINVAL
    assert lib.fastid_refs_info(P, None, None, None, None) == B.EINVAL
    assert lib.fastid_scores(P, P, P, 1, 1, P, P, 4, 1, P) == B.EINVAL
    assert lib.fastid_topk(P, P, P, 1, 1, P, 16, 0, P, P, P) == B.EINVAL
    assert lib.fastid_compare(P, P, P, 1, 1, P, 0, 0, P, P, P, P, P) == B.EINVAL
    assert lib.fastid_last_error(P) == b""
    assert lib.fastid_memory_info(P, None, None, None) == B.EINVAL


def test_library_missing_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        B.load_library(str(tmp_path / "nope.so"))


def test_debug_build_exports_match():
    """The FASTID_DEBUG build (device-side consistency checks, schedule
    self-check) compiles and exports the same entry points."""
    path = build(debug=True)
    assert os.path.basename(path) == "libfastid_debug.so"
    assert exported_functions(path) == declared_functions()


def test_peaks_library_builds_and_exports():
    """The roofline microbenchmarks compile for sm_103a and export their
    three entry points."""
    from paper_1707_00516_gb300.build import build_peaks
    path = build_peaks()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    names = sorted({ln.split()[-1] for ln in out.splitlines() if " T fastid_peaks_" in ln})
    assert names == ["fastid_peaks_alu", "fastid_peaks_b1", "fastid_peaks_mma"]


def test_peaks_operand_encoding():
    """e4m3: +1 = 0x38 (exponent 7 = bias), -1 = 0xB8; e2m1: +1 = 0x2
    (exponent 1 = bias), -1 = 0xA; element 2i in the low nibble of byte i."""
    import numpy as np
    from paper_1707_00516_gb300.peaks import encode
    v = np.array([[1, -1, 0, 1]])
    assert encode(v, False).tolist() == [[0x38, 0xB8, 0x00, 0x38]]
    assert encode(v, True).tolist() == [[0xA2, 0x20]]


def test_readme_c_example_compiles_and_links(lib, tmp_path):
    """The README's C example compiles as C11 against include/fastid.h with
    every warning an error, and links against libfastid.so and the CUDA
    runtime with no undefined symbol (nothing is run)."""
    import shutil
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("CUDA headers missing")
    readme = open(os.path.join(os.path.dirname(INCLUDE), "README.md")).read()
    blocks = re.findall(r"```c\n(.*?)```", readme, flags=re.S)
    assert len(blocks) == 1
    src = tmp_path / "example.c"
    src.write_text(blocks[0])
    libdir = os.path.dirname(LIB)
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.exists(os.path.join(d, "libcudart.so"))), None)
    if cudalib is None:
        pytest.skip("libcudart missing")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-shared", "-fPIC", "-I", INCLUDE,
                    "-I", os.path.join(cuda, "include"), str(src), "-o", str(tmp_path / "libexample.so"),
                    "-L", libdir, "-lfastid", "-L", cudalib, "-lcudart", "-Wl,--no-undefined"],
                   check=True, capture_output=True, text=True)
