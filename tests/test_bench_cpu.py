"""bench.py host logic (no GPU): the kernel source hash that keys recorded
ncu figures ignores comments and whitespace but not code."""
import bench


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1707_00516_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "common.cuh").write_text("struct A { int x; };  // the A\n")
    (csrc / "tensor.cu").write_text("/* kernel */\nint f(int a) {\n    return a + 1;  // one\n}\n")
    (csrc / "plain.cu").write_text("int g() { return 2; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash("tensor")
    (csrc / "tensor.cu").write_text("// a new comment\nint f(int a) {\n  return a + 1;\n}\n/* more */\n")
    assert bench.kernel_source_hash("tensor") == h0
    (csrc / "tensor.cu").write_text("int f(int a) {\n    return a + 2;\n}\n")
    assert bench.kernel_source_hash("tensor") != h0
    assert bench.kernel_source_hash("plain") != h0


def test_recorded_traffic_matches_current_sources():
    """Every recorded ncu figure names the source it was taken on; a stale key
    is reported as null traffic, so this only checks the keys are well formed."""
    for key, (bytes_, h) in bench.NCU_TRAFFIC.items():
        form, config = key.split("/")
        assert form in ("tensor", "plain") and config in bench.WORKLOADS
        assert bytes_ > 0 and len(h) == 16
