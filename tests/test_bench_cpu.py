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


def test_reference_arm_json_line(capsys):
    """`bench.py --impl reference` prints one JSON line with the contract's keys:
    the oracle timed on the host, its cpu_baseline and an e2e block with no
    host-device bytes (run on the small 64 x 10k workload)."""
    import json

    import bench
    bench.main(["--impl", "reference", "--config", "c1", "--steps", "1", "--warmup", "0"])
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == bench.WORKLOADS["c1"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
