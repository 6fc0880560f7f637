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
        assert form in bench.FORMS and config in bench.WORKLOADS
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
    assert d["config"] == bench.workload_config(bench.WORKLOADS["c1"])  # the GPU arm's config keys
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_multi_gpu_refused(monkeypatch):
    """The library compares on one device per call: bench.py refuses --gpus
    other than 1 and a multi-process launch before touching a GPU."""
    import pytest

    import bench
    with pytest.raises(SystemExit) as e:
        bench.main(["--gpus", "2", "--steps", "1"])
    assert e.value.code == 2
    monkeypatch.setenv("WORLD_SIZE", "2")
    with pytest.raises(SystemExit) as e:
        bench.main(["--steps", "1"])
    assert e.value.code == 2


def test_roofline_peaks_from_probe():
    """Each form's peak is the probe's per-clock rate x SMs x the maximum SM
    clock, in the form's own unit."""
    import bench
    probe = {"popc": {"per_clk_sm": 16.0}, "carry_save8": {"per_clk_sm": 26.5},
             "fp8_f8f6f4": {"flops_per_clk_sm": 16384.0},
             "fp4_mxf4_n224": {"flops_per_clk_sm": 32768.0, "shape": "M128xN224xK64"},
             "fp4_mxf4_n256": {"flops_per_clk_sm": 32760.0, "shape": "M128xN256xK64"}}
    mhz = float(bench.load_peaks()[0].get("sm_max_mhz", 2070.0))
    p, unit, _ = bench.roof_peak("plain", probe, 152)
    assert unit == "Tpopc/s" and abs(p - 26.5 * 152 * mhz * 1e6 / 1e12) < 1e-9
    p8, unit, _ = bench.roof_peak("fp8", probe, 152)
    assert unit == "TFLOP/s" and abs(p8 - 16384 * 152 * mhz * 1e6 / 1e12) < 1e-6
    assert bench.roof_peak("fp8packed", probe, 152)[0] == p8
    p4, _, how = bench.roof_peak("fp4", probe, 152)
    assert abs(p4 - 32768 * 152 * mhz * 1e6 / 1e12) < 1e-6 and "N224" in how


def test_cpu_baseline_reports_all_cores_and_one_thread():
    """The default line's cpu_baseline: the oracle on every host core over a
    calibrated sample, and the same oracle on one thread beside it (a small
    C3-shaped workload, so that the test takes seconds)."""
    import gen
    import oracle
    oracle.build()
    w = dict(bench.WORKLOADS["c3"])
    w["n_refs"] = 100_000
    recipe = bench.recipe_for("c3", n_refs=w["n_refs"], n_q=64)
    thr = gen.maf_thresholds(gen.config_seed(w["cfg"]), w["n_loci"])
    cb = bench.cpu_baseline(w, recipe, thr, target_s=0.5)
    assert cb["kind"] == "oracle" and cb["cores"] == oracle.max_threads() and cb["value"] > 0
    one = cb["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0 and one["unit"] == cb["unit"]
    # one thread is never much faster than all of them
    assert one["value"] < 1.5 * cb["value"]
