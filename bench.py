#!/usr/bin/env python3
"""FastID all-pairs comparison benchmark on one GB300.

Metric: query x reference comparisons per second at N loci, bit-exact
(results are checked against the CPU oracle by the tests), and for the
serving and batched workloads the p50/p99 batch latency.  One step = one pass
of the whole path over one batch of queries: pack the queries' contributor
alleles, build the mixtures (OR), compare every query with every resident
reference and reduce to the per-query top-k under a threshold.  The
reference database is resident in HBM (loaded once, outside the timed region).

Default workload: 2048 unknowns (1024 individuals, 1024 mixtures of 2-5
people) x 20,000,000 references, N = 2048 loci, top-32, threshold 512, timed
in the plain, FP8 and FP4 forms (the fastest is the headline), followed by
the serving workload (Poisson requests, p50/p99 latency) and the batched
workload (256 uneven batches over 4 loci panels, one graph replay) as the
line's `serving` and `batched` objects.

    python bench.py [--steps K] [--warmup W] [--form all|plain|fp8|fp4|...]
    python bench.py --config c4|c5        (batched / serving alone)
    python bench.py --impl reference ...  (the CPU oracle on a bounded sample)

The library compares on one device per call; bench.py runs on one GPU
(--gpus 1) and refuses a multi-process launch.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gen  # noqa: E402

# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

WORKLOADS = {
    "c3": dict(workload="2048q_x_20M_refs_N2048_top32_T512", n_q=2048, n_refs=20_000_000, n_loci=2048,
               k=32, threshold=512, cfg=3, output="per-query top-k"),
    "c2": dict(workload="2048mix_x_1M_refs_N4096_top16_T0", n_q=2048, n_refs=1_000_000, n_loci=4096,
               k=16, threshold=0, cfg=2, output="per-query top-k"),
    "c1": dict(workload="64q_x_10k_refs_N1024_full_uint16_matrices", n_q=64, n_refs=10_000, n_loci=1024,
               k=32, threshold=0xFFFFFFFF, cfg=1,
               output="both full uint16 score matrices (both scores of every pair)"),
    "c4": dict(workload="256_batches_1-512q_panels_N512-2048-8192-16384_x_4M_refs_top16", n_refs=4_000_000,
               panels=(512, 2048, 8192, 16384), n_batches=256, k=16, threshold=0xFFFFFFFF, cfg=4),
    "c5": dict(workload="serving_poisson200bps_1-256q_N2048_x_20M_refs_top16", n_refs=20_000_000, n_loci=2048,
               rate=200.0, k=16, threshold=0xFFFFFFFF, cfg=5),
}

METRIC = "query x reference comparisons/s at N loci, bit-exact"
UNIT = "comparisons/s"

# Compute forms: FASTID_FORM_* name, the database copy it reads, the
# arithmetic type of the line's dtype key.
FORMS = {
    "plain": ("FORM_PLAIN", 0, "u32"),
    "fp8": ("FORM_TENSOR", "REFS_TENSOR", "e4m3xe4m3->f32"),
    "fp8packed": ("FORM_TENSOR_PACKED", 0, "e4m3xe4m3->f32"),
    "fp4": ("FORM_TENSOR_FP4", "REFS_FP4", "e2m1xe2m1->f32 (unit ue8m0 block scales)"),
    "fp4packed": ("FORM_TENSOR_FP4_PACKED", 0, "e2m1xe2m1->f32 (unit ue8m0 block scales)"),
}
DEFAULT_FORMS = ("plain", "fp8", "fp4")
# Nominal dense rates relative to bf16 (2.25 PFLOP/s): e4m3 4.5, e2m1 13.5.
NOMINAL_OVER_BF16 = {"fp8": 2.0, "fp4": 6.0}


def workload_config(w: dict) -> dict:
    """The `config` object of both arms (the same keys for the same workload)."""
    c = {"workload": w["workload"], "n_queries": w.get("n_q"), "n_refs": w["n_refs"], "n_loci": w.get("n_loci"),
         "k": w["k"], "threshold": w["threshold"], "output": w.get("output")}
    if "n_loci" in w:
        c["l2"] = ("inputs larger than L2 (packed database %.2f GB; FP8 copy %.1f GB, FP4 copy %.1f GB)" % (
            w["n_refs"] * w["n_loci"] / 8 / 1e9, w["n_refs"] * w["n_loci"] / 1e9, w["n_refs"] * w["n_loci"] / 2e9)
            if w["n_refs"] * w["n_loci"] / 8 > 129e6 else
            "database smaller than L2 (%.1f MB packed): steps re-read it from L2" % (w["n_refs"] * w["n_loci"] / 8e6))
    return c


def recipe_for(name: str, n_refs: int | None = None, n_q: int | None = None):
    w = WORKLOADS[name]
    n_refs = w["n_refs"] if n_refs is None else n_refs
    n_q = w["n_q"] if n_q is None else n_q
    seed = gen.config_seed(w["cfg"])
    if name == "c3":
        return gen.recipe_c3(seed, n_refs=n_refs, n_q=n_q, n_loci=w["n_loci"])
    if name == "c2":
        return gen.recipe_c2(seed, n_refs=n_refs, n_q=n_q, n_loci=w["n_loci"])
    r = gen.recipe_individuals(n_q, n_refs, w["n_loci"], seed, n_planted=min(8, n_q))
    return r


def build_db(searcher, seed: int, n_refs: int, n_loci: int, flags: int = 0, chunk: int = 1 << 20):
    """Generate the reference database on the device (gen/gen_gpu.cu), pack it
    with fastid_pack and load it.  Returns (RefDB, thresholds)."""
    import torch
    from paper_1707_00516_gb300 import binding as B
    thr = gen.maf_thresholds(seed, n_loci)
    dev = searcher.device
    thr_dev = torch.from_numpy(thr.view(np.int32)).to(dev)
    w = (n_loci + 63) // 64
    packed = torch.empty((n_refs, w), dtype=torch.int64, device=dev)
    chunk = min(chunk, n_refs)
    alle = torch.empty((chunk, n_loci), dtype=torch.uint8, device=dev)
    for r0 in range(0, n_refs, chunk):
        n = min(chunk, n_refs - r0)
        gen.allele_rows_device(seed, gen.STREAM_DB, thr_dev, alle[:n], row0=r0)
        B.fastid_pack(searcher.ctx, alle[:n], n_loci, packed[r0:r0 + n])
    db = B.fastid_load_refs(searcher.ctx, packed, n_loci, flags)
    torch.cuda.synchronize()
    del packed, alle
    torch.cuda.empty_cache()
    return db, thr


def query_inputs(recipe, thr):
    """Host arrays of a recipe: contributor alleles, group offsets, modes."""
    src = gen.source_alleles(recipe, thr)
    return src, recipe.offsets.astype(np.int32), recipe.modes.astype(np.uint8)


# ----------------------------------------------------------------------------
# Clocks sampled during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 200):
        self.gpu = gpu_index
        self.interval_ms = int(interval_ms)
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def refuse_multi_gpu(args):
    """The library compares on one device per call: bench.py times one GPU."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus != 1 or world > 1:
        print(f"bench.py: this library runs each comparison on one GPU; run it with --gpus 1 and without "
              f"a multi-process launcher (got --gpus {args.gpus}, WORLD_SIZE {world})", file=sys.stderr)
        sys.exit(2)


# ----------------------------------------------------------------------------
# CPU oracle legs
# ----------------------------------------------------------------------------

def oracle_sample_step(q_alleles: np.ndarray, modes: np.ndarray, seed: int, n_refs: int, thr: np.ndarray,
                       sample_rows: np.ndarray, k: int, threshold: int, threads: int = 0):
    """The oracle on a bounded sample: every query against the sampled
    references (per-locus scores, then top-k over the sample), on `threads`
    host threads (0: all)."""
    import oracle
    R = gen.allele_rows(seed, gen.STREAM_DB, sample_rows, thr)
    t0 = time.perf_counter()
    mis, une = oracle.scores(R, q_alleles, threads)
    s = oracle.select(mis, une, modes)
    oracle.topk(s, k, threshold, ref_ids=sample_rows)
    return time.perf_counter() - t0


def cpu_baseline(w: dict, recipe, thr, target_s: float = 12.0):
    import oracle
    src, off, modes = query_inputs(recipe, thr)
    q = oracle.mix(src, off)
    seed = gen.config_seed(w["cfg"])
    rng = np.random.default_rng(seed)
    S = 16
    t = oracle_sample_step(q, modes, seed, w["n_refs"], thr, np.sort(rng.choice(w["n_refs"], S, replace=False)),
                           w["k"], w["threshold"])
    for _ in range(3):  # calibrate: small samples overstate the per-reference time
        S_max = min(1 << 16, w["n_refs"])
        S = int(min(S_max, max(16, S * target_s / max(t, 1e-3))))
        rows = np.sort(rng.choice(w["n_refs"], S, replace=False))
        t = oracle_sample_step(q, modes, seed, w["n_refs"], thr, rows, w["k"], w["threshold"])
        if t >= 0.6 * target_s or S == S_max:
            break
    cores = oracle.max_threads()
    # the same oracle on one host thread, over a sample sized to about 3 s
    S1 = int(max(8, min(S, 3.0 * S / (max(t, 1e-3) * max(1, cores)))))
    rows1 = np.sort(rng.choice(w["n_refs"], S1, replace=False))
    t1 = oracle_sample_step(q, modes, seed, w["n_refs"], thr, rows1, w["k"], w["threshold"], threads=1)
    return {"value": q.shape[0] * S / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {q.shape[0]} queries x {S} sampled references (per-locus scores + top-{w['k']}), "
                      f"{t:.1f} s",
            "single_thread": {"value": q.shape[0] * S1 / t1, "unit": UNIT, "cores": 1,
                              "sample": f"all {q.shape[0]} queries x {S1} sampled references, {t1:.1f} s"}}


def run_reference(args, w):
    """--impl reference: the CPU oracle, each step a bounded sample.  Under a
    multi-process launcher only rank 0 runs."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    oracle.build()
    seed = gen.config_seed(w["cfg"])
    recipe = recipe_for(args.config, n_refs=w["n_refs"], n_q=w.get("n_q"))
    thr = gen.maf_thresholds(seed, w["n_loci"])
    src, off, modes = query_inputs(recipe, thr)
    q = oracle.mix(src, off)
    rng = np.random.default_rng(seed + 1)
    # size one step to about 8 s on this host, and the whole run to about 150 s
    step_s = min(8.0, 150.0 / max(1, args.steps + args.warmup))
    S = 16
    t = oracle_sample_step(q, modes, seed, w["n_refs"], thr, np.sort(rng.choice(w["n_refs"], S, replace=False)),
                           w["k"], w["threshold"])
    S = int(min(1 << 16, w["n_refs"], max(16, S * step_s / max(t, 1e-3))))
    times = []
    for i in range(args.warmup + args.steps):
        rows = np.sort(rng.choice(w["n_refs"], S, replace=False))
        dt = oracle_sample_step(q, modes, seed, w["n_refs"], thr, rows, w["k"], w["threshold"])
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = q.shape[0] * S * len(times) / tot
    sample = f"per step: all {q.shape[0]} queries x {S} sampled references (per-locus scores + top-{w['k']})"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# Roofline denominators
# ----------------------------------------------------------------------------

def kernel_source_hash(form: str) -> str:
    """Hash of the kernel's source with comments and whitespace removed, so
    that edits to comments alone keep the recorded ncu figures valid."""
    h = hashlib.sha256()
    for f in ("plain.cu" if form == "plain" else "tensor.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1707_00516_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


# DRAM bytes per launch of the main compare kernel from an ncu capture
# (profiles/), keyed by form and workload, with the source hash it was taken
# at.  A changed kernel reports null.
NCU_TRAFFIC = {
    # profiles/tensor_kernel_fp4_c3_2048x20M.md: dram__bytes_read.sum 25.01 GB + dram__bytes_write.sum 39.98 MB
    "fp4/c3": (25.012413952e9 + 39.982848e6, "9f95518100d29482"),
    # profiles/tensor_kernel_c3_2048x20M.md: dram__bytes_read.sum 76.39 GB + dram__bytes_write.sum 78.66 MB
    "fp8/c3": (76.389554176e9 + 78.660864e6, "9f95518100d29482"),
    # profiles/plain_kernel_c3_2048x20M.md: dram__bytes_read.sum 45.61 GB + dram__bytes_write.sum 28.82 MB
    "plain/c3": (45.612705280e9 + 28.819456e6, "a0d17b3f0ba88167"),
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def roof_peak(form: str, probe: dict, n_sms: int) -> tuple[float, str, str]:
    """Peak of a form's bound from the microbenchmarks (paper_1707_00516_gb300
    .peaks, run by this process on this GPU): the measured rate per SM clock x
    SMs x the maximum SM clock.  Returns (peak, unit, how)."""
    peaks, src = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    if form == "plain":
        # word pairs (one 32-bit AND + popcount each) through the kernel's own
        # step -- 8 ANDs, 4 full adders, 4 POPCs -- timed alone by the probe
        per = probe["carry_save8"]["per_clk_sm"]
        return (per * n_sms * sm_max * 1e6 / 1e12, "Tpopc/s",
                f"the plain kernel's carry-save step: {per:.2f} word pairs/clk/SM measured (probe, registers only) x "
                f"{n_sms} SMs x {sm_max:.0f} MHz max SM clock; POPC alone {probe['popc']['per_clk_sm']:.2f}/clk/SM")
    kind = form.removesuffix("packed")
    if kind == "fp8":
        per, shape = probe["fp8_f8f6f4"]["flops_per_clk_sm"], "tcgen05 kind::f8f6f4 M128xN256xK32"
    else:
        key = max(("fp4_mxf4_n224", "fp4_mxf4_n256"), key=lambda k: probe[k]["flops_per_clk_sm"])
        per, shape = probe[key]["flops_per_clk_sm"], f"tcgen05 kind::mxf4 {probe[key]['shape']}"
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    return (per * n_sms * sm_max * 1e6 / 1e12, "TFLOP/s",
            f"{shape}: {per:.0f} flop/clk/SM measured (probe, smem operands, one CTA per SM) x {n_sms} SMs x "
            f"{sm_max:.0f} MHz max SM clock; nominal-ratio figure bf16 {bf16:.0f} ({src}) x "
            f"{NOMINAL_OVER_BF16[kind]:g} = {bf16 * NOMINAL_OVER_BF16[kind]:.0f}")


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def form_code(form: str) -> int:
    from paper_1707_00516_gb300 import binding as B
    return getattr(B, FORMS[form][0])


def form_flags(forms) -> int:
    from paper_1707_00516_gb300 import binding as B
    f = 0
    for name in forms:
        if FORMS[name][1]:
            f |= getattr(B, FORMS[name][1])
    return f


def time_form(args, s, form, step_fn, pairs_per_step, n_loci, dev, probe):
    """Warm up and time `args.steps` steps of one compute form; returns the
    device-timed result and the roofline of its main compare kernel."""
    import torch
    from paper_1707_00516_gb300 import binding as B
    B.fastid_set_form(s.ctx, form_code(form))
    for _ in range(args.warmup):
        step_fn()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index)
    clk.start()
    B.fastid_profile(s.ctx, True)
    B.fastid_profile_read(s.ctx, reset=True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step_fn()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = B.fastid_profile_read(s.ctx, reset=True)
    B.fastid_profile(s.ctx, False)
    clocks = clk.stop()
    st = B.fastid_sync_status(s.ctx)
    if st != B.OK:
        raise RuntimeError(f"device status {st} after the timed region ({form})")
    value = pairs_per_step * args.steps / (ms / 1e3)

    main_s = prof["main_ms"] / max(1, prof["main_launches"]) / 1e3
    # compare launches per step (several when references stream in blocks)
    main_per_step = max(1, prof["main_launches"]) / args.steps
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, unit, how = roof_peak(form, probe, n_sms)
    if form == "plain":
        words32 = 2 * ((n_loci + 63) // 64)
        achieved = pairs_per_step * words32 / (main_s * main_per_step) / 1e12
        roof = {"bound": "alu", "kernel": "plain_kernel<EPI_TOPK>"}
    else:
        achieved = 2.0 * pairs_per_step * n_loci / (main_s * main_per_step) / 1e12
        kind = "kind::mxf4 block-scaled e2m1" if form.startswith("fp4") else "kind::f8f6f4 e4m3"
        roof = {"bound": "tensor", "kernel": f"tensor_kernel (tcgen05 {kind}, EPI_TOPK" +
                (", packed rows expanded on chip)" if form.endswith("packed") else ")")}
    roof.update({"achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak, "peak_source": how,
                 "kernel_ms": main_s * 1e3})
    if form != "plain":
        peaks, _ = load_peaks()
        nominal = float(peaks.get("bf16_tflops", 1900.0)) * NOMINAL_OVER_BF16[form.removesuffix("packed")]
        roof["frac_of_nominal_ratio_peak"] = achieved / nominal
    key = f"{form}/{args.config}"
    # the captured counters hold for the unmodified workload only
    tr = None if (args.refs or args.queries or args.k) else NCU_TRAFFIC.get(key)
    roof["traffic"] = tr[0] if tr and tr[1] == kernel_source_hash(form) else None
    return {"value": value, "ms_per_step": ms / args.steps, "roofline": roof, "clocks": clocks,
            "gpu_launches": int(prof["all_launches"])}


def run_gpu(args, w):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300 import peaks as P
    from paper_1707_00516_gb300.build import build
    from paper_1707_00516_gb300.search import Searcher
    gen.build_gpu()
    build()
    probe = P.measure()

    forms = list(DEFAULT_FORMS) if args.form == "all" else args.form.split(",")
    s = Searcher(0, B.FORM_AUTO)
    seed = gen.config_seed(w["cfg"])
    n_refs, n_loci, k, T = w["n_refs"], w["n_loci"], w["k"], w["threshold"]
    db, thr = build_db(s, seed, n_refs, n_loci, form_flags(forms))
    recipe = recipe_for(args.config, n_refs=n_refs, n_q=w.get("n_q"))
    src, off, modes = query_inputs(recipe, thr)
    n_q = recipe.n_queries
    d_src = torch.from_numpy(src).to(dev)
    d_off = torch.from_numpy(off).to(dev)
    d_mod = torch.from_numpy(modes).to(dev)
    sc = torch.empty((n_q, k), dtype=torch.int32, device=dev)
    ix = torch.empty((n_q, k), dtype=torch.int64, device=dev)
    full = args.config == "c1"  # the two full uint16 score matrices, one per mode
    if full:
        m_mis = torch.full((n_q,), gen.MODE_MISMATCH, dtype=torch.uint8, device=dev)
        m_une = torch.full((n_q,), gen.MODE_UNEXPLAINED, dtype=torch.uint8, device=dev)
        out_mis = torch.empty((n_q, n_refs), dtype=torch.int16, device=dev)
        out_une = torch.empty((n_q, n_refs), dtype=torch.int16, device=dev)

    def step():
        q = s.build_queries(d_src, d_off, n_loci)
        if full:
            B.fastid_scores(s.ctx, db, q, m_mis, out_mis)
            B.fastid_scores(s.ctx, db, q, m_une, out_une)
        else:
            B.fastid_topk(s.ctx, db, q, d_mod, k, T, sc, ix)

    pairs_per_step = n_q * n_refs
    res = {f: time_form(args, s, f, step, pairs_per_step, n_loci, dev, probe) for f in forms}
    head = max(res, key=lambda f: res[f]["value"])
    hr = res[head]

    # end to end through the host-buffer API, headline form
    B.fastid_set_form(s.ctx, form_code(head))
    if full:  # contributor alleles in, both score matrices out, through pinned buffers
        h_src = torch.from_numpy(src).pin_memory()
        h_mis = torch.empty((n_q, n_refs), dtype=torch.int16, pin_memory=True)
        h_une = torch.empty((n_q, n_refs), dtype=torch.int16, pin_memory=True)

        def e2e_step():
            d_src.copy_(h_src, non_blocking=True)
            step()
            h_mis.copy_(out_mis, non_blocking=True)
            h_une.copy_(out_une, non_blocking=True)
            torch.cuda.synchronize()
            return h_src.numel(), 4 * n_q * n_refs
    else:  # the inputs wait in pinned host memory, as an application's would
        h_src = torch.from_numpy(src).pin_memory()
        h_off = torch.from_numpy(off).pin_memory()
        h_mod = torch.from_numpy(modes).pin_memory()

        def e2e_step():
            _, _, h2d_, d2h_ = s.search_host(db, h_src, h_off, h_mod, k, T)
            return h2d_, d2h_
    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h2d, d2h = e2e_step()
    e2e_s = time.perf_counter() - t0
    e2e_value = pairs_per_step * args.steps / e2e_s

    line = {"metric": METRIC + "; p50/p99 batch latency (serving, batched)", "value": hr["value"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": hr["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": FORMS[head][2],
            "data": "synthetic", "config": workload_config(w),
            "form": head, "forms_timed": forms,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h),
                    "path": "Searcher.search_host: torch copies from pinned host buffers through the Python "
                            "binding, then fastid_pack / fastid_mix / fastid_topk, results copied back"},
            "gpu_launches": hr["gpu_launches"], "roofline": hr["roofline"], "clocks": hr["clocks"],
            "forms": {f: {"value": r["value"], "ms_per_step": r["ms_per_step"], "roofline": r["roofline"],
                          "clocks": r["clocks"]} for f, r in res.items()},
            "peaks_probe": {"fp8_f8f6f4_flop_per_clk_sm": probe["fp8_f8f6f4"]["flops_per_clk_sm"],
                            "fp4_mxf4_flop_per_clk_sm": max(probe["fp4_mxf4_n224"]["flops_per_clk_sm"],
                                                            probe["fp4_mxf4_n256"]["flops_per_clk_sm"]),
                            "popc_per_clk_sm": probe["popc"]["per_clk_sm"],
                            "lop3_per_clk_sm": probe["lop3"]["per_clk_sm"],
                            "and_popc_iadd3_popc_per_clk_sm": probe["and_popc_add"]["per_clk_sm"],
                            "harley_seal_word_pairs_per_clk_sm": probe["harley_seal"]["per_clk_sm"],
                            "carry_save8_word_pairs_per_clk_sm": probe["carry_save8"]["per_clk_sm"],
                            "b1_mma_bit_macs_per_clk_sm": probe["b1_and_popc"]["bit_macs_per_clk_sm"]}}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, recipe, thr)
    db.close()
    del db
    if args.config == "c3" and not args.no_extras:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        line["serving"] = serving_measure(s, WORKLOADS["c5"], seconds=args.serving_seconds, warmup_seconds=2.0,
                                          slots=args.slots, max_wave=args.max_wave, hbm_budget=args.hbm_budget,
                                          clock_ms=args.clock_ms, server=args.server, parts=args.parts)
        if args.server == "sweep":  # the same requests with one wave in flight at a time, for comparison
            alt = serving_measure(s, WORKLOADS["c5"], seconds=args.serving_seconds, warmup_seconds=2.0, slots=1,
                                  max_wave=args.max_wave, hbm_budget=args.hbm_budget, clock_ms=args.clock_ms,
                                  server="waves")
            line["serving"]["one_wave_in_flight"] = {"value": alt["value"], "latency_ms": alt["latency_ms"],
                                                     "config": alt["config"], "clocks": alt["clocks"]}
        torch.cuda.empty_cache()
        line["batched"] = batched_measure(s, WORKLOADS["c4"], steps=args.batched_steps, warmup=3, e2e=False,
                                          probe=probe)
    print(json.dumps(line), flush=True)
    s.ctx.close()


def run_streamed(args, w):
    """The workload with its references in pinned HOST memory, streamed
    through the device in blocks by fastid_topk_streamed: FP4 over each
    block's packed rows (the library's AUTO choice), or with --form fp8 each
    block expanded to the FP8 operand, or fp8packed / plain over the rows."""
    import torch
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300 import peaks as P
    from paper_1707_00516_gb300.build import build
    from paper_1707_00516_gb300.search import Searcher, words64
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    gen.build_gpu()
    build()
    probe = P.measure()
    form = args.form if args.form in ("fp8", "fp8packed", "fp4packed", "plain") else "fp4packed"
    s = Searcher(0, getattr(B, FORMS[form][0]))
    sflags = B.REFS_TENSOR if form == "fp8" else 0
    seed = gen.config_seed(w["cfg"])
    n_refs, n_loci, k, T = w["n_refs"], w["n_loci"], w["k"], w["threshold"]
    thr = gen.maf_thresholds(seed, n_loci)
    thr_dev = torch.from_numpy(thr.view(np.int32)).to(dev)
    host = torch.empty((n_refs, words64(n_loci)), dtype=torch.int64, pin_memory=True)
    chunk = min(1 << 20, n_refs)
    alle = torch.empty((chunk, n_loci), dtype=torch.uint8, device=dev)
    packed = torch.empty((chunk, words64(n_loci)), dtype=torch.int64, device=dev)
    for r0 in range(0, n_refs, chunk):
        n = min(chunk, n_refs - r0)
        gen.allele_rows_device(seed, gen.STREAM_DB, thr_dev, alle[:n], row0=r0)
        B.fastid_pack(s.ctx, alle[:n], n_loci, packed[:n])
        host[r0:r0 + n].copy_(packed[:n])
    del alle, packed
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    recipe = recipe_for(args.config, n_refs=n_refs, n_q=w.get("n_q"))
    q, modes = device_queries(s, seed, recipe, thr_dev, n_loci)
    n_q = q.size(0)
    sc = torch.empty((n_q, k), dtype=torch.int32, device=dev)
    ix = torch.empty((n_q, k), dtype=torch.int64, device=dev)
    block = args.streamed
    # host-to-device bandwidth of this machine from pinned memory (1 GiB probe)
    probe_h = host[: (1 << 30) // host.stride(0) // 8]
    probe_d = torch.empty_like(probe_h, device=dev)
    probe_d.copy_(probe_h, non_blocking=True)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for _ in range(3):
        probe_d.copy_(probe_h, non_blocking=True)
    p1.record()
    torch.cuda.synchronize()
    h2d_gbps = 3 * probe_h.numel() * 8 / (p0.elapsed_time(p1) / 1e3) / 1e9
    del probe_d

    def step():
        B.fastid_topk_streamed(s.ctx, host, n_loci, sflags, block, q, modes, k, T, sc, ix)

    r = time_form(args, s, form, step, n_q * n_refs, n_loci, dev, probe)
    # end to end: packed queries in from pinned memory, results out, each step
    hq = q.cpu().pin_memory()
    hm = modes.cpu().pin_memory()
    hs = torch.empty((n_q, k), dtype=torch.int32, pin_memory=True)
    hi = torch.empty((n_q, k), dtype=torch.int64, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q.copy_(hq, non_blocking=True)
        modes.copy_(hm, non_blocking=True)
        step()
        hs.copy_(sc, non_blocking=True)
        hi.copy_(ix, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    n_blocks, done, nxt = 0, 0, max(min(block, n_refs, 256), min(block, n_refs) // 8)
    while done < n_refs:  # the library's block sizes: from block / 8, doubling
        done += min(nxt, n_refs - done)
        nxt = min(min(block, n_refs), 2 * nxt)
        n_blocks += 1
    cfg = workload_config(w)
    cfg.update({"workload": w["workload"] + f"_refs_streamed_from_pinned_host_block{block}", "form": form,
                "blocks_per_step": n_blocks, "host_bytes_per_step": int(host.numel() * 8),
                "h2d_gbps_pinned_probe": h2d_gbps,
                "l2": "inputs larger than L2 (references copied from host every step)"})
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": FORMS[form][2], "data": "synthetic", "config": cfg,
            "e2e": {"value": n_q * n_refs * args.steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(hq.numel() * 8 + hm.numel() + host.numel() * 8),
                    "d2h_bytes_per_step": int(hs.numel() * 4 + hi.numel() * 8)},
            "gpu_launches": r["gpu_launches"], "roofline": r["roofline"], "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)
    s.ctx.close()


def device_queries(s, seed: int, recipe, thr_dev, n_loci: int):
    """Packed queries of a recipe built on the device: contributor alleles from
    gen/gen_gpu.cu, then fastid_pack and fastid_mix."""
    import torch
    dev = s.device
    n_src = recipe.n_sources
    src = torch.empty((max(n_src, 1), n_loci), dtype=torch.uint8, device=dev)
    for stream in (gen.STREAM_DB, gen.STREAM_FRESH):
        sel = np.nonzero(recipe.src_stream == stream)[0]
        if sel.size == 0:
            continue
        rows = torch.from_numpy(recipe.src_row[sel].astype(np.int64)).to(dev)
        tmp = torch.empty((sel.size, n_loci), dtype=torch.uint8, device=dev)
        gen.allele_rows_device(seed, stream, thr_dev, tmp, rows_dev=rows)
        src[torch.from_numpy(sel).to(dev)] = tmp
    q = s.build_queries(src[:n_src], torch.from_numpy(recipe.offsets).to(dev), n_loci).clone()
    return q, torch.from_numpy(recipe.modes).to(dev)


# ----------------------------------------------------------------------------
# Batched workload (configuration 4)
# ----------------------------------------------------------------------------

def _c4_batches(w):
    seed = gen.config_seed(w["cfg"])
    sizes = [int(x) for x in gen.log_uniform_sizes(w["n_batches"], 1, 512, seed, salt=0xC4)]
    rng = np.random.default_rng([seed, 0xC44])
    panels = [int(x) for x in rng.integers(0, len(w["panels"]), w["n_batches"])]
    return seed, sizes, panels


def _c4_recipe(w, b, n, p, seed):
    n_loci = w["panels"][p]
    rec = gen.recipe_mixtures(int(n), w["n_refs"], n_loci, seed + 10 * p, 1, 4, fresh_base=(b + 1) << 24,
                              salt=0xB000 + b)
    rec.modes = np.where(np.diff(rec.offsets) == 1, gen.MODE_MISMATCH, gen.MODE_UNEXPLAINED).astype(np.uint8)
    return rec


def batched_measure(s, w, steps: int, warmup: int, e2e: bool = True, probe: dict | None = None) -> dict:
    """256 batches over 4 loci panels in one persistent launch per step (graph
    replay), variant from the autotuner.  Returns the batched workload's
    figures (throughput, per-replay latency, roofline, clocks)."""
    import torch
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300.batched import BatchedSearch
    from paper_1707_00516_gb300.tune import Autotuner
    dev = s.device
    seed, sizes, panels = _c4_batches(w)
    dbs, thrs = [], []
    for p, n_loci in enumerate(w["panels"]):
        db, thr = build_db(s, seed + 10 * p, w["n_refs"], n_loci, B.REFS_TENSOR | B.REFS_FP4,
                           chunk=(1 << 28) // n_loci)
        dbs.append(db)
        thrs.append(torch.from_numpy(thr.view(np.int32)).to(dev))
    tuner = Autotuner()
    bs = BatchedSearch(s.ctx, dbs, panels, sizes, w["k"], w["threshold"], tuner=tuner)
    host_q, host_m = [], []
    for b, (n, p) in enumerate(zip(sizes, panels)):
        n, p = int(n), int(p)
        rec = _c4_recipe(w, b, n, p, seed)
        q, m = device_queries(s, seed + 10 * p, rec, thrs[p], w["panels"][p])
        bs.set_queries(b, q, m)
        host_q.append(q.cpu().numpy().view(np.uint64))
        host_m.append(m.cpu().numpy())
    torch.cuda.synchronize()
    for _ in range(warmup):
        bs.run_device()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    clk = ClockSampler(dev.index)
    clk.start()
    ev[0].record()
    for i in range(steps):
        bs.run_device()
        ev[i + 1].record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    st = B.fastid_sync_status(s.ctx)
    if st != B.OK:
        raise RuntimeError(f"device status {st}")
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    pairs = int(sum(int(n) * w["n_refs"] for n in sizes))
    flops = float(sum(2.0 * int(n) * w["n_refs"] * w["panels"][p] for n, p in zip(sizes, panels)))
    value = pairs * steps / (total_ms / 1e3)
    from paper_1707_00516_gb300 import peaks as P
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    from paper_1707_00516_gb300.tune import FP4_VARIANTS
    fp4 = bs.variant in FP4_VARIANTS
    peak, unit, how = roof_peak("fp4" if fp4 else "fp8", probe if probe is not None else P.measure(), n_sms)
    achieved = flops * steps / (total_ms / 1e3) / 1e12
    info = bs.plan.info()
    tune_ms = tuner.last_timings or tuner._cache.get(tuner.key(bs.dbs, bs.batches, w["k"]), {}).get("ms", {})
    out = {"workload": w["workload"], "value": value, "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": total_ms / steps,
           "batch_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                                "note": "every batch of a step completes with its graph replay"},
           "config": {"n_batches": int(len(sizes)), "n_queries": int(sum(sizes)), "panels": list(w["panels"]),
                      "n_refs_per_panel": w["n_refs"], "k": w["k"], "variant": int(bs.variant),
                      "autotune_ms": {str(k): v for k, v in tune_ms.items()}, "grid": info["grid"],
                      "units": info["n_units"],
                      "launch": "one persistent launch per step, CUDA graph replay (prep + compare + merge)"},
           "dtype": FORMS["fp4" if fp4 else "fp8"][2], "gpu_launches": 3 * steps,
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": unit,
                        "frac": achieved / peak, "traffic": None, "peak_source": how,
                        "kernel": "tensor_kernel over 4 panels (whole graph time incl. prep and merge)"},
           "clocks": clocks}
    if e2e:
        t0 = time.perf_counter()
        for _ in range(steps):
            _, _, h2d, d2h = bs.run_host(host_q, host_m)
        e2e_s = time.perf_counter() - t0
        out["e2e"] = {"value": pairs * steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h)}
    bs.close()
    for d in dbs:
        d.close()
    return out


def run_c4(args, w):
    """Batched uneven workload alone: one JSON line."""
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300.build import build
    from paper_1707_00516_gb300.search import Searcher
    gen.build_gpu()
    build()
    s = Searcher(0, B.FORM_TENSOR)
    r = batched_measure(s, w, args.steps, args.warmup)
    cfg = {"workload": w["workload"], **r["config"]}
    line = {"metric": METRIC + " (mixed-N panels); p50/p99 batch latency", "value": r["value"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"],
            "data": "synthetic", "config": cfg, "batch_latency_ms": r["batch_latency_ms"], "e2e": r["e2e"],
            "gpu_launches": r["gpu_launches"], "roofline": r["roofline"], "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)
    s.ctx.close()


# ----------------------------------------------------------------------------
# Serving workload (configuration 5)
# ----------------------------------------------------------------------------

# Serving defaults: waves join a running pass over the database's two halves
# and share its launches (serve.SweepServer, parts=2), waves of at most 256
# queries (two query tiles).  Measured at 200 requests/s against 20M x 2048
# (FP4 AUTO, 10 s): p50 / p99 3.07 / 7.88 ms with 2 parts, 3.61 / 8.31 with 4,
# 4.61 / 9.43 with 8; one wave in flight at a time (serve.Server, one slot)
# 2.53 / 6.49 ms -- splitting a pass adds per-launch costs that earlier joining
# does not repay at this load, and the line reports both.  The waves server's
# budget is 4 GB.  Clocks are sampled once a second: the serving window is
# latency-measured, and with the 200 ms sampling of the device-timed configs
# some runs showed a 94-124 ms stall that runs sampled once a second did not.
C5_DEFAULTS = dict(server="sweep", parts=2, slots=1, max_wave=256, hbm_budget=4 << 30, clock_ms=1000)


def c5_requests(w, seed: int, horizon: float):
    """Serving requests over `horizon` seconds: Poisson arrival times (mean
    w["rate"] per second), request sizes log-uniform on 1-256, and one recipe
    of mixtures of 1-5 contributors over all requests' queries in order (a
    single contributor is an individual query, mismatch mode)."""
    rng = np.random.default_rng([seed, 0xC5])
    n_req = int(w["rate"] * horizon * 1.2) + 16
    arrivals = np.cumsum(rng.exponential(1.0 / w["rate"], n_req))
    n_req = int(np.searchsorted(arrivals, horizon))
    arrivals = arrivals[:n_req]
    sizes = gen.log_uniform_sizes(n_req, 1, 256, seed, salt=0xC55)
    rec = gen.recipe_mixtures(int(sizes.sum()), w["n_refs"], w["n_loci"], seed, 1, 5, salt=0xC555)
    rec.modes = np.where(np.diff(rec.offsets) == 1, gen.MODE_MISMATCH, gen.MODE_UNEXPLAINED).astype(np.uint8)
    return arrivals, sizes, rec


def make_server(kind: str, ctx, db, k: int, threshold: int, parts: int, slots: int, max_wave: int,
                hbm_budget: int):
    """The serving layer under test: "sweep" (waves join a running pass over
    the database's parts and share its launches) or "waves" (each wave is one
    fastid_topk on a slot)."""
    from paper_1707_00516_gb300.serve import Server, SweepServer
    if kind == "sweep":
        return SweepServer(ctx, db, k, threshold, parts=parts, capacity=max(4 * max_wave, 1024), max_wave=max_wave)
    return Server(ctx, db, k, threshold, hbm_budget_bytes=hbm_budget, max_wave=max_wave, max_slots=slots)


def serving_measure(s, w, seconds: float, warmup_seconds: float, slots: int, max_wave: int, hbm_budget: int,
                    clock_ms: int, flags: int | None = None, server: str = "sweep", parts: int = 4) -> dict:
    """Poisson arrivals of query batches against a resident 20M database,
    continuous batching (serve.SweepServer or serve.Server), latency from
    submit to result on the host.  Returns the serving figures."""
    import torch
    from paper_1707_00516_gb300 import binding as B
    B.fastid_set_form(s.ctx, B.FORM_AUTO)
    dev = s.device
    seed = gen.config_seed(w["cfg"])
    n_refs, n_loci, k = w["n_refs"], w["n_loci"], w["k"]
    db, thr = build_db(s, seed, n_refs, n_loci, B.REFS_FP4 if flags is None else flags)
    thr_dev = torch.from_numpy(thr.view(np.int32)).to(dev)
    horizon = warmup_seconds + seconds
    arrivals, sizes, rec = c5_requests(w, seed, horizon)
    n_req = arrivals.size
    total = int(sizes.sum())
    q, m = device_queries(s, seed, rec, thr_dev, n_loci)
    hq = q.cpu().numpy().view(np.uint64)
    hm = m.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    srv = make_server(server, s.ctx, db, k, w["threshold"], parts, slots, max_wave, hbm_budget)
    futs = []
    launches0 = None
    B.fastid_profile_read(s.ctx, reset=True)
    t_start = time.perf_counter()
    clk = ClockSampler(dev.index, clock_ms)
    clk.start()
    for i in range(n_req):
        delay = t_start + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        if launches0 is None and arrivals[i] >= warmup_seconds:  # kernel launches from here on
            launches0 = B.fastid_profile_read(s.ctx, reset=False)["all_launches"]
        futs.append(srv.submit(hq[offs[i]:offs[i + 1]], hm[offs[i]:offs[i + 1]]))
    for f in futs:
        f.result(timeout=600)
    t_end = time.perf_counter()
    launches = B.fastid_profile_read(s.ctx, reset=False)["all_launches"] - (launches0 or 0)
    clocks = clk.stop()
    st = srv.stats()
    meas = arrivals >= warmup_seconds
    lat = np.array([l for (ts, l) in srv.records if ts - t_start >= warmup_seconds])
    srv.close()
    served = int(sizes[meas].sum()) * n_refs
    window = (t_end - t_start) - warmup_seconds
    out = {"workload": w["workload"], "value": served / window, "unit": UNIT,
           "offered": float(int(sizes[meas].sum()) * n_refs / seconds),
           "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                          "max": float(lat.max() * 1e3), "from": "submit to result on the host"},
           "config": {"seconds": seconds, "warmup_seconds": warmup_seconds, "requests": int(meas.sum()),
                      "queries": int(sizes[meas].sum()), "server": server, "slots": st["slots"],
                      "steps": st.get("steps"), "waves": st["waves"],
                      "mean_wave_queries": st["mean_wave"], "max_wave": max_wave, "hbm_budget_bytes": hbm_budget},
           "e2e": {"h2d_bytes_per_request": int(hq.nbytes / n_req), "d2h_bytes_per_request": int(12 * k * total / n_req)},
           "gpu_launches": int(launches), "clocks": clocks}
    db.close()
    return out


def run_c5(args, w):
    """Serving alone: one JSON line."""
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300.build import build
    from paper_1707_00516_gb300.search import Searcher
    gen.build_gpu()
    build()
    s = Searcher(0, B.FORM_AUTO)
    r = serving_measure(s, w, args.seconds, args.warmup_seconds, args.slots, args.max_wave, args.hbm_budget,
                        args.clock_ms, server=args.server, parts=args.parts)
    cfg = {"workload": w["workload"], **r["config"], "offered_comparisons_per_s": r["offered"]}
    line = {"metric": METRIC + "; p50/p99 request latency", "value": r["value"], "unit": UNIT,
            "n_gpus": 1, "steps": r["config"]["requests"], "warmup": 0,
            "ms_per_step": 1e3 * args.seconds / max(1, r["config"]["requests"]), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "by wave: " + FORMS["fp8packed"][2],
            "data": "synthetic", "config": cfg, "latency_ms": r["latency_ms"],
            "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": r["e2e"]["h2d_bytes_per_request"],
                    "d2h_bytes_per_step": r["e2e"]["d2h_bytes_per_request"]},
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)
    s.ctx.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1, help="must be 1: one GPU per comparison")
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", default="all",
                    help="all (plain, fp8, fp4) or a comma-separated list of " + ", ".join(FORMS))
    ap.add_argument("--config", choices=sorted(WORKLOADS), default="c3",
                    help="c3 (default): the headline 2048 x 20M workload; c4 batched panels; c5 serving")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="c3: skip the serving and batched sub-objects")
    ap.add_argument("--refs", type=int, default=None,
                    help="override the number of references (smaller captures for profiling)")
    ap.add_argument("--queries", type=int, default=None,
                    help="c1-c3: override the number of queries (the recipe's first N)")
    ap.add_argument("--k", type=int, default=None, help="c1-c3: top-k size instead of the workload's")
    ap.add_argument("--seconds", type=float, default=30.0, help="c5: measured serving time")
    ap.add_argument("--serving-seconds", type=float, default=10.0, help="c3: measured time of the serving sub-run")
    ap.add_argument("--batched-steps", type=int, default=10, help="c3: graph replays of the batched sub-run")
    ap.add_argument("--warmup-seconds", type=float, default=3.0, help="c5: warm-up serving time")
    ap.add_argument("--max-wave", type=int, default=C5_DEFAULTS["max_wave"], help="serving: queries per wave at most")
    ap.add_argument("--hbm-budget", type=int, default=C5_DEFAULTS["hbm_budget"],
                    help="serving: bytes of HBM for in-flight waves")
    ap.add_argument("--server", choices=["sweep", "waves"], default=C5_DEFAULTS["server"],
                    help="serving: waves join a running pass over the database's parts (sweep) or run one "
                         "fastid_topk each on a slot (waves)")
    ap.add_argument("--parts", type=int, default=C5_DEFAULTS["parts"], help="serving (sweep): parts of the database")
    ap.add_argument("--slots", type=int, default=C5_DEFAULTS["slots"], help="serving (waves): waves in flight at most")
    ap.add_argument("--clock-ms", type=int, default=C5_DEFAULTS["clock_ms"],
                    help="serving: nvidia-smi clock sampling interval during the serving window")
    ap.add_argument("--streamed", type=int, default=0, metavar="BLOCK",
                    help="c1-c3: keep the references in pinned host memory and stream them in blocks of BLOCK "
                         "references (fastid_topk_streamed)")

    args = ap.parse_args(argv)
    if args.form != "all":
        bad = [f for f in args.form.split(",") if f not in FORMS]
        if bad:
            ap.error(f"unknown form(s) {bad}; choose from {sorted(FORMS)}")
    w = dict(WORKLOADS[args.config])
    if args.refs:
        w["n_refs"] = args.refs
        w["workload"] = w["workload"].replace("20M", f"{args.refs}").replace("1M", f"{args.refs}")
    if args.queries:
        if "n_q" not in w:
            ap.error("--queries applies to c1, c2 and c3")
        old = w["n_q"]
        w["n_q"] = args.queries
        w["workload"] = w["workload"].replace(f"{old}q_", f"{args.queries}q_").replace(f"{old}mix_",
                                                                                       f"{args.queries}mix_")
    if args.k:
        if "n_q" not in w:
            ap.error("--k applies to c1, c2 and c3")
        w["workload"] = w["workload"].replace(f"top{w['k']}", f"top{args.k}")
        w["k"] = args.k
    if args.impl == "reference":
        run_reference(args, w)
        return
    refuse_multi_gpu(args)
    if args.config == "c4":
        run_c4(args, w)
    elif args.config == "c5":
        run_c5(args, w)
    elif args.streamed:
        run_streamed(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
