#!/usr/bin/env python3
"""FastID all-pairs comparison benchmark on GB300.

Metric: query x reference comparisons per second at N loci, bit-exact
(results are checked against the CPU oracle on a sample by the tests and by
--check here).  One step = one pass of the whole path over one batch of
queries: pack the queries' contributor alleles, build the mixtures (OR),
compare every query with every resident reference and reduce to the
per-query top-k under a threshold.  The reference database is resident in
HBM (loaded once, outside the timed region).

Default workload: 2048 unknowns (1024 individuals, 1024 mixtures of 2-5
people) x 20,000,000 references, N = 2048 loci, top-32, threshold 512.

    python bench.py [--steps K] [--warmup W] [--form plain|tensor|both]
    python bench.py --impl reference ...   (the CPU oracle on a bounded sample)
    torchrun --nproc-per-node N bench.py --gpus N   (N independent replicas)

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import os
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
               k=32, threshold=512, cfg=3),
    "c2": dict(workload="2048mix_x_1M_refs_N4096_top16_T0", n_q=2048, n_refs=1_000_000, n_loci=4096,
               k=16, threshold=0, cfg=2),
    "c1": dict(workload="64q_x_10k_refs_N1024_full_uint16_matrices", n_q=64, n_refs=10_000, n_loci=1024,
               k=32, threshold=0xFFFFFFFF, cfg=1),
    "c4": dict(workload="256_batches_1-512q_panels_N512-2048-8192-16384_x_4M_refs_top16", n_refs=4_000_000,
               panels=(512, 2048, 8192, 16384), n_batches=256, k=16, threshold=0xFFFFFFFF, cfg=4),
    "c5": dict(workload="serving_poisson200bps_1-256q_N2048_x_20M_refs_top16", n_refs=20_000_000, n_loci=2048,
               rate=200.0, k=16, threshold=0xFFFFFFFF, cfg=5),
}

METRIC = "query x reference comparisons/s at N loci, bit-exact"
UNIT = "comparisons/s"

# Peak popcount rate of the plain form's bound: POPC issues 16 results per
# clock per SM (integer-pipe throughput table for compute capability 10.x),
# 152 SMs, at the maximum SM clock.
POPC_PER_CLK_PER_SM = 16
# Dense e4m3 tensor rate relative to bf16 (nominal 4.5 vs 2.25 PFLOP/s).
FP8_OVER_BF16 = 2.0


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


# ----------------------------------------------------------------------------
# Distributed helpers (independent replicas; barrier + max over ranks only)
# ----------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(backend: str):
    import torch.distributed as dist
    world, rank, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return world, rank


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# CPU oracle legs
# ----------------------------------------------------------------------------

def oracle_sample_step(q_alleles: np.ndarray, modes: np.ndarray, seed: int, n_refs: int, thr: np.ndarray,
                       sample_rows: np.ndarray, k: int, threshold: int):
    """The oracle on a bounded sample: every query against the sampled
    references (per-locus scores, then top-k over the sample)."""
    import oracle
    R = gen.allele_rows(seed, gen.STREAM_DB, sample_rows, thr)
    t0 = time.perf_counter()
    mis, une = oracle.scores(R, q_alleles)
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
    return {"value": q.shape[0] * S / t, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"all {q.shape[0]} queries x {S} sampled references (per-locus scores + top-{w['k']}), "
                      f"{t:.1f} s"}


def run_reference(args, w):
    """--impl reference: the CPU oracle, each step a bounded sample."""
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
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
            "data": "synthetic", "config": {"workload": w["workload"], "n_loci": w["n_loci"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
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
    # profiles/tensor_kernel_c3_2048x20M.md: dram__bytes_read.sum 157.24 GB + dram__bytes_write.sum 79.17 MB
    "tensor/c3": (157.2376e9 + 79.17e6, "d71ef4c0a9ea8d21"),
    # profiles/plain_kernel_c3_2048x20M.md: dram__bytes_read.sum 20.39 GB + dram__bytes_write.sum 17.27 MB
    "plain/c3": (20.3915e9 + 17.27e6, "c528944b13d66b2a"),
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def form_code(args, form_name):
    """FASTID_FORM_* of a bench form: plain, or the tensor form over the FP8
    copy (default) or over the packed rows (--operand packed)."""
    from paper_1707_00516_gb300 import binding as B
    if form_name == "plain":
        return B.FORM_PLAIN
    return B.FORM_TENSOR_PACKED if args.operand == "packed" else B.FORM_TENSOR


def time_form(args, s, db, form_name, step_fn, pairs_per_step, n_loci, world, dev):
    """Warm up and time `args.steps` steps of one compute form; returns the
    device-timed result and the roofline of its main compare kernel."""
    import torch
    from paper_1707_00516_gb300 import binding as B
    B.fastid_set_form(s.ctx, form_code(args, form_name))
    for _ in range(args.warmup):
        step_fn()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index)
    clk.start()
    B.fastid_profile(s.ctx, True)
    B.fastid_profile_read(s.ctx, reset=True)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world, dev)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step_fn()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world, dev)
    ms = e0.elapsed_time(e1)
    prof = B.fastid_profile_read(s.ctx, reset=True)
    B.fastid_profile(s.ctx, False)
    clocks = clk.stop()
    st = B.fastid_sync_status(s.ctx)
    if st != B.OK:
        raise RuntimeError(f"device status {st} after the timed region ({form_name})")
    ms_max = max_over_ranks(ms, world, dev)
    value = pairs_per_step * args.steps * world / (ms_max / 1e3)

    peaks, peak_src = load_peaks()
    main_s = prof["main_ms"] / max(1, prof["main_launches"]) / 1e3
    # compare launches per step (several when references stream in blocks)
    main_per_step = max(1, prof["main_launches"]) / args.steps
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if form_name == "plain":
        words32 = 2 * ((n_loci + 63) // 64)
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak = POPC_PER_CLK_PER_SM * n_sms * sm_max * 1e6 / 1e12
        achieved = pairs_per_step * words32 / (main_s * main_per_step) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tpopc/s",
                "kernel": "plain_kernel<EPI_TOPK>",
                "peak_source": f"{POPC_PER_CLK_PER_SM} POPC/clk/SM x {n_sms} SMs x {sm_max:.0f} MHz "
                               f"(max SM clock, {peak_src})"}
    else:
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        peak = bf16 * FP8_OVER_BF16
        achieved = 2.0 * pairs_per_step * n_loci / (main_s * main_per_step) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "kernel": "tensor_kernel (tcgen05 kind::f8f6f4, EPI_TOPK" +
                          (", packed rows expanded on chip)" if args.operand == "packed" else ")"),
                "peak_source": f"bf16 dense burst {bf16:.1f} TFLOP/s ({peak_src}) x {FP8_OVER_BF16:g} "
                               f"(nominal e4m3/bf16 dense ratio, 4.5/2.25 PFLOP/s)"}
    roof["frac"] = achieved / peak
    roof["kernel_ms"] = main_s * 1e3
    key = f"{form_name}/{args.config}"
    # the captured counters hold for the unmodified workload only
    tr = None if (args.refs or args.queries or args.operand != "fp8") else NCU_TRAFFIC.get(key)
    roof["traffic"] = tr[0] if tr and tr[1] == kernel_source_hash(form_name) else None
    return {"value": value, "ms_per_step": ms_max / args.steps, "roofline": roof, "clocks": clocks,
            "gpu_launches": int(prof["all_launches"])}


def run_gpu(args, w):
    import torch
    world, rank = dist_init("nccl")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300.search import Searcher
    from paper_1707_00516_gb300.build import build
    gen.build_gpu()
    build()

    forms = ["plain", "tensor"] if args.form == "both" else [args.form]
    s = Searcher(local, B.FORM_AUTO)
    seed = gen.config_seed(w["cfg"])
    n_refs, n_loci, k, T = w["n_refs"], w["n_loci"], w["k"], w["threshold"]
    flags = B.REFS_TENSOR if "tensor" in forms and args.operand == "fp8" else 0
    db, thr = build_db(s, seed, n_refs, n_loci, flags)
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
    res = {f: time_form(args, s, db, f, step, pairs_per_step, n_loci, world, dev) for f in forms}
    head = max(res, key=lambda f: res[f]["value"])
    hr = res[head]

    # end to end through the host-buffer API, headline form
    B.fastid_set_form(s.ctx, form_code(args, head))
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
    barrier(world, dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h2d, d2h = e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = pairs_per_step * args.steps * world / e2e_s

    line = {"metric": METRIC, "value": hr["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": hr["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32" if head == "plain" else "e4m3xe4m3->f32",
            "data": "synthetic",
            "config": {"workload": w["workload"], "n_queries": n_q, "n_refs": n_refs, "n_loci": n_loci, "k": k,
                       "threshold": T, "form": head, "operand": args.operand if head == "tensor" else None,
                       "parallelism": f"replicas{world}",
                       "output": "both full uint16 score matrices (both scores of every pair)" if full
                       else "per-query top-k",
                       "l2": "inputs larger than L2 (packed database %.2f GB%s)" % (
                           n_refs * n_loci / 8 / 1e9,
                           ", e4m3 copy %.1f GB" % (n_refs * n_loci / 1e9) if flags else "")},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": hr["gpu_launches"], "roofline": hr["roofline"], "clocks": hr["clocks"],
            "forms": {f: {"value": r["value"], "ms_per_step": r["ms_per_step"], "roofline": r["roofline"],
                          "clocks": r["clocks"]} for f, r in res.items()}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, recipe, thr)
    if rank == 0:
        print(json.dumps(line), flush=True)
    db.close()
    s.ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_streamed(args, w):
    """The workload with its references in pinned HOST memory, streamed
    through the device in blocks by fastid_topk_streamed (tensor form)."""
    import torch
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300.build import build
    from paper_1707_00516_gb300.search import Searcher, words64
    world, rank = dist_init("nccl")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gen.build_gpu()
    build()
    s = Searcher(local, B.FORM_TENSOR)
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
        B.fastid_topk_streamed(s.ctx, host, n_loci, B.REFS_TENSOR, block, q, modes, k, T, sc, ix)

    r = time_form(args, s, None, "tensor", step, n_q * n_refs, n_loci, world, dev)
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
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    n_blocks, done, nxt = 0, 0, max(min(block, n_refs, 256), min(block, n_refs) // 8)
    while done < n_refs:  # the library's block sizes: from block / 8, doubling
        done += min(nxt, n_refs - done)
        nxt = min(min(block, n_refs), 2 * nxt)
        n_blocks += 1
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "e4m3xe4m3->f32", "data": "synthetic",
            "config": {"workload": w["workload"] + f"_refs_streamed_from_pinned_host_block{block}",
                       "n_queries": n_q, "n_refs": n_refs, "n_loci": n_loci, "k": k, "threshold": T,
                       "blocks_per_step": n_blocks, "host_bytes_per_step": int(host.numel() * 8),
                       "h2d_gbps_pinned_probe": h2d_gbps,
                       "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (references copied from host every step)"},
            "e2e": {"value": n_q * n_refs * args.steps * world / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(hq.numel() * 8 + hm.numel() + host.numel() * 8),
                    "d2h_bytes_per_step": int(hs.numel() * 4 + hi.numel() * 8)},
            "gpu_launches": r["gpu_launches"], "roofline": r["roofline"], "clocks": r["clocks"]}
    if rank == 0:
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


def run_c4(args, w):
    """Batched uneven workload: 256 batches over 4 loci panels in one
    persistent launch (graph replay), variant from the autotuner."""
    import torch
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300.batched import BatchedSearch
    from paper_1707_00516_gb300.build import build
    from paper_1707_00516_gb300.search import Searcher
    from paper_1707_00516_gb300.tune import Autotuner
    gen.build_gpu()
    build()
    dev = torch.device("cuda", 0)
    s = Searcher(0, B.FORM_TENSOR)
    seed, sizes, panels = _c4_batches(w)
    dbs, thrs = [], []
    for p, n_loci in enumerate(w["panels"]):
        db, thr = build_db(s, seed + 10 * p, w["n_refs"], n_loci, B.REFS_TENSOR, chunk=(1 << 28) // n_loci)
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
    for _ in range(args.warmup):
        bs.run_device()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    clk = ClockSampler(0)
    clk.start()
    ev[0].record()
    for i in range(args.steps):
        bs.run_device()
        ev[i + 1].record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    st = B.fastid_sync_status(s.ctx)
    if st != B.OK:
        raise RuntimeError(f"device status {st}")
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    pairs = int(sum(int(n) * w["n_refs"] for n in sizes))
    flops = float(sum(2.0 * int(n) * w["n_refs"] * w["panels"][p] for n, p in zip(sizes, panels)))
    value = pairs * args.steps / (total_ms / 1e3)
    peaks, peak_src = load_peaks()
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    achieved = flops * args.steps / (total_ms / 1e3) / 1e12
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, _, h2d, d2h = bs.run_host(host_q, host_m)
    e2e_s = time.perf_counter() - t0
    info = bs.plan.info()
    line = {"metric": METRIC + " (mixed-N panels); p50/p99 batch latency", "value": value, "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "e4m3xe4m3->f32",
            "data": "synthetic",
            "config": {"workload": w["workload"], "n_batches": int(len(sizes)), "n_queries": int(sum(sizes)),
                       "panels": list(w["panels"]), "n_refs_per_panel": w["n_refs"], "k": w["k"],
                       "variant": int(bs.variant), "autotune_ms": {str(k): v for k, v in tuner.last_timings.items()},
                       "grid": info["grid"], "units": info["n_units"], "launch": "one persistent launch per step, "
                       "CUDA graph replay (prep + compare + merge)"},
            "batch_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "e2e": {"value": pairs * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": 3 * args.steps,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16 * FP8_OVER_BF16, "unit": "TFLOP/s",
                         "frac": achieved / (bf16 * FP8_OVER_BF16), "traffic": None,
                         "kernel": "tensor_kernel over 4 panels (whole graph time incl. prep and merge)",
                         "peak_source": f"bf16 dense burst {bf16:.1f} TFLOP/s ({peak_src}) x {FP8_OVER_BF16:g}"},
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    bs.close()
    for d in dbs:
        d.close()
    s.ctx.close()


# Serving defaults: one wave in flight (a wave of up to 128 queries costs about
# the same as a wave of one, so arrivals are best coalesced into the next wave)
# of at most 256 queries (two query tiles), in a 4 GB budget.  Clocks are
# sampled once a second: the serving window is latency-measured, and with the
# 200 ms sampling of the device-timed configs some runs showed a 94-124 ms
# stall (p99 23-25 ms) that runs sampled once a second did not (p99 15.7 ms).
C5_DEFAULTS = dict(slots=1, max_wave=256, hbm_budget=4 << 30, clock_ms=1000)


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


def run_c5(args, w):
    """Serving: Poisson arrivals of query batches against a resident 20M
    database, continuous batching, p50/p99 request latency."""
    import torch
    from paper_1707_00516_gb300 import binding as B
    from paper_1707_00516_gb300.build import build
    from paper_1707_00516_gb300.search import Searcher
    from paper_1707_00516_gb300.serve import Server
    gen.build_gpu()
    build()
    dev = torch.device("cuda", 0)
    s = Searcher(0, B.FORM_AUTO)  # FP8 operand for large waves, packed rows for small ones
    seed = gen.config_seed(w["cfg"])
    n_refs, n_loci, k = w["n_refs"], w["n_loci"], w["k"]
    db, thr = build_db(s, seed, n_refs, n_loci, B.REFS_TENSOR)
    thr_dev = torch.from_numpy(thr.view(np.int32)).to(dev)
    horizon = args.warmup_seconds + args.seconds
    arrivals, sizes, rec = c5_requests(w, seed, horizon)
    n_req = arrivals.size
    total = int(sizes.sum())
    q, m = device_queries(s, seed, rec, thr_dev, n_loci)
    hq = q.cpu().numpy().view(np.uint64)
    hm = m.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    srv = Server(s.ctx, db, k, w["threshold"], hbm_budget_bytes=args.hbm_budget, max_wave=args.max_wave,
                 max_slots=args.slots)
    futs, t_sub = [], []
    launches0 = None
    B.fastid_profile_read(s.ctx, reset=True)
    t_start = time.perf_counter()
    clk = ClockSampler(0, args.clock_ms)
    clk.start()
    for i in range(n_req):
        delay = t_start + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        if launches0 is None and arrivals[i] >= args.warmup_seconds:  # kernel launches from here on
            launches0 = B.fastid_profile_read(s.ctx, reset=False)["all_launches"]
        futs.append(srv.submit(hq[offs[i]:offs[i + 1]], hm[offs[i]:offs[i + 1]]))
    for f in futs:
        f.result(timeout=600)
    t_end = time.perf_counter()
    launches = B.fastid_profile_read(s.ctx, reset=False)["all_launches"] - (launches0 or 0)
    clocks = clk.stop()
    st = srv.stats()
    # measured window: requests that arrived after the warm-up
    meas = arrivals >= args.warmup_seconds
    lat = np.array([l for (ts, l) in srv.records if ts - t_start >= args.warmup_seconds])
    srv.close()
    served = int(sizes[meas].sum()) * n_refs
    window = (t_end - t_start) - args.warmup_seconds
    line = {"metric": METRIC + "; p50/p99 request latency", "value": served / window, "unit": UNIT,
            "n_gpus": 1, "steps": int(meas.sum()), "warmup": int((~meas).sum()),
            "ms_per_step": 1e3 * window / max(1, int(meas.sum())), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "e4m3xe4m3->f32", "data": "synthetic",
            "config": {"workload": w["workload"], "seconds": args.seconds, "requests": n_req,
                       "queries": total, "offered_comparisons_per_s": float(total * n_refs / horizon),
                       "slots": st["slots"], "waves": st["waves"], "mean_wave_queries": st["mean_wave"],
                       "max_wave": args.max_wave, "hbm_budget_bytes": args.hbm_budget},
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                           "max": float(lat.max() * 1e3)},
            "e2e": {"value": served / window, "unit": UNIT, "h2d_bytes_per_step": int(hq.nbytes / n_req),
                    "d2h_bytes_per_step": int(12 * k * total / n_req)},
            "gpu_launches": int(launches), "clocks": clocks}
    print(json.dumps(line), flush=True)
    db.close()
    s.ctx.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["plain", "tensor", "both"], default="both")
    ap.add_argument("--config", choices=sorted(WORKLOADS), default="c3",
                    help="c3 (default): the headline 2048 x 20M workload; c4 batched panels; c5 serving")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--refs", type=int, default=None,
                    help="override the number of references (smaller captures for profiling)")
    ap.add_argument("--queries", type=int, default=None,
                    help="c1-c3: override the number of queries (the recipe's first N)")
    ap.add_argument("--operand", choices=["fp8", "packed"], default="fp8",
                    help="c1-c3, tensor form: reference operand read from the FP8 copy or from the packed rows "
                         "(expanded on chip)")
    ap.add_argument("--seconds", type=float, default=30.0, help="c5: measured serving time")
    ap.add_argument("--warmup-seconds", type=float, default=3.0, help="c5: warm-up serving time")
    ap.add_argument("--max-wave", type=int, default=C5_DEFAULTS["max_wave"], help="c5: queries per wave at most")
    ap.add_argument("--hbm-budget", type=int, default=C5_DEFAULTS["hbm_budget"],
                    help="c5: bytes of HBM for in-flight waves")
    ap.add_argument("--slots", type=int, default=C5_DEFAULTS["slots"], help="c5: waves in flight at most")
    ap.add_argument("--clock-ms", type=int, default=C5_DEFAULTS["clock_ms"],
                    help="c5: nvidia-smi clock sampling interval during the serving window")
    ap.add_argument("--streamed", type=int, default=0, metavar="BLOCK",
                    help="c1-c3: keep the references in pinned host memory and stream them in blocks of BLOCK "
                         "references (fastid_topk_streamed)")

    args = ap.parse_args(argv)
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
    if args.operand == "packed":
        w["workload"] += "_packed_operand"
    if args.impl == "reference":
        run_reference(args, w)
    elif args.config == "c4":
        run_c4(args, w)
    elif args.config == "c5":
        run_c5(args, w)
    elif args.streamed:
        run_streamed(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
