#!/usr/bin/env python
"""Benchmark of all-pairs support counting over BatMaps (frequent pair mining).

One step = the whole hot path on one instance whose tidlists are already in
HBM: BatMap build (sizes, 2-of-3 placement, bytes, failed insertions and
their corrections, compare schedule), the all-pairs compare, the failure
correction and the support-threshold compaction, ending with the number of
frequent pairs on the host.  The metric is pair supports per second
(n(n-1)/2 per step).

Default workload: the density sweep at scale, m = 4,194,304 transactions,
n = 8,192 items, Bernoulli density 5% (1.7e9 tids, 12.9 GB of BatMaps, all
33,550,336 pair supports); inputs exceed the 129 MB L2, so no flush is
needed.  The same line carries, as sub-records, the Zipf workload (m = 10^6,
n = 2,000) and the batched form against plain per-instance calls on 64
instances of uneven size.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle on the same metric

Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen  # noqa: E402

METRIC = "item-pair supports/sec and achieved HBM GB/s, batched vs plain, bit-exact"
UNIT = "pair-supports/s"
WORKLOAD_DESC = {
    "bern_m10k_n200": "plain frequent pair mining, m=10,000, n=200, Bernoulli p=0.05, s=25",
    "zipf_m1m_n2000": "plain all-pairs mining, m=1,000,000, n=2,000, Zipf(1) items at mean density 2%, s=1,000",
    "bern_m4m_n8192_p0.1": "density sweep, m=4,194,304, n=8,192, Bernoulli p=0.001",
    "bern_m4m_n8192_p1": "density sweep, m=4,194,304, n=8,192, Bernoulli p=0.01",
    "bern_m4m_n8192_p5": "density sweep, m=4,194,304, n=8,192, Bernoulli p=0.05",
}
OPS_PER_WORD_PAIR = 4  # LOP3, IADD, LOP3, IDP4A per 32-bit word pair
WITNESS_OPS = 5        # per word-triple against the pair's prepared pattern: 2 masked XORs, IADD, AND-NOT, IDP4A


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _traffic_record(workload: str, kernel: str = "k_compare", source: str = "compare.cu"):
    """DRAM bytes per launch of a kernel from a committed ncu record
    (profiles/*traffic*.json: kernel, workload, SHA-256 of the kernel's source
    file), or None if no record matches this workload or the source changed
    since the counters were taken."""
    import glob
    src = open(os.path.join(ROOT, "paper_1102_1003_gb300", "csrc", source), "rb").read()
    digest = hashlib.sha256(src).hexdigest()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*traffic*.json"))):
        try:
            rec = json.load(open(path))
        except (OSError, ValueError):
            continue
        if (rec.get("kernel") == kernel and rec.get("workload") == workload
                and rec.get(source.replace(".", "_") + "_sha256") == digest):
            return rec
    return None


def _traffic(workload: str, kernel: str = "k_compare", source: str = "compare.cu"):
    rec = _traffic_record(workload, kernel, source)
    return rec["traffic_bytes_per_launch"] if rec else None


def max_over_ranks(value: float, device=None) -> float:
    """The job's time is the slowest rank's: all-reduce(MAX) across the process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sample_pairs(n, k, seed):
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, k)
    j = rng.integers(0, n - 1, k)
    j = np.where(j >= i, j + 1, j)
    return np.minimum(i, j), np.maximum(i, j)


def cpu_oracle_rate(inst, seconds: float, seed: int = 0):
    """Oracle pair supports/s on a uniform sample of the workload's pairs, run on
    all host cores (the same single-threaded merge on disjoint blocks)."""
    import oracle
    cores = os.cpu_count() or 1
    n = inst.n
    k = 2000
    t0 = time.perf_counter()
    ii, jj = _sample_pairs(n, k, seed)
    oracle.pairs_list(inst.offsets, inst.tids, ii, jj, threads=cores)
    dt = max(time.perf_counter() - t0, 1e-6)
    k = int(min(max(k * seconds / dt, 2000), n * (n - 1) // 2))
    ii, jj = _sample_pairs(n, k, seed + 1)
    t0 = time.perf_counter()
    oracle.pairs_list(inst.offsets, inst.tids, ii, jj, threads=cores)
    dt = time.perf_counter() - t0
    return k / dt, cores, k, dt


def merge_micro(n: int = 1 << 24, repeats: int = 5):
    """Sec. IV-B's merging experiment on this host: count the identical elements
    of two sorted arrays of n 32-bit integers with the oracle's single-threaded
    merge, on one core and as simultaneous runs on every core.  Returns set
    elements (2 n per merge) per second for both."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    a, b = datagen.sorted_u32(n, 1), datagen.sorted_u32(n, 2)
    common = oracle.intersect_count(a, b)
    assert common == np.intersect1d(a, b, assume_unique=True).size
    t0 = time.perf_counter()
    for _ in range(repeats):
        oracle.intersect_count(a, b)
    one = 2 * n * repeats / (time.perf_counter() - t0)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:  # ctypes releases the GIL during each merge
        list(ex.map(lambda _: [oracle.intersect_count(a, b) for _ in range(repeats)], range(cores)))
    par = 2 * n * repeats * cores / (time.perf_counter() - t0)
    return {"n": n, "repeats": repeats, "elements_per_s_1core": one, "elements_per_s_all_cores": par,
            "cores": cores, "common": int(common),
            "inputs": "two sorted uint32 arrays, gaps uniform in [1, 255], seeds 1 and 2",
            "paper_context": "Sec. IV-B on its own CPU: 2.25e8 elements/s on one core, 1.71e9 on 8"}


def run_reference(args, inst, rank, world):
    if rank != 0:
        return
    per_step = max(2.0, min(8.0, 150.0 / max(args.steps + args.warmup, 1)))
    for w in range(args.warmup):
        cpu_oracle_rate(inst, per_step / 4, seed=100 + w)
    rates, times, samples, cores = [], [], 0, 1
    for k in range(args.steps):
        r, cores, kk, dt = cpu_oracle_rate(inst, per_step, seed=1000 + k)
        rates.append(r)
        times.append(dt)
        samples += kk
    total_t = sum(times)
    value = samples / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": {"workload": args.workload, "desc": WORKLOAD_DESC[args.workload],
                                        "m": inst.m, "n": inst.n, "s": inst.s, "pairs": inst.n * (inst.n - 1) // 2},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{samples} uniformly sampled pairs over {args.steps} steps "
                                   "(single-threaded sorted merge on disjoint blocks, one per core)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def dense_leg(args, inst, off, tids, n_out_ref, peaks, peak_kind, steps=None, warmup=None, workload=None):
    """The dense-bitmap tensor-core comparison path on the same workload."""
    import torch
    import paper_1102_1003_gb300 as pkg
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    npairs = inst.n * (inst.n - 1) // 2
    pairs = torch.empty((max(n_out_ref, 1), 3), dtype=torch.int32, device=off.device)
    for _ in range(warmup):
        pkg.pair_support_dense(inst.m, off, tids, inst.s, pairs=pairs)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    gemm, build = [], []
    ev0.record(stream)
    for _ in range(steps):
        k, _, t = pkg.pair_support_dense(inst.m, off, tids, inst.s, pairs=pairs)
        gemm.append(t["compare_ms"])
        build.append(t["build_ms"])
    ev1.record(stream)
    torch.cuda.synchronize()
    assert k == n_out_ref, (k, n_out_ref)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    # tensor work actually issued: upper-triangle blocks of two 128 x 256 tiles over the padded K
    n, bm, bn = inst.n, 128, 256
    tiles = 2 * sum(min((n + 2 * bm - 1) // (2 * bm), bj + 1) for bj in range((n + bn - 1) // bn))
    kpad = (inst.m + 127) // 128 * 128
    flops_issued = 2.0 * tiles * bm * bn * kpad
    flops_alg = 2.0 * npairs * inst.m  # 2 m per pair i < j
    g = statistics.mean(gemm) / 1e3
    # e4m3 dense peak: the measured bf16 peak x the nominal fp8 / bf16 ratio (4.5 / 2.25)
    peak = 2.0 * peaks.get("bf16_tflops", 1900.0)
    return {"value": npairs * steps / elapsed, "unit": UNIT, "ms_per_step": 1e3 * elapsed / steps,
            "phases_ms": {"bitmap": statistics.mean(build), "tensor_kernel": statistics.mean(gemm)},
            "roofline": {"bound": "tensor", "achieved": flops_alg / g / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops_alg / g / 1e12 / peak, "kernel": "k_dense_mmt",
                         "traffic": _traffic(workload or args.workload, "k_dense_mmt", "dense.cu"),
                         "peak_kind": f"e4m3 dense = 2 x {peak_kind} bf16 burst (nominal 4.5/2.25 ratio)",
                         "algorithmic_flops": "2 m n(n-1)/2 (pairs i < j only)",
                         "issued_definition": "two 128 x 256 tiles per upper-triangle block (diagonal "
                                              "blocks included) over the padded K",
                         "issued_TFLOPs": flops_issued / g / 1e12,
                         "issued_frac": flops_issued / g / 1e12 / peak},
            "dtype": "e4m3 {0,1} operands, fp32 accumulate (exact integers < 2^24)"}


def _desc(workload: str) -> str:
    base, _, first = workload.partition("_first")
    return WORKLOAD_DESC[base] + (f", first {first} items only (profiling case)" if first else "")


def _alu_peak(dev, peaks):
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12, sms


PROBE_LOG = 0  # batmap_params.probe_log of the timed builds (0 = the library's default)


def _build_params():
    """Build parameters of the timed BatMap builds: the defaults, with
    probe_log from --probe-log."""
    import paper_1102_1003_gb300 as pkg
    return pkg.batmap_default_params(probe_log=PROBE_LOG)


def plain_leg(inst, dev, steps, warmup, peaks, peak_kind, workload, sampler=None, dist=None):
    """Time `steps` plain steps (batmap_build + pair_support_all) on resident tidlists."""
    import torch
    import paper_1102_1003_gb300 as pkg
    from paper_1102_1003_gb300 import batmap as B
    L = pkg.load_library()
    off = torch.from_numpy(inst.offsets.astype(np.int64)).to(dev)
    tids = torch.from_numpy(inst.tids.view(np.int32)).to(dev)
    npairs = inst.n * (inst.n - 1) // 2
    bset = pkg.batmap_build(inst.m, off, tids, None, params=_build_params())
    n_out, _ = pkg.pair_support_all(bset, inst.s)
    info = bset.info
    bset.free()
    pairs_buf = torch.empty((max(n_out, 1), 3), dtype=torch.int32, device=dev)
    timing = B.batmap_timing()
    compare_ms, build_ms, compact_ms, scan_ms, probe_ms = [], [], [], [], []

    def step(record):
        bs = pkg.batmap_build(inst.m, off, tids, None, params=_build_params())
        k, _ = pkg.pair_support_all(bs, inst.s, pairs=pairs_buf)
        if record:
            L.batmap_get_timing(bs.handle, ctypes.byref(timing))
            compare_ms.append(timing.compare_ms)
            scan_ms.append(timing.scan_ms)
            probe_ms.append(timing.probe_ms)
            build_ms.append(timing.build_ms)
            compact_ms.append(timing.compact_ms)
        bs.free()
        return k

    for _ in range(warmup):
        step(False)
    if sampler:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = L.batmap_kernel_launches()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        got = step(True)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = L.batmap_kernel_launches() - launches0
    elapsed = ev0.elapsed_time(ev1) / 1e3
    if dist:
        elapsed = max_over_ranks(elapsed, dev)
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    assert got == n_out
    cmp_s = statistics.mean(compare_ms) / 1e3
    scan_s = statistics.mean(scan_ms) / 1e3
    wp = info["word_pairs"]
    wp_probe = info["probe_word_pairs"]
    wp_scan = wp - wp_probe
    alu_peak, sms = _alu_peak(dev, peaks)
    achieved = OPS_PER_WORD_PAIR * wp_scan / scan_s / 1e12
    logical_gbs = 8.0 * wp / cmp_s / 1e9
    rec = {
        "value": npairs * steps / elapsed, "unit": UNIT, "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * elapsed / steps, "elapsed_s": elapsed,
        "config": {"workload": workload, "desc": _desc(workload), "m": inst.m, "n": inst.n,
                   "s": inst.s, "pairs": npairs, "tids": int(inst.tids.size), "batmap_bytes": info["bytes"],
                   "width_classes": info["n_classes"], "l2": "inputs larger than L2 (no flush)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                     "frac": achieved / alu_peak, "kernel": "k_compare",
                     "traffic": _traffic(workload),
                     "peak_kind": f"{sms} SMs x 128 INT32 lanes x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz "
                                  f"({peak_kind} max clock)",
                     "algorithmic_ops": f"{OPS_PER_WORD_PAIR} x {wp_scan:.4g} word pairs (the scan-routed pairs' "
                                        f"max(|B_i|,|B_j|)/4) per scan time {1e3 * scan_s:.3f} ms"},
        "logical_hbm": {"achieved_GBps": logical_gbs, "peak_GBps": peaks["hbm_gbs"],
                        "frac": logical_gbs / peaks["hbm_gbs"],
                        "definition": "sum over pairs of 2*max(|B_i|,|B_j|) bytes / compare time (Sec. IV-A)"},
        "set_elements_per_s": (inst.n - 1) * int(inst.tids.size) / cmp_s,
        "phases_ms": {"build": statistics.mean(build_ms), "compare": statistics.mean(compare_ms),
                      "compare_scan": statistics.mean(scan_ms), "compare_probe": statistics.mean(probe_ms),
                      "correct_compact": statistics.mean(compact_ms)},
        "frequent_pairs": n_out, "failed_insertions": info["n_failed"], "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if wp_probe > 0:
        probe_s = statistics.mean(probe_ms) / 1e3
        rec["compare_equiv"] = {
            "frac": OPS_PER_WORD_PAIR * wp / cmp_s / 1e12 / alu_peak,
            "definition": "the whole compare step (scan + probe kernels) on the scan's work for every pair: "
                          "4 x sum over pairs of max(|B_i|,|B_j|)/4 / compare time / lane-op peak"}
        rec["probe"] = {
            "kernel": "k_pair_probe", "ms": 1e3 * probe_s, "routed_word_pairs": wp_probe,
            "routed_share": wp_probe / wp, "words_read": info["probe_words"],
            "scan_equivalent_frac": OPS_PER_WORD_PAIR * wp_probe / probe_s / 1e12 / alu_peak,
            "definition": "pairs whose BatMap widths differ by 2^probe_log or more (default 4x) are eligible; "
                          "per width class the scheduler's cost model picks the rows it counts by probing the "
                          "narrower BatMap's nonempty slots; routed_word_pairs is the scan's work for them "
                          "(max(|B_i|,|B_j|)/4 per pair), words_read the probe's (min(|B_i|,|B_j|)/4 per "
                          "pair); scan_equivalent_frac = 4 x routed_word_pairs / probe time / lane-op peak",
            "traffic": _traffic(workload, "k_pair_probe"),
        }
    return rec, off, tids, n_out


def run_mine(args, inst, rank, world):
    import torch
    import paper_1102_1003_gb300 as pkg

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.load_library()
    peaks, peak_kind = _peaks()
    npairs = inst.n * (inst.n - 1) // 2
    label = args.workload if not args.scale_n else f"{args.workload}_first{args.scale_n}"
    rec, off, tids, n_out = plain_leg(inst, dev, args.steps, args.warmup, peaks, peak_kind, label,
                                      sampler=ClockSampler(local), dist=dist)

    # end to end through the C ABI from pinned host buffers (library-made permutations)
    h_off = torch.from_numpy(inst.offsets.astype(np.uint64).view(np.int64)).pin_memory().numpy().view(np.uint64)
    h_tids = torch.from_numpy(inst.tids.view(np.int32)).pin_memory().numpy().view(np.uint32)
    h_pairs = torch.empty(3 * max(n_out, 1), dtype=torch.int32).pin_memory().numpy()
    e2e_steps = max(2, min(args.steps, 5))
    pkg.pair_support_host(inst.m, h_off, h_tids, None, inst.s, h_pairs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        k = pkg.pair_support_host(inst.m, h_off, h_tids, None, inst.s, h_pairs)
    e2e_t = (time.perf_counter() - t0) / e2e_steps
    assert k == n_out
    del h_tids

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    line = {
        "metric": METRIC, "value": world * rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": dict(rec["config"], parallelism="replicas" if world > 1 else "single GPU"),
        "roofline": rec["roofline"], "logical_hbm": rec["logical_hbm"],
        "set_elements_per_s": rec["set_elements_per_s"],
        "set_elements_definition": "sum over pairs of |S_i| + |S_j| = (n-1) * tids, per compare time (Sec. IV-B)",
        "phases_ms": rec["phases_ms"], "frequent_pairs": n_out, "failed_insertions": rec["failed_insertions"],
        "gpu_launches": rec["gpu_launches"],
        "e2e": {"value": npairs / e2e_t, "unit": UNIT,
                "h2d_bytes_per_step": int(h_off.nbytes + 4 * inst.tids.size),
                "d2h_bytes_per_step": int(12 * n_out + 8)},
        "clocks": rec["clocks"],
    }
    if "probe" in rec:
        line["probe"] = rec["probe"]
        line["compare_equiv"] = rec["compare_equiv"]
    if not args.no_dense and inst.m <= (1 << 24):
        line["dense"] = dense_leg(args, inst, off, tids, n_out, peaks, peak_kind, workload=label)
    del off, tids
    pkg.batmap_release_scratch()
    torch.cuda.empty_cache()
    if world == 1 and not args.no_cpu_baseline:
        rate, cores, k, dt = cpu_oracle_rate(inst, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{k} uniformly sampled pairs of the same workload, {dt:.1f} s "
                                          "(single-threaded sorted merge on disjoint blocks, one per core)",
                                "merge_micro": merge_micro()}
    if world == 1 and not args.no_sub and not args.scale_n:
        sub = {}
        if args.workload != "zipf_m1m_n2000":
            z = datagen.workload_instance("zipf_m1m_n2000")
            zr, zoff, ztids, zn = plain_leg(z, dev, 5, 3, peaks, peak_kind, "zipf_m1m_n2000")
            zr["dense"] = dense_leg(args, z, zoff, ztids, zn, peaks, peak_kind, steps=5, warmup=3,
                                    workload="zipf_m1m_n2000")
            del zoff, ztids
            sub["zipf_m1m_n2000"] = zr
        pkg.batmap_release_scratch()
        torch.cuda.empty_cache()
        sub["batched"] = batch_record(args, steps=3, warmup=2)
        line["sub"] = sub
        line["extra_keys"] = sorted(k for k in line if k not in (
            "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
            "gpu_launches", "clocks"))
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def batch_record(args, steps, warmup, small=False, instances=64, autotune=True):
    """Batched form: `instances` independent instances (m log-uniform in [1e4, 1e6],
    n uniform in [100, 4000], density uniform in [1%, 10%], Zipf items); one batched,
    graph-captured persistent pass vs the same instances as plain pair_support_all
    calls, each timed with events; outputs compared, a sample against the oracle."""
    import torch
    import paper_1102_1003_gb300 as pkg
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    if small:
        # many small instances, where per-call launches and synchronisations dominate
        specs = datagen.batch_specs(instances, 5000, m_range=(1e3, 1e5), n_range=(50, 400))
    else:
        specs = datagen.batch_specs(instances, 1000)
    t0 = time.perf_counter()
    insts = datagen.batch_instances(specs, workers=os.cpu_count() or 8)
    gen_s = time.perf_counter() - t0
    sets, npairs, wp = [], 0, 0.0
    t0 = time.perf_counter()
    for inst in insts:
        off = torch.from_numpy(inst.offsets.view(np.int64)).to(dev)
        tids = torch.from_numpy(inst.tids.view(np.int32)).to(dev)
        sets.append(pkg.batmap_build(inst.m, off, tids, None, params=_build_params()))
        npairs += inst.n * (inst.n - 1) // 2
        del off, tids
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    eff = pkg.batmap_autotune(sets) if autotune else None
    wp = sum(b.info["word_pairs"] for b in sets)
    # output sizes from one plain pass
    n_out = [pkg.pair_support_all(b, i.s)[0] for b, i in zip(sets, insts)]
    bufs = [torch.empty((max(k, 1), 3), dtype=torch.int32, device=dev) for k in n_out]
    s_list = [i.s for i in insts]
    cmp_plain, cmp_batch = [], []

    def plain(record):
        got = [pkg.pair_support_all(b, s, pairs=buf)[0] for b, s, buf in zip(sets, s_list, bufs)]
        if record:
            cmp_plain.append(sum(pkg.batmap_get_timing(b)["compare_ms"] for b in sets))
        return got

    def batched(record):
        got = pkg.pair_support_batch(sets, s_list, bufs)
        if record:
            cmp_batch.append(pkg.batmap_get_timing(sets[0])["compare_ms"])
        return got

    results = {}
    for name, fn in (("plain", plain), ("batched", batched)):
        for _ in range(warmup):
            fn(False)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            got = fn(True)
        ev1.record(stream)
        torch.cuda.synchronize()
        el = ev0.elapsed_time(ev1) / 1e3
        results[name] = {"value": npairs * steps / el, "ms_per_step": 1e3 * el / steps}
        assert list(got) == n_out, name
    peaks, peak_kind = _peaks()
    alu_peak, sms = _alu_peak(dev, peaks)
    for name, c in (("plain", cmp_plain), ("batched", cmp_batch)):
        t = statistics.mean(c) / 1e3
        results[name]["compare_ms"] = 1e3 * t
        results[name]["compare_equiv_lane_op_frac"] = OPS_PER_WORD_PAIR * wp / t / 1e12 / alu_peak
    results["compare_equiv_definition"] = (
        "4 x sum over all pairs of max(|B_i|,|B_j|)/4 word pairs (the scan's work for every pair, "
        "probe-routed pairs included) / compare time / lane-op peak")
    results["probe_routed_share"] = sum(b.info["probe_word_pairs"] for b in sets) / wp
    # batched and plain give identical outputs; a sampled oracle check per instance
    batch_pairs = [b[:k].cpu().numpy().copy() for b, k in zip(bufs, n_out)]
    plain(False)
    same = all(np.array_equal(b[:k].cpu().numpy(), bp) for b, k, bp in zip(bufs, n_out, batch_pairs))
    rng = np.random.default_rng(3)
    exact = True
    for q in rng.choice(len(insts), 6, replace=False):
        inst = insts[q]
        full = torch.empty(inst.n * (inst.n - 1) // 2, dtype=torch.int32, device=dev)
        pkg.pair_support_all(sets[q], inst.s, full=full)
        ii = rng.integers(0, inst.n - 1, 400)
        jj = np.minimum(inst.n - 1, ii + 1 + rng.integers(0, inst.n, 400) % np.maximum(inst.n - 1 - ii, 1))
        ref = oracle.pairs_list(inst.offsets, inst.tids, ii, jj, threads=os.cpu_count() or 4)
        idx = ii * inst.n - ii * (ii + 1) // 2 + (jj - ii - 1)
        exact &= bool(np.array_equal(full.cpu().numpy()[idx].astype(np.uint32), ref))
    for b in sets:
        b.free()
    pkg.batmap_release_scratch()
    torch.cuda.empty_cache()
    return {"workload": "batch", "unit": UNIT, "value": results["batched"]["value"],
            "ms_per_step": results["batched"]["ms_per_step"], "steps": steps, "warmup": warmup,
            "batched": results["batched"], "plain": results["plain"],
            "compare_equiv_definition": results["compare_equiv_definition"],
            "probe_routed_share": results["probe_routed_share"],
            "speedup_batched_over_plain": results["batched"]["value"] / results["plain"]["value"],
            "config": {"instances": len(insts), "small": bool(small), "pairs": npairs,
                       "tids": int(sum(i.tids.size for i in insts)), "word_pairs": wp,
                       "m_range": [min(i.m for i in insts), max(i.m for i in insts)],
                       "n_range": [min(i.n for i in insts), max(i.n for i in insts)],
                       "autotuned": eff is not None},
            "shape_eff": eff, "gen_s": gen_s, "build_s": build_s,
            "batched_equals_plain": same, "oracle_sample_exact": exact}


def run_batch(args):
    """Batched workload: one JSON line (see batch_record)."""
    import torch
    torch.cuda.set_device(0)
    rec = batch_record(args, args.steps, args.warmup, small=args.batch_small, instances=args.instances,
                       autotune=not args.no_autotune)
    print(json.dumps(dict({"metric": METRIC}, **rec)), flush=True)


def run_nsweep(args):
    """Sec. IV-A / Fig. 5 shape: all pair supports at a constant instance size of
    10^7 items and 5% density for a growing number of distinct items n."""
    import torch
    import paper_1102_1003_gb300 as pkg
    import oracle
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    rows = []
    for n in args.nsweep:
        inst = datagen.nsweep_instance(n)
        off = torch.from_numpy(inst.offsets.view(np.int64)).to(dev)
        tids = torch.from_numpy(inst.tids.view(np.int32)).to(dev)
        perm = torch.from_numpy(datagen.permutations(inst.m, 3).view(np.int32)).to(dev)
        npairs = n * (n - 1) // 2
        full = torch.empty(npairs, dtype=torch.int32, device=dev)
        nopairs = torch.empty((1, 3), dtype=torch.int32, device=dev)
        times = []
        for rep in range(1 + args.steps):
            t0 = time.perf_counter()
            b = pkg.batmap_build(inst.m, off, tids, perm)
            pkg.pair_support_all(b, 2**32 - 1, pairs=nopairs, full=full)  # every support, no list
            torch.cuda.synchronize()
            if rep:
                times.append((time.perf_counter() - t0, pkg.batmap_get_timing(b)))
            info = b.info
            b.free()
        rng = np.random.default_rng(n)
        ii = rng.integers(0, n - 1, 500)
        jj = ii + 1 + (rng.integers(0, n, 500) % (n - 1 - ii))
        ref = oracle.pairs_list(inst.offsets, inst.tids, ii, jj, threads=os.cpu_count() or 4)
        got = full.cpu().numpy()[oracle.packed_index(n, ii, jj)].astype(np.uint32)
        wall = statistics.mean(t for t, _ in times)
        rows.append({"n": n, "m": inst.m, "tids": int(inst.tids.size), "pairs": npairs,
                     "batmap_bytes": int(info["bytes"]), "step_ms": 1e3 * wall,
                     "build_ms": statistics.mean(t["build_ms"] for _, t in times),
                     "compare_ms": statistics.mean(t["compare_ms"] for _, t in times),
                     "pair_supports_per_s": npairs / wall,
                     "logical_GBps": 8.0 * info["word_pairs"] / (statistics.mean(t["compare_ms"] for _, t in times) / 1e3) / 1e9,
                     "sampled_exact": bool(np.array_equal(got, ref))})
        del full, off, tids, perm
        pkg.batmap_release_scratch()
        torch.cuda.empty_cache()
    print(json.dumps({"metric": METRIC, "workload": "nsweep", "unit": UNIT,
                      "config": "10^7 items, density 5%, m = 10^7 / (0.05 n) (Sec. IV-A, Fig. 5 shape)",
                      "rows": rows}), flush=True)


def run_cross(args):
    """Sparse boolean matrix multiplication / join-project (Sec. I): the supports
    |A_i cap B_j| of every pair across two families and the pairs with a
    nonempty intersection (s = 1).  One step = cross build + compare + list."""
    import torch
    import paper_1102_1003_gb300 as pkg
    import oracle
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    L = pkg.load_library()
    union, na = datagen.cross_instance()
    nb = union.n - na
    npairs = na * nb
    off = torch.from_numpy(union.offsets.view(np.int64)).to(dev)
    tids = torch.from_numpy(union.tids.view(np.int32)).to(dev)
    perm = torch.from_numpy(datagen.permutations(union.m, 5).view(np.int32)).to(dev)
    full = torch.empty(npairs, dtype=torch.int32, device=dev)
    b = pkg.batmap_build_cross(union.m, na, off, tids, perm, params=_build_params())
    n_out, _ = pkg.pair_support_all(b, 1)
    info = b.info
    b.free()
    pairs = torch.empty((max(n_out, 1), 3), dtype=torch.int32, device=dev)

    def step():
        bs = pkg.batmap_build_cross(union.m, na, off, tids, perm, params=_build_params())
        k, _ = pkg.pair_support_all(bs, 1, pairs=pairs, full=full)
        t = pkg.batmap_get_timing(bs)
        bs.free()
        return k, t

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    launches0 = L.batmap_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    phases = []
    for _ in range(args.steps):
        k, t = step()
        phases.append(t)
    ev1.record(stream)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = L.batmap_kernel_launches() - launches0
    clocks = sampler.stop()
    assert k == n_out
    # sampled parity against the oracle on the union (B's items follow A's)
    rng = np.random.default_rng(5)
    ia = rng.integers(0, na, 4000)
    jb = rng.integers(0, nb, 4000)
    ref = oracle.pairs_list(union.offsets, union.tids, ia, na + jb, threads=os.cpu_count() or 4)
    got = full.cpu().numpy().astype(np.uint32)[ia * nb + jb]
    peaks, peak_kind = _peaks()
    scan_s = statistics.mean(t["scan_ms"] for t in phases) / 1e3
    wp_scan = info["word_pairs"] - info["probe_word_pairs"]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = OPS_PER_WORD_PAIR * wp_scan / scan_s / 1e12
    line = {"metric": "A x B pair supports/sec (sparse boolean matrix multiplication), bit-exact",
            "workload": "cross", "unit": UNIT, "value": npairs * args.steps / elapsed, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "cross", "m": union.m, "n_a": na, "n_b": nb, "s": 1, "pairs": npairs,
                       "desc": "A: Zipf(1) sizes at mean density 1%; B: Bernoulli p=0.002",
                       "tids": int(union.tids.size), "batmap_bytes": int(info["bytes"]),
                       "l2": "inputs larger than L2 (no flush)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                         "frac": achieved / alu_peak, "kernel": "k_compare", "traffic": None,
                         "peak_kind": f"{sms} SMs x 128 INT32 lanes x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz "
                                      f"({peak_kind} max clock)",
                         "algorithmic_ops": f"{OPS_PER_WORD_PAIR} x {wp_scan:.4g} word pairs (the scan-routed pairs' "
                                        f"max(|B_i|,|B_j|)/4) per scan time {1e3 * scan_s:.3f} ms"},
            "phases_ms": {p: statistics.mean(t[p] for t in phases)
                          for p in ("build_ms", "compare_ms", "scan_ms", "probe_ms", "compact_ms")},
            "probe_routed_share": info["probe_word_pairs"] / max(info["word_pairs"], 1.0),
            "nonempty_pairs": n_out, "failed_insertions": info["n_failed"], "gpu_launches": int(launches),
            "parity_sample": {"pairs": int(ia.size), "exact": bool(np.array_equal(got, ref))},
            "clocks": clocks}
    if not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        kk = 20000
        t0 = time.perf_counter()
        oracle.pairs_list(union.offsets, union.tids, rng.integers(0, na, kk), na + rng.integers(0, nb, kk),
                          threads=cores)
        dt = time.perf_counter() - t0
        kk = int(min(max(kk * args.cpu_seconds / max(dt, 1e-6), kk), npairs))
        ia, jb = rng.integers(0, na, kk), rng.integers(0, nb, kk)
        t0 = time.perf_counter()
        oracle.pairs_list(union.offsets, union.tids, ia, na + jb, threads=cores)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": kk / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{kk} uniformly sampled A x B pairs, {dt:.1f} s"}
    print(json.dumps(line), flush=True)


def run_triples(args):
    """Frequent itemsets of size 3 (Apriori level 3) over 3-of-4 BatMaps: one step =
    2-of-3 build + frequent pairs + 3-of-4 build + candidates + witness supports +
    compaction, tidlists resident in HBM."""
    import torch
    import paper_1102_1003_gb300 as pkg
    import oracle
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    L = pkg.load_library()
    inst = datagen.triples_instance()
    s = inst.s
    off = torch.from_numpy(inst.offsets.view(np.int64)).to(dev)
    tids = torch.from_numpy(inst.tids.view(np.int32)).to(dev)
    perm4 = torch.from_numpy(datagen.permutations(inst.m, 9, count=4).view(np.int32)).to(dev)
    perm3 = perm4[:3].contiguous()
    b2 = pkg.batmap_build(inst.m, off, tids, perm3)
    n_pairs, pairs = pkg.pair_support_all(b2, s)
    pairs_buf = torch.empty((max(n_pairs, 1), 3), dtype=torch.int32, device=dev)
    b2.free()
    b3 = pkg.batmap_build_d(3, inst.m, off, tids, perm4)
    n_trip, trip, n_cand = pkg.frequent_triples(b3, s, pairs)
    info3 = b3.info
    b3.free()
    out = torch.empty((max(n_trip, 1), 4), dtype=torch.int32, device=dev)

    def step():
        a = pkg.batmap_build(inst.m, off, tids, perm3)
        k2, p = pkg.pair_support_all(a, s, pairs=pairs_buf)
        t2 = pkg.batmap_get_timing(a)
        a.free()
        b = pkg.batmap_build_d(3, inst.m, off, tids, perm4)
        k3, t, nc = pkg.frequent_triples(b, s, p, out=out)
        t3 = pkg.batmap_get_timing(b)
        b.free()
        return k2, k3, nc, t2, t3

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    launches0 = L.batmap_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rec = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = L.batmap_kernel_launches() - launches0
    clocks = sampler.stop()
    assert all(r[0] == n_pairs and r[1] == n_trip and r[2] == n_cand for r in rec)
    # sampled parity of the frequent triples and candidate supports against the oracle
    cand_ref = None
    from oracle import dof_rules as R
    pairs_ref = oracle.pairs_threshold(inst.offsets, inst.tids, s)
    exact_pairs = bool(np.array_equal(pairs_buf[:n_pairs].cpu().numpy().astype(np.uint32), pairs_ref))
    cand_ref = R.triple_candidates(pairs_ref[:, :2])
    got = out[:n_trip].cpu().numpy().astype(np.uint32)
    rng = np.random.default_rng(3)
    pick = rng.choice(cand_ref.shape[0], min(2000, cand_ref.shape[0]), replace=False)
    sup = oracle.kway_counts(inst.offsets, inst.tids, cand_ref[pick].tolist())
    keep = {tuple(x) for x in got[:, :3].tolist()}
    got_sup = {tuple(x[:3]): x[3] for x in got.tolist()}
    ok_sample = all(((tuple(c) in keep) == (v >= s)) and (v < s or got_sup[tuple(c)] == v)
                    for c, v in zip(cand_ref[pick].tolist(), sup.tolist()))
    peaks, peak_kind = _peaks()
    wit_s = statistics.mean(r[4]["compare_ms"] for r in rec) / 1e3
    scan_s = statistics.mean(r[4]["scan_ms"] for r in rec) / 1e3
    probe_s = statistics.mean(r[4]["probe_ms"] for r in rec) / 1e3
    sz = inst.sizes
    r0 = info3["r0"]
    rr = np.array([max(r0, 1 << int(np.ceil(np.log2(max(2 * int(x), 1))))) for x in sz], dtype=np.int64)
    rc = rr[cand_ref]
    wt = int(rc.max(axis=1).sum())
    # the library's route: the probe kernel takes the candidates whose widest
    # BatMap is at least 8x the narrowest, the scan kernel the rest
    probe = rc.max(axis=1) >= 8 * rc.min(axis=1)
    wt_scan = int(rc[~probe].max(axis=1).sum())
    narrow = np.argmin(rc, axis=1)
    probe_words = int(rc[probe].min(axis=1).sum())
    probe_slots = int(3 * sz[cand_ref[np.arange(cand_ref.shape[0]), narrow]][probe].sum())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = WITNESS_OPS * wt_scan / scan_s / 1e12
    line = {"metric": "candidate itemset supports/sec (Apriori level 3 over 3-of-4 BatMaps), bit-exact",
            "workload": "triples", "unit": "candidate-supports/s", "value": n_cand * args.steps / elapsed,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "triples", "m": inst.m, "n": inst.n, "s": s, "tids": int(inst.tids.size),
                       "desc": "Zipf(1) items at mean density 2%", "frequent_pairs": n_pairs,
                       "candidates": n_cand, "frequent_triples": n_trip, "batmap3_bytes": int(info3["bytes"]),
                       "word_triples": wt},
            "phases_ms": {"build_2of3": statistics.mean(r[3]["build_ms"] for r in rec),
                          "pairs": statistics.mean(r[3]["pairs_ms"] for r in rec),
                          "build_3of4": statistics.mean(r[4]["build_ms"] for r in rec),
                          "witness": 1e3 * wit_s, "witness_scan": 1e3 * scan_s, "witness_probe": 1e3 * probe_s,
                          "candidates_compact": statistics.mean(r[4]["compact_ms"] for r in rec)},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                         "frac": achieved / alu_peak, "kernel": "k_witness_group",
                         "traffic": _traffic("triples", "k_witness_group", "witness.cu"),
                         "peak_kind": f"{sms} SMs x 128 INT32 lanes x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz "
                                      f"({peak_kind} max clock)",
                         "algorithmic_ops": f"{WITNESS_OPS} x {wt_scan:.4g} word-triples (max_j r_j words per "
                                            f"scan-routed candidate, {int((~probe).sum())} of {probe.size})",
                         "note": "the 3-of-4 BatMaps (24.6 MB) are L2-resident"},
            "probe": {"kernel": "k_witness_probe", "candidates": int(probe.sum()), "ms": 1e3 * probe_s,
                      "traffic": _traffic("triples", "k_witness_probe", "witness.cu"),
                      "narrow_words": probe_words, "slots": probe_slots,
                      "slots_per_s": probe_slots / probe_s if probe_s > 0 else None,
                      "bound": "L2 latency: two random byte probes per nonempty slot of the narrowest BatMap",
                      "slots_definition": "3 |S| of each probed candidate's narrowest set (copies stored)",
                      "scan_equivalent_word_triples": int(rc[probe].max(axis=1).sum())},
            "gpu_launches": int(launches), "failed_insertions_3of4": info3["n_failed"],
            "parity": {"pairs_exact": exact_pairs, "sampled_candidates": int(pick.size), "exact": bool(ok_sample)},
            "clocks": clocks}
    if not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        k = 2000
        t0 = time.perf_counter()
        oracle.kway_counts(inst.offsets, inst.tids, cand_ref[rng.choice(cand_ref.shape[0], k)].tolist())
        dt = max(time.perf_counter() - t0, 1e-6)
        line["cpu_baseline"] = {"value": k / dt, "unit": "candidate-supports/s", "cores": 1, "kind": "oracle",
                                "sample": f"{k} uniformly sampled candidates, single-threaded k-way merge, {dt:.1f} s"}
    print(json.dumps(line), flush=True)


def run_quads(args):
    """Frequent itemsets of size 4 (Apriori level 4) over 4-of-5 BatMaps: one step =
    2-of-3 build + frequent pairs + 4-of-5 build + frequent triples + frequent
    quadruples (candidates, witness supports, compaction), tidlists resident in HBM."""
    import torch
    import paper_1102_1003_gb300 as pkg
    import oracle
    from oracle import dof_rules as R
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    L = pkg.load_library()
    inst = datagen.triples_instance()
    s = inst.s
    off = torch.from_numpy(inst.offsets.view(np.int64)).to(dev)
    tids = torch.from_numpy(inst.tids.view(np.int32)).to(dev)
    b2 = pkg.batmap_build(inst.m, off, tids, None)
    n_pairs, pairs = pkg.pair_support_all(b2, s)
    pairs_buf = torch.empty((max(n_pairs, 1), 3), dtype=torch.int32, device=dev)
    b2.free()
    b4 = pkg.batmap_build_d(4, inst.m, off, tids, None)
    n_trip, trip, n_c3 = pkg.frequent_triples(b4, s, pairs)
    trip_buf = torch.empty((max(n_trip, 1), 4), dtype=torch.int32, device=dev)
    n_quad, quad, n_c4 = pkg.frequent_quadruples(b4, s, trip)
    quad_buf = torch.empty((max(n_quad, 1), 5), dtype=torch.int32, device=dev)
    info4 = b4.info
    b4.free()

    def step():
        a = pkg.batmap_build(inst.m, off, tids, None)
        k2, p = pkg.pair_support_all(a, s, pairs=pairs_buf)
        t2 = pkg.batmap_get_timing(a)
        a.free()
        b = pkg.batmap_build_d(4, inst.m, off, tids, None)
        tb = pkg.batmap_get_timing(b)
        k3, t, c3 = pkg.frequent_triples(b, s, p, out=trip_buf)
        t3 = pkg.batmap_get_timing(b)
        k4, q, c4 = pkg.frequent_quadruples(b, s, t, out=quad_buf)
        t4 = pkg.batmap_get_timing(b)
        b.free()
        return k2, k3, k4, c4, t2, tb, t3, t4

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()
    torch.cuda.synchronize()
    launches0 = L.batmap_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rec = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = L.batmap_kernel_launches() - launches0
    clocks = sampler.stop()
    assert all(r[0] == n_pairs and r[1] == n_trip and r[2] == n_quad and r[3] == n_c4 for r in rec)
    # parity: the frequent pairs in full; sampled triple and quadruple candidates against the oracle
    pairs_ref = oracle.pairs_threshold(inst.offsets, inst.tids, s)
    exact_pairs = bool(np.array_equal(pairs_buf[:n_pairs].cpu().numpy().astype(np.uint32), pairs_ref))
    rng = np.random.default_rng(4)
    got3 = trip_buf[:n_trip].cpu().numpy().astype(np.uint32)
    got4 = quad_buf[:n_quad].cpu().numpy().astype(np.uint32)

    def sampled_ok(cands, got, width):
        pick = rng.choice(cands.shape[0], min(2000, cands.shape[0]), replace=False)
        sup = oracle.kway_counts(inst.offsets, inst.tids, cands[pick].tolist())
        keep = {tuple(x[:width]): x[width] for x in got.tolist()}
        return all(((tuple(c) in keep) == (v >= s)) and (v < s or keep[tuple(c)] == v)
                   for c, v in zip(cands[pick].tolist(), sup.tolist())), int(pick.size)

    c3 = R.triple_candidates(pairs_ref[:, :2])
    ok3, k3 = sampled_ok(c3, got3, 3)
    c4 = R.quadruple_candidates(got3[:, :3]) if n_trip else np.zeros((0, 4), np.int64)
    ok4, k4 = sampled_ok(c4, got4, 4) if c4.shape[0] else (True, 0)
    line = {"metric": "candidate itemset supports/sec (Apriori levels 3 and 4 over 4-of-5 BatMaps), bit-exact",
            "workload": "quads", "unit": "candidate-supports/s", "value": (n_c3 + n_c4) * args.steps / elapsed,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "quads", "m": inst.m, "n": inst.n, "s": s, "tids": int(inst.tids.size),
                       "desc": "Zipf(1) items at mean density 2%", "frequent_pairs": n_pairs,
                       "triple_candidates": n_c3, "frequent_triples": n_trip,
                       "quadruple_candidates": n_c4, "frequent_quadruples": n_quad,
                       "batmap4_bytes": int(info4["bytes"])},
            "phases_ms": {"build_2of3": statistics.mean(r[4]["build_ms"] for r in rec),
                          "pairs": statistics.mean(r[4]["pairs_ms"] for r in rec),
                          "build_4of5": statistics.mean(r[5]["build_ms"] for r in rec),
                          "triples": statistics.mean(r[6]["pairs_ms"] for r in rec),
                          "triple_witness_scan": statistics.mean(r[6]["scan_ms"] for r in rec),
                          "triple_witness_probe": statistics.mean(r[6]["probe_ms"] for r in rec),
                          "quadruples": statistics.mean(r[7]["pairs_ms"] for r in rec),
                          "quadruple_witness": statistics.mean(r[7]["compare_ms"] for r in rec),
                          "quadruple_witness_scan": statistics.mean(r[7]["scan_ms"] for r in rec),
                          "quadruple_witness_probe": statistics.mean(r[7]["probe_ms"] for r in rec)},
            "gpu_launches": int(launches), "failed_insertions_4of5": info4["n_failed"],
            "parity": {"pairs_exact": exact_pairs, "sampled_triple_candidates": k3, "triples_exact": bool(ok3),
                       "sampled_quadruple_candidates": k4, "quadruples_exact": bool(ok4)},
            "clocks": clocks}
    if not args.no_cpu_baseline and c4.shape[0]:
        k = 2000
        t0 = time.perf_counter()
        oracle.kway_counts(inst.offsets, inst.tids, c4[rng.choice(c4.shape[0], k)].tolist())
        dt = max(time.perf_counter() - t0, 1e-6)
        line["cpu_baseline"] = {"value": k / dt, "unit": "candidate-supports/s", "cores": 1, "kind": "oracle",
                                "sample": f"{k} uniformly sampled quadruple candidates, single-threaded k-way "
                                          f"merge, {dt:.1f} s"}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving workload: pool of sets over 2^26 with Zipf sizes on [10, 1e6],
    Poisson-arriving queries (80% pairs, 20% 3..8-way), continuous batching."""
    import math
    import torch
    import paper_1102_1003_gb300 as pkg
    import oracle
    U, lo, hi, seed = 1 << 26, 10, 10**6, 5
    count = args.pool_sets
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    sizes = datagen.pool_sizes(count, lo, hi, seed)
    ub = int(sum(int(k + 6 * math.sqrt(k) + 16) for k in sizes))
    t0 = time.perf_counter()
    d_tids = torch.empty(ub, dtype=torch.int32, device=dev)
    real = np.zeros(count, dtype=np.int64)
    pos = 0
    for a, got, arr in datagen.pool_blocks(count, U, lo, hi, seed, workers=os.cpu_count() or 8):
        d_tids[pos:pos + arr.size].copy_(torch.from_numpy(arr.view(np.int32)))
        real[a:a + got.size] = got
        pos += arr.size
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    offsets = np.zeros(count + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(real)
    d_off = torch.from_numpy(offsets.view(np.int64)).to(dev)
    perm = torch.from_numpy(datagen.permutations(U, seed).view(np.int32)).to(dev)
    t0 = time.perf_counter()
    pool = pkg.batmap_pool_create(U, d_off, d_tids[:pos], perm)
    build_s = time.perf_counter() - t0
    info = pool.info
    del d_tids
    torch.cuda.empty_cache()
    rng = np.random.default_rng(77)
    nq = args.queries
    queries = []
    for _ in range(nq):
        k = 2 if rng.random() < 0.8 else int(rng.integers(3, 9))
        queries.append(rng.integers(0, count, k).tolist())
    opts = pkg.batmap_serve_opts(max_batch=args.max_batch, slots=args.slots, work_budget=1 << 26, reserved=0)
    pkg.batmap_serve(pool, queries[:2000], np.zeros(2000), opts)  # warm-up
    counts, lat, st_max = pkg.batmap_serve(pool, queries, np.zeros(nq), opts)
    qps_max = st_max["queries_per_s"]
    # one query per launch, no batching, for comparison
    n_plain = min(nq, 3000)
    t0 = time.perf_counter()
    for q in range(n_plain):
        pkg.intersect_query(pool, [queries[q]])
    torch.cuda.synchronize()
    qps_plain = n_plain / (time.perf_counter() - t0)
    loads = []
    for f in (0.25, 0.5, 0.75, 0.9):
        arrival = np.cumsum(np.random.default_rng(int(f * 100)).exponential(1.0 / (f * qps_max), nq))
        c2, lat2, st2 = pkg.batmap_serve(pool, queries, arrival, opts)
        assert np.array_equal(c2, counts)
        loads.append({"offered_fraction": f, "offered_qps": f * qps_max, "achieved_qps": st2["queries_per_s"],
                      "p50_ms": 1e3 * st2["p50_s"], "p99_ms": 1e3 * st2["p99_s"], "batches": st2["batches"],
                      "max_inflight": st2["max_inflight"]})
    # parity on a sample: regenerate the named sets on the CPU and run the oracle
    sample = np.random.default_rng(5).choice(nq, min(nq, 300), replace=False)
    ids = sorted({c for q in sample for c in queries[q]})
    remap = {c: j for j, c in enumerate(ids)}
    sub = datagen.from_lists([datagen.pool_set(U, int(sizes[c]), seed, c) for c in ids], U)
    ref = oracle.kway_counts(sub.offsets, sub.tids, [[remap[c] for c in queries[q]] for q in sample])
    exact = bool(np.array_equal(counts[sample], ref))
    line = {"metric": "serving queries/sec and p50/p99 latency", "workload": "serve", "unit": "queries/s",
            "value": qps_max, "plain_one_query_per_launch_qps": qps_plain, "loads": loads,
            "closed_loop": {"p50_ms": 1e3 * st_max["p50_s"], "p99_ms": 1e3 * st_max["p99_s"],
                            "batches": st_max["batches"], "max_inflight": st_max["max_inflight"]},
            "config": {"pool_sets": count, "universe": U, "sizes": "Zipf(1) on [10, 1e6]",
                       "elements": int(info["n_elements"]), "batmap_sets": info["n_batmaps"],
                       "batmap_bytes": int(info["batmap_bytes"]), "queries": nq,
                       "mix": "80% pairwise, 20% k in 3..8, uniform set ids", "max_batch": args.max_batch,
                       "slots": args.slots},
            "gen_s": gen_s, "pool_build_s": build_s, "parity_sample": {"queries": int(sample.size), "exact": exact}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--workload", choices=sorted(WORKLOAD_DESC) + ["serve", "batch", "nsweep", "cross", "triples", "quads"], default="bern_m4m_n8192_p5")
    ap.add_argument("--nsweep", type=int, nargs="+", default=[1000, 2000, 4000, 8000, 16000, 32000, 64000])
    ap.add_argument("--instances", type=int, default=64, help="instances (batch workload)")
    ap.add_argument("--batch-small", action="store_true",
                    help="batch workload of small instances (m in [1e3, 1e5], n in [50, 400])")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--probe-log", type=int, default=0,
                    help="batmap_params.probe_log: pairs whose widths differ by 2^k or more are probed "
                         "(0 = library default, 32 = scan every pair)")
    ap.add_argument("--pool-sets", type=int, default=100_000, help="serving pool size (serve workload)")
    ap.add_argument("--queries", type=int, default=200_000, help="queries per serving run (serve workload)")
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense tensor-core comparison leg")
    ap.add_argument("--scale-n", type=int, default=None,
                    help="keep only the first N items of the workload (small profiling cases)")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the sub-records (Zipf workload, batched vs plain) of the default line")
    args = ap.parse_args()
    global PROBE_LOG
    PROBE_LOG = args.probe_log
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload in ("serve", "batch", "nsweep", "cross", "triples", "quads"):
        if rank == 0:
            {"serve": run_serve, "batch": run_batch, "nsweep": run_nsweep, "cross": run_cross,
             "triples": run_triples, "quads": run_quads}[args.workload](args)
        return
    inst = datagen.workload_instance(args.workload, scale_n=args.scale_n, workers=os.cpu_count() or 8)
    if args.impl == "reference":
        run_reference(args, inst, rank, world)
    else:
        run_mine(args, inst, rank, world)


if __name__ == "__main__":
    main()
