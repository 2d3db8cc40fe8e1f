#!/usr/bin/env python3
"""Benchmark of the GB300 Aho-Corasick scan.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload genome|chromosome|small|batch|serve] [--n-bases B] [--minimal]

One step = one pass of the whole scan path (encode is outside: the workload
text is already 2-bit packed in HBM; the scan kernel with fused emission, then
the count kernel, then the 8-byte read of the occurrence count) over one text.
Rank 0 prints ONE JSON line. ``value`` = bases scanned by all ranks / the
slowest rank's device time (CUDA events on the launching stream), in Gbases/s.

Default workload: the 3 Gbase synthetic genome (order-2 Markov chain, 41% GC,
5% short tandem repeats) against 100,000 keywords of length 20-25. With the
full run the line also carries the batched workload (4,096 lognormal texts,
batched graph replay vs a per-text loop) and a short serving run (Poisson
arrivals over 8 resident machines, p50/p99 latency).

N > 1 ranks (torchrun): each rank scans its own copy of the workload (weak
scaling, no data-path collective); the only collective is the max-reduce of
the timings. ``--impl reference`` times the CPU oracle (the textbook
goto/failure/output scan) on a bounded sample of the same workload on the
host cores, rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import queue
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gbases/s scanned (bit-exact), batched vs plain on 1 GB300; serving p50/p99 ms"
UNIT = "Gbases/s"


# ------------------------------------------------------------------ helpers


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# DRAM traffic of the scan kernel per base of the genome workload, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum of one launch over a
# 1 Gbase slice of the same generator); a 3 Gbase launch is scaled by its bases
# (traffic grows with the text). It holds only for the same kernel and table
# builder code (hash of the sources without comments), the same table sizes
# and the same launch shape; otherwise traffic is null.
TRAFFIC_CAPTURE = {"workload": "genome", "sources_sha256": "4310ab2dae039c21a27db16010619cf9f071b57f905882ea5ebb9afd989ab880",
                   "bytes_per_base": (6.128241e9 + 2.629430e9) / 1e9,
                   "shape": {"stride": 3, "threads": 640, "interleave": 1, "hot_states": 0},
                   "table2_bytes": 1462719 * 64, "table3_bytes": 1462719 * 256,
                   "capture": "profiles/scan_kernel_genome_1gbase_full.md"}
TRAFFIC_SOURCES = ("ac_kernels.cu", "ac_builder.cpp")


def code_without_comments(src: str) -> str:
    """C/C++ source with comments and whitespace removed (string literals kept)."""
    import re

    src = re.sub(r'//[^\n]*|/\*.*?\*/|("(?:\\.|[^"\\])*")', lambda m: m.group(1) or " ", src, flags=re.S)
    return re.sub(r"\s+", "", src)


def library_sources_sha() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1403_7294_gb300", "csrc", f)) as fh:
            h.update(code_without_comments(fh.read()).encode())
    return h.hexdigest()


def measured_traffic(workload: str, n_bases: int, shape: dict, info: dict):
    c = TRAFFIC_CAPTURE
    same = (workload == c["workload"] and library_sources_sha() == c["sources_sha256"]
            and all(shape.get(k) == v for k, v in c["shape"].items())
            and info.get("table2_bytes") == c["table2_bytes"] and info.get("table3_bytes") == c["table3_bytes"])
    return int(round(c["bytes_per_base"] * n_bases)) if same else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx.append(float(c[2]))
                    power.append(float(c[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "power_w_max": max(power),
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- workloads


def make_workload(name: str, n_bases: int | None, device: str, rank: int):
    from paper_1403_7294_gb300 import synth

    seed_off = 1000 * rank  # weak scaling: every rank its own text
    if name == "genome":
        return synth.plain_genome(device=device, seed=synth.BASE_SEED + 2 + seed_off, n=n_bases or 3_000_000_000)
    if name == "chromosome":
        return synth.plain_chromosome(device=device, seed=synth.BASE_SEED + 1 + seed_off, n=n_bases or 268_435_456)
    if name == "small":
        return synth.plain_small(device=device, seed=synth.BASE_SEED + seed_off, n=n_bases or 1_000_000)
    raise ValueError(name)


def run_plain_configs(args, world, rank, local) -> dict:
    """The other two plain-scan configurations (1 Mbase uniform text with 100
    keywords; 256 Mbase chromosome with 10,000 keywords), timed like the main
    line (autotuned, device-resident text, CUDA events), for the per-config table."""
    import copy

    res = {}
    for name in ("small", "chromosome"):
        sub = copy.copy(args)
        sub.workload, sub.n_bases, sub.minimal, sub.shape = name, None, True, None
        o, _ = run_plain(sub, world, rank, local)
        res[name] = {"workload": o["config"]["workload"], "gbases_s": o["value"], "ms_per_step": o["ms_per_step"],
                     "occurrences_per_step": o["config"]["occurrences_per_step"], "states": o["config"]["states"],
                     "shape": o["config"]["shape"], "hbm_frac": o["roofline"]["frac"],
                     "kernel_ms": o["roofline"]["kernel_ms"]}
        torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------- plain scan


def run_plain(args, world, rank, local):
    import ctypes

    import paper_1403_7294_gb300 as acg
    from paper_1403_7294_gb300 import _native as N

    lib = acg.lib()
    t0 = time.time()
    w = make_workload(args.workload, args.n_bases, "cuda", rank)
    n = int(w.text.ascii.numel())
    if args.uniform_patterns:  # the walk-only case: keywords of the same shape that never occur
        from paper_1403_7294_gb300 import synth

        lo, hi = {"genome": (20, 25), "chromosome": (18, 30), "small": (8, 20)}[args.workload]
        w.patterns = synth.uniform_patterns(len(w.patterns), lo, hi, synth.BASE_SEED + 77)
        w.name += "-uniform-keywords"
    log(f"[bench] workload {w.name}: generated in {time.time() - t0:.1f}s")
    t0 = time.time()
    dfa = acg.build(w.patterns)
    log(f"[bench] machine: {dfa.info['n_states']} states, build {dfa.info['build_ms']:.0f} ms")
    packed = acg.pack(w.text.ascii)
    torch.cuda.synchronize()
    ascii_prefix = None
    if not args.minimal and rank == 0:
        ascii_prefix = w.text.ascii[: min(n, 400_000_000)].cpu().numpy()
    ascii_input = args.workload == "small"  # that configuration's input is uint8 ASCII: packing is in the step
    ascii_dev = w.text.ascii if ascii_input else None
    del w.text.ascii
    torch.cuda.empty_cache()
    # inputs smaller than L2 (129 MB) are flushed from it between timed steps
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda") if n // 4 < (256 << 20) else None
    P = len(w.patterns)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    opts = N.ScanOpts()
    opts.hot_states = -1
    if args.shape:  # a fixed launch shape instead of the tuned one
        opts.stride, opts.threads, opts.interleave, opts.hot_states = (int(x) for x in args.shape.split(","))
    else:
        t0 = time.time()
        tuned = acg.autotune(dfa, packed, n)  # cached per (device, machine size, text size); untimed
        log(f"[bench] autotune {tuned} in {time.time() - t0:.1f}s")
    desc = (N.Text(ascii_dev.data_ptr(), n, N.AC_TEXT_ASCII, 1) if ascii_input
            else N.Text(packed.data_ptr(), n, N.AC_TEXT_PACKED2, 1))
    counts = torch.empty(P, dtype=torch.int64, device="cuda")
    # size the occurrence buffer with one counting pass
    r = N.Result(None, 0, 0, counts.data_ptr(), 1, 0, 0)
    st = lib.ac_scan(dfa.h, ctypes.byref(desc), ctypes.byref(r), ctypes.byref(opts), sp, None)
    assert st in (N.AC_OK, N.AC_ERR_OVERFLOW), st
    n_matches = int(r.n_matches)
    cap = n_matches + 1024
    raw = torch.empty((cap, 2), dtype=torch.int64, device="cuda")
    res = N.Result(raw.data_ptr(), cap, 0, counts.data_ptr(), 1, 0, 0)
    stats = N.ScanStats()

    call_ms = []  # device time of each whole ac_scan call (events inside it, on its stream)

    def step():
        if flush is not None:
            flush.fill_(1)  # evicts the text and tables from L2 (not inside the call's events)
        s = lib.ac_scan(dfa.h, ctypes.byref(desc), ctypes.byref(res), ctypes.byref(opts), sp, ctypes.byref(stats))
        if s != N.AC_OK:
            raise acg.AcError(s, "ac_scan")
        call_ms.append(stats.total_ms)
        return stats.scan_ms

    for _ in range(args.warmup):
        step()
    assert int(res.n_matches) == n_matches
    assert int(counts.sum().item()) == n_matches
    clocks = Clocks(torch.cuda.current_device())
    torch.cuda.synchronize()
    barrier(world)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    scan_ms = []
    for _ in range(args.steps):
        scan_ms.append(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if flush is not None:  # the region between ev0 and ev1 holds the flushes too: count only the calls
        ms = float(np.sum(call_ms[-args.steps:]))
    barrier(world)
    ms_max = max_over_ranks(ms, world)
    value = args.steps * n * world / (ms_max / 1e3) / 1e9

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {
            "workload": w.name, "n_bases": n, "patterns": P, "pattern_len": "20-25" if args.workload == "genome" else None,
            "states": dfa.info["n_states"],
            "encoding": "uint8 ASCII resident in HBM, packed inside each step" if ascii_input else "2-bit packed, resident in HBM",
            "occurrences_per_step": n_matches,
            "l2": (f"L2 flushed between steps (512 MB write; {n // 4 / 1e6:.1f} MB packed text vs 129 MB L2), "
                   "step time = device time of each ac_scan call") if flush is not None
                  else f"inputs larger than L2 ({n // 4 / 1e6:.0f} MB packed text vs 129 MB L2)",
            "parallelism": f"replicas x{world}", "build_ms": round(dfa.info["build_ms"], 1),
            "shape": {k: getattr(stats, k) for k in ("stride", "chunk", "chunks_per_lane", "threads", "interleave",
                                                     "hot_states", "grid", "blocks_per_sm")},
            "autotuned": not args.shape,
        },
        "gpu_launches": (3 if ascii_input else 2) * args.steps,  # (pack kernel +) scan kernel + count kernel per step
        "clocks": clk,
    }
    # roofline of the dominant kernel (the scan): algorithmic bytes per launch
    peak, peak_kind = load_peaks()
    scan_avg = float(np.mean(scan_ms))
    # algorithmic bytes: the packed text, the occurrences, the per-keyword counts and the base
    # transition table once (16 B a state)
    alg_bytes = n / 4 + 16 * n_matches + 8 * P + 16 * dfa.info["n_states"]
    achieved = alg_bytes / (scan_avg / 1e3) / 1e9
    out["roofline"] = {
        "bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
        "frac": round(achieved / peak, 5), "peak_source": peak_kind,
        "traffic": measured_traffic(args.workload, n, {k: getattr(stats, k) for k in ("stride", "threads", "interleave",
                                                                                     "hot_states")}, dfa.info),
        "kernel": "scan_kernel", "kernel_ms": round(scan_avg, 4),
        "algorithmic_bytes": int(alg_bytes),
        "walked_bases_per_s": round(stats.bases_walked / (scan_avg / 1e3), 1),  # owned bases plus halo re-reads
        # one table lookup per step of `stride` bases (exact when every state has a row at that stride)
        "table_lookups_per_s": round(stats.bases_walked / max(stats.stride, 1) / (scan_avg / 1e3), 1),
        "kernel_ms_median": round(float(np.median(scan_ms)), 4), "kernel_ms_min": round(float(np.min(scan_ms)), 4),
    }
    if args.minimal:
        return out, None

    # ---- walk-only ceilings on the same text (no occurrences): the lookup roofline
    probe = lookup_probe(packed, n)
    ceiling = probe["uniform100k_default"]["walked_bases_per_s"]
    out["roofline"]["lookup"] = {
        "achieved_walked_bases_per_s": out["roofline"]["walked_bases_per_s"], "ceiling_walked_bases_per_s": ceiling,
        "frac": round(out["roofline"]["walked_bases_per_s"] / ceiling, 4),
        "ceiling_source": "same kernel, same text, 100,000 uniform keywords (no occurrences)", "probe": probe}

    # ---- end to end through the public API: host text in, host results out
    host_packed = packed.cpu().pin_memory()
    raw_h = torch.empty((cap, 2), dtype=torch.int64).pin_memory()
    cnt_h = torch.empty(P, dtype=torch.int64).pin_memory()
    desc_h = N.Text(host_packed.data_ptr(), n, N.AC_TEXT_PACKED2, 0)
    res_h = N.Result(raw_h.data_ptr(), cap, 0, cnt_h.data_ptr(), 0, 0, 0)
    k_e2e = max(1, min(args.steps, 10))
    import gc

    gc.collect()  # objects of the earlier phases go now, not inside a timed call
    gc.disable()
    for _ in range(3):
        lib.ac_scan(dfa.h, ctypes.byref(desc_h), ctypes.byref(res_h), ctypes.byref(opts), sp, None)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    call_ms = []
    for _ in range(k_e2e):
        t1 = time.perf_counter()
        s = lib.ac_scan(dfa.h, ctypes.byref(desc_h), ctypes.byref(res_h), ctypes.byref(opts), sp, None)
        assert s == N.AC_OK, s
        call_ms.append(round((time.perf_counter() - t1) * 1e3, 2))  # ac_scan returns with its results on the host
    torch.cuda.synchronize()
    gc.enable()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    assert int(res_h.n_matches) == n_matches and int(cnt_h.sum()) == n_matches
    h2d_bytes, d2h_bytes = int(host_packed.numel() * 4), int(16 * n_matches + 8 * P + 16)
    # the host link in the same run: pinned copies of the same sizes, timed with CUDA events
    link = host_link_bandwidth(host_packed, raw_h, raw, stream)
    floor_ms = max(h2d_bytes / (link["h2d_gbs"] * 1e6), d2h_bytes / (link["d2h_gbs"] * 1e6))
    med = float(np.median(call_ms))
    out["e2e"] = {"value": round(k_e2e * n * world / e2e_s / 1e9, 3), "unit": UNIT,
                  "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes, "steps": k_e2e,
                  "call_ms": call_ms, "median_call_ms": med, "max_call_ms": float(np.max(call_ms)),
                  "value_at_median_call": round(n * world / (med / 1e3) / 1e9, 3),
                  # the call overlaps its copies in and out with the scan: the longer copy bounds it
                  "roofline": {"bound": "host link (pinned copies)", "h2d_gbs": link["h2d_gbs"],
                               "d2h_gbs": link["d2h_gbs"], "copy_floor_ms": round(floor_ms, 3),
                               "frac": round(floor_ms / med, 4), "how": link["how"]}}
    del host_packed, raw_h
    return out, (dfa, w, ascii_prefix)


def host_link_bandwidth(host_src: torch.Tensor, host_dst: torch.Tensor, dev_src: torch.Tensor, stream) -> dict:
    """Pinned host-to-device and device-to-host copy bandwidth (GB/s), each the best of three copies of
    the given buffers' sizes, timed with CUDA events on the stream."""
    dev_dst = torch.empty(host_src.numel(), dtype=host_src.dtype, device="cuda")
    res = {}
    for name, dst, src in (("h2d_gbs", dev_dst, host_src), ("d2h_gbs", host_dst, dev_src)):
        best = 1e30
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        res[name] = round(src.numel() * src.element_size() / (best / 1e3) / 1e9, 2)
    res["how"] = (f"best of 3 pinned copies: {host_src.numel() * host_src.element_size() / 1e6:.0f} MB in, "
                  f"{dev_src.numel() * dev_src.element_size() / 1e6:.0f} MB out, CUDA events")
    del dev_dst
    return res


# ------------------------------------------------------ lookup roofline


def lookup_probe(packed: torch.Tensor, n: int, steps: int = 3) -> dict:
    """Walk-only ceilings of the scan kernel on the resident text: machines
    whose keywords (uniform random) essentially never occur, so the time is
    the dependent table lookups alone. Three placements: a 100,000-keyword
    machine of the workload's shape (default shared-memory prefix + L2), the
    same machine entirely through L2, and a 100-keyword machine that fits in
    shared memory."""
    import ctypes

    import paper_1403_7294_gb300 as acg
    from paper_1403_7294_gb300 import _native as N
    from paper_1403_7294_gb300 import synth

    lib = acg.lib()
    sp = torch.cuda.current_stream().cuda_stream
    big = acg.build(synth.uniform_patterns(100_000, 20, 25, synth.BASE_SEED + 77))
    small = acg.build(synth.uniform_patterns(100, 8, 20, synth.BASE_SEED + 78))
    desc = N.Text(packed.data_ptr(), n, N.AC_TEXT_PACKED2, 1)
    raw = torch.empty((1 << 16, 2), dtype=torch.int64, device="cuda")
    out = {}
    for name, d, hot in (("uniform100k_default", big, -1), ("uniform100k_all_l2", big, 0),
                         ("uniform100_all_smem", small, -1)):
        o = N.ScanOpts()
        o.hot_states = hot
        r = N.Result(raw.data_ptr(), 1 << 16, 0, None, 1, 0, 0)
        st = N.ScanStats()
        ms = []
        for i in range(steps + 1):
            rc = lib.ac_scan(d.h, ctypes.byref(desc), ctypes.byref(r), ctypes.byref(o), sp, ctypes.byref(st))
            assert rc in (0, N.AC_ERR_OVERFLOW), rc
            if i:
                ms.append(st.scan_ms)
        t = float(np.median(ms))
        out[name] = {"states": d.info["n_states"], "hot_states": st.hot_states, "occurrences": int(r.n_matches),
                     "kernel_ms": round(t, 4), "gbases_s": round(n / t / 1e6, 2),
                     "walked_bases_per_s": round(st.bases_walked / (t / 1e3), 1), "stride": st.stride}
    big.close()
    small.close()
    return out


# --------------------------------------------------------- CPU baseline


def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_throughput(patterns, ascii_host: np.ndarray, target_s: float = 12.0, machine=None):
    """Single-threaded oracle over a bounded prefix of the workload text."""
    import oracle

    t0 = time.perf_counter()
    m = machine if machine is not None else oracle.Machine(patterns)
    build_s = time.perf_counter() - t0
    probe = min(len(ascii_host), 2_000_000)
    t0 = time.perf_counter()
    m.scan(ascii_host[:probe])
    dt = time.perf_counter() - t0
    k = int(min(len(ascii_host), max(probe, probe * target_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    pos, _, _ = m.scan(ascii_host[:k])
    dt = time.perf_counter() - t0
    return k, dt, build_s, len(pos)


def oracle_threaded(patterns, ascii_host: np.ndarray, threads: int, rate1: float, machine, target_s: float = 6.0):
    """The oracle's two threaded forms (Sec. IV.A approaches 1 and 2) at
    ``threads`` host threads, each on a prefix sized for about target_s."""
    import oracle

    lmax = max(len(p) for p in patterns)
    rows = []
    k = int(min(len(ascii_host), max(1 << 20, rate1 * threads * target_s)))
    t0 = time.perf_counter()
    pos, _, _ = oracle.scan_text_chunks(machine, ascii_host[:k], threads, lmax)
    dt = time.perf_counter() - t0
    rows.append({"form": "text ranges with an L_max-1 halo (approach 1)", "threads": threads,
                 "value": round(k / dt / 1e9, 6), "unit": UNIT, "bases": k, "occurrences": int(len(pos)),
                 "seconds": round(dt, 2)})
    split = oracle.pattern_split(patterns, threads)
    t0 = time.perf_counter()
    machines = oracle._run_threads([lambda piece=piece: oracle.Machine(piece) for _, piece in split], threads)
    build_s = time.perf_counter() - t0
    k = int(min(len(ascii_host), max(1 << 20, rate1 * target_s)))
    t0 = time.perf_counter()
    pos, _, _ = oracle.scan_pattern_split(split, ascii_host[:k], threads, machines)
    dt = time.perf_counter() - t0
    for mm in machines:
        mm.close()
    rows.append({"form": "keyword list split, one machine per thread (approach 2, the paper's)",
                 "threads": threads, "value": round(k / dt / 1e9, 6), "unit": UNIT, "bases": k,
                 "occurrences": int(len(pos)), "seconds": round(dt, 2), "build_s": round(build_s, 2)})
    return rows


def cpu_baseline(patterns, ascii_host):
    import oracle

    m = oracle.Machine(patterns)
    k, dt, build_s, occ = oracle_throughput(patterns, ascii_host)
    out = {"value": round(k / dt / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"first {k} bases of the workload text ({occ} occurrences), machine of all "
                     f"{len(patterns)} keywords built once in {build_s:.1f}s (not timed); {dt:.1f}s of scan"}
    out["threaded"] = oracle_threaded(patterns, ascii_host, host_threads(), k / dt, m)
    m.close()
    return out


def run_cpu_sweep(args, rank):
    """Host analogue of the paper's thread-count figures (Sec. V, Fig. 4-5):
    the oracle's two threaded forms at 1, 2, 4, ... host threads on a prefix
    of the workload text, with the speed-up over one thread."""
    if rank != 0:
        return None
    import oracle

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    # without a GPU to draw the full genome, a sample-sized text of the same model (its own keywords)
    w = make_workload("genome", args.n_bases if dev == "cuda" else args.sweep_bases, dev, 0)
    n_sample = min(int(w.text.ascii.numel()), args.sweep_bases)
    text = w.text.ascii[:n_sample].cpu().numpy()
    del w.text.ascii
    T = host_threads()
    counts = sorted({1, T} | {1 << i for i in range(8) if (1 << i) < T})
    m = oracle.Machine(w.patterns)
    lmax = max(len(p) for p in w.patterns)
    rows = []
    for form in ("text", "patterns"):
        base = None
        split_cache = {}
        for t in counts:
            if form == "text":
                t0 = time.perf_counter()
                pos, _, _ = oracle.scan_text_chunks(m, text, t, lmax)
                dt = time.perf_counter() - t0
                extra = {}
            else:
                split = split_cache.setdefault(t, oracle.pattern_split(w.patterns, t))
                t0 = time.perf_counter()
                machines = oracle._run_threads([lambda piece=piece: oracle.Machine(piece) for _, piece in split], t)
                build_s = time.perf_counter() - t0
                t0 = time.perf_counter()
                pos, _, _ = oracle.scan_pattern_split(split, text, t, machines)
                dt = time.perf_counter() - t0
                for mm in machines:
                    mm.close()
                extra = {"build_s": round(build_s, 3)}
            base = base or dt
            rows.append({"form": form, "threads": t, "seconds": round(dt, 3), "gbases_s": round(n_sample / dt / 1e9, 6),
                         "speedup": round(base / dt, 2), "occurrences": int(len(pos)), **extra})
            log(f"[bench/sweep] {form} T={t}: {dt:.2f}s")
    best = max(rows, key=lambda r: r["gbases_s"])
    return {"impl": "reference", "metric": METRIC, "value": best["gbases_s"], "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": round(n_sample / best["gbases_s"] / 1e6, 3),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"cpu-sweep-{w.name}-first{n_sample}b", "host_threads": T},
            "cpu_baseline": {"value": best["gbases_s"], "unit": UNIT, "cores": best["threads"], "kind": "oracle",
                             "sample": f"first {n_sample} bases of {w.name}"},
            "e2e": {"value": best["gbases_s"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sweep": rows}


# --------------------------------------------------------- batched (cfg 4)


def run_batched(args, steps: int):
    """The batch workload: one graph-replayed persistent launch over the 4,096 texts against a per-text
    loop of ac_scan. Both sides are timed on one clock at a time: device time by CUDA events (the plan's
    replays against the sum of every loop call's own event-timed device time, and the batch kernel
    against the sum of the loop's scan-kernel times) and host wall time (ac_scan_batch calls against the
    loop's calls, each of which waits for its count)."""
    import ctypes

    import paper_1403_7294_gb300 as acg
    from paper_1403_7294_gb300 import _native as N
    from paper_1403_7294_gb300 import synth

    lib = acg.lib()
    w = synth.batched(device="cuda")
    lens = [int(t.numel()) for t in w.texts]
    total = int(sum(lens))
    dfa = acg.build(w.patterns)
    packed = [acg.pack(t.contiguous()) for t in w.texts]
    whole = acg.pack(torch.cat([t for t in w.texts]))  # the batch as one text: the tuner's sample for the shape
    tuned = acg.autotune(dfa, whole, total)
    tuned_chunk = acg.autotune_batch(dfa, packed, lens)  # the work-item chunk, on the batch itself
    del w.texts, whole
    sp = torch.cuda.current_stream().cuda_stream
    # size outputs
    probe = acg.scan_batch(dfa, packed, encoding=N.AC_TEXT_PACKED2, n_bases=lens, capacity=1 << 20)
    n_occ = probe.n_matches
    cap = n_occ + 1024
    plan = acg.BatchPlan(dfa, packed, lens, capacity=cap)
    for _ in range(3):
        assert plan.run() == n_occ
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(steps):
        plan.run(sync=False)
    ev1.record()
    torch.cuda.synchronize()
    graph_ms = ev0.elapsed_time(ev1) / steps
    # the same batch through ac_scan_batch (host planning each call)
    raw = torch.empty((cap, 2), dtype=torch.int64, device="cuda")
    cnt = torch.empty(len(w.patterns), dtype=torch.int64, device="cuda")
    descs = (N.Text * len(packed))(*[N.Text(p.data_ptr(), n, N.AC_TEXT_PACKED2, 1) for p, n in zip(packed, lens)])
    r = N.Result(raw.data_ptr(), cap, 0, cnt.data_ptr(), 1, 0, 0)
    stt = N.ScanStats()
    for _ in range(2):
        lib.ac_scan_batch(dfa.h, descs, len(packed), ctypes.byref(r), None, sp, ctypes.byref(stt))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kern, bwalk = [], 0
    for _ in range(steps):
        assert lib.ac_scan_batch(dfa.h, descs, len(packed), ctypes.byref(r), None, sp, ctypes.byref(stt)) == 0
        kern.append(stt.scan_ms)
        bwalk = stt.bases_walked
    batch_call_ms = (time.perf_counter() - t0) * 1e3 / steps
    batch_shape = {k: getattr(stt, k) for k in ("stride", "chunk", "threads", "interleave", "hot_states", "grid")}
    if getattr(args, "minimal", False):  # replays and batch calls only: no per-text loop, no walk-only ceiling
        plan.close()
        bk = float(np.mean(kern))
        return {"workload": w.name, "texts": len(lens), "bases": total, "occurrences": n_occ,
                "states": dfa.info["n_states"], "tuned": {**tuned, "batch_chunk": tuned_chunk}, "shape": batch_shape,
                "graph_replay_gbases_s": round(total / (graph_ms / 1e3) / 1e9, 3),
                "graph_replay_ms": round(graph_ms, 4), "batch_call_wall_ms": round(batch_call_ms, 4),
                "batch_kernel_ms": round(bk, 4)}
    # the plain per-text loop: one ac_scan per text, each with its own event-timed device time
    single = [(N.Text(p.data_ptr(), n, N.AC_TEXT_PACKED2, 1)) for p, n in zip(packed, lens)]
    loop_passes = max(1, min(steps, 3))
    loop_dev, loop_kern = [], []
    st1 = N.ScanStats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    occ_loop = 0
    for _ in range(loop_passes):
        occ_loop, dev_ms, kern_ms = 0, 0.0, 0.0
        for i, d in enumerate(single):
            rr = N.Result(raw.data_ptr(), cap, 0, cnt.data_ptr(), 1, 0, 0)
            o = N.ScanOpts()
            o.hot_states = -1
            o.text_id = i
            assert lib.ac_scan(dfa.h, ctypes.byref(d), ctypes.byref(rr), ctypes.byref(o), sp, ctypes.byref(st1)) == 0
            occ_loop += rr.n_matches
            dev_ms += st1.total_ms
            kern_ms += st1.scan_ms
        loop_dev.append(dev_ms)
        loop_kern.append(kern_ms)
    loop_ms = (time.perf_counter() - t0) * 1e3 / loop_passes
    assert occ_loop == n_occ
    plan.close()
    loop_dev_ms, loop_kern_ms = float(np.median(loop_dev)), float(np.median(loop_kern))
    # walk-only ceiling of the batch kernel: the same texts and shape, 50,000 uniform keywords (no occurrences)
    uni = acg.build(synth.uniform_patterns(len(w.patterns), 15, 25, synth.BASE_SEED + 79))
    o_u = N.ScanOpts()
    o_u.hot_states, o_u.chunk = -1, batch_shape["chunk"]
    ru = N.Result(raw.data_ptr(), cap, 0, None, 1, 0, 0)
    su = N.ScanStats()
    uk = []
    for i in range(4):
        rc = lib.ac_scan_batch(uni.h, descs, len(packed), ctypes.byref(ru), ctypes.byref(o_u), sp, ctypes.byref(su))
        assert rc in (0, N.AC_ERR_OVERFLOW), rc
        if i:
            uk.append(su.scan_ms)
    uni.close()
    peak, peak_kind = load_peaks()
    bk = float(np.mean(kern))
    alg = total / 4 + 16 * n_occ + 8 * len(w.patterns) + 16 * dfa.info["n_states"]  # as the plain scan's
    return {
        "workload": w.name, "texts": len(lens), "bases": total, "occurrences": n_occ,
        "states": dfa.info["n_states"], "tuned": {**tuned, "batch_chunk": tuned_chunk}, "shape": batch_shape,
        "graph_replay_gbases_s": round(total / (graph_ms / 1e3) / 1e9, 3), "graph_replay_ms": round(graph_ms, 4),
        "batch_call_gbases_s": round(total / (batch_call_ms / 1e3) / 1e9, 3),
        "batch_call_wall_ms": round(batch_call_ms, 4),
        "batch_kernel_ms": round(bk, 4),
        "per_text_loop": {
            "device_ms": round(loop_dev_ms, 3), "device_gbases_s": round(total / (loop_dev_ms / 1e3) / 1e9, 3),
            "kernels_ms": round(loop_kern_ms, 3), "kernels_gbases_s": round(total / (loop_kern_ms / 1e3) / 1e9, 3),
            "wall_ms": round(loop_ms, 2), "wall_gbases_s": round(total / (loop_ms / 1e3) / 1e9, 3),
            "calls": len(single)},
        # ratios on one clock each
        "batched_over_loop_device": round(loop_dev_ms / graph_ms, 2),  # events: loop calls' device time vs replay
        "batch_kernel_over_loop_kernels": round(loop_kern_ms / bk, 2),  # events: scan kernels only
        "batched_over_loop_wall": round(loop_ms / batch_call_ms, 2),  # host wall: ac_scan loop vs ac_scan_batch
        "roofline": {"bound": "hbm", "kernel": "batch_kernel", "kernel_ms": round(bk, 4),
                     "algorithmic_bytes": int(alg), "achieved": round(alg / (bk / 1e3) / 1e9, 2), "peak": peak,
                     "unit": "GB/s", "frac": round(alg / (bk / 1e3) / 1e9 / peak, 5), "peak_source": peak_kind,
                     "walked_bases_per_s": round(bwalk / (bk / 1e3), 1),
                     "lookup": {"ceiling_kernel_ms": round(float(np.median(uk)), 4),
                                "ceiling_walked_bases_per_s": round(su.bases_walked / (float(np.median(uk)) / 1e3), 1),
                                "frac": round(float(np.median(uk)) / bk, 4),
                                "ceiling_source": "same texts, shape and chunk, 50,000 uniform keywords of 15-25 "
                                                  "(no occurrences)"}},
    }


# ---------------------------------------------------------- serving (cfg 5)


def run_serving(args, seconds: float, warm_s: float):
    import paper_1403_7294_gb300 as acg
    from paper_1403_7294_gb300 import synth

    t0 = time.time()
    genome = synth.markov_text(64 << 20, synth.BASE_SEED + 4, device="cuda")
    sets = synth.serve_sets(genome.ascii)
    g_host = genome.ascii.cpu().numpy()
    del genome
    dfas = [acg.build(s) for s in sets]
    log(f"[bench] serving: 8 machines ({sum(d.info['n_states'] for d in dfas)} states) in {time.time() - t0:.1f}s")
    srv = acg.Server(device_budget_bytes=40 << 30, n_streams=4, max_batch=256)
    slots = [srv.add_dfa(d) for d in dfas]
    n_req = int((seconds + warm_s) * 2000 * 1.1) + 10
    t_arr, lens, offs, which = synth.serve_requests(n_req, synth.BASE_SEED + 5, len(g_host))
    q: queue.Queue = queue.Queue()
    lat, done_bases, errors, sub_ms = [], [], [], []
    lock = threading.Lock()
    horizon = seconds + warm_s

    def waiter():
        while True:
            item = q.get()
            if item is None:
                return
            tk, slot, ts, n, counted = item
            try:
                srv.wait(tk, slot)  # exact size: one copy of the occurrences
                te = time.perf_counter()
                if counted:
                    with lock:
                        lat.append((te - ts) * 1e3)
                        done_bases.append((te, n))
            except Exception as e:  # noqa: BLE001
                errors.append(repr(e))

    ws = [threading.Thread(target=waiter, daemon=True) for _ in range(16)]
    [t.start() for t in ws]
    start = time.perf_counter()
    rejected = 0
    i = 0
    while i < n_req and t_arr[i] < horizon:
        now = time.perf_counter() - start
        if t_arr[i] > now:
            time.sleep(min(t_arr[i] - now, 0.002))
            continue
        a, n, s = int(offs[i]), int(lens[i]), int(which[i])
        ts = time.perf_counter()
        tk = srv.try_submit(slots[s], g_host[a : a + n])
        if t_arr[i] >= warm_s:
            sub_ms.append((time.perf_counter() - ts) * 1e3)  # the caller's side of submit: checks and copies
        if tk is None:
            rejected += 1
        else:
            q.put((tk, slots[s], ts, n, t_arr[i] >= warm_s))
        i += 1
    submit_end = time.perf_counter()
    for _ in ws:
        q.put(None)
    [t.join() for t in ws]
    end = time.perf_counter()
    st = srv.stats()
    srv.close()
    window = submit_end - (start + warm_s)
    bases_in_window = sum(n for te, n in done_bases)
    lat_a = np.array(lat) if lat else np.zeros(1)
    return {
        "workload": f"serve-8sets-{len(sets[-1])}maxpat-poisson2000hz-{seconds:.0f}s",
        "requests": len(lat), "rejected": rejected, "errors": len(errors),
        "p50_ms": round(float(np.percentile(lat_a, 50)), 3), "p99_ms": round(float(np.percentile(lat_a, 99)), 3),
        "mean_ms": round(float(lat_a.mean()), 3),
        "server_p50_ms": round(st["p50_ms"], 3), "server_p99_ms": round(st["p99_ms"], 3),  # submit -> results ready
        "submit_p99_ms": round(float(np.percentile(sub_ms, 99)), 3) if sub_ms else None,
        "sustained_gbases_s": round(bases_in_window / max(end - (start + warm_s), 1e-9) / 1e9, 3),
        "offered_gbases_s": round(float(lens[(t_arr >= warm_s) & (t_arr < horizon)].sum()) / window / 1e9, 3),
        "device_busy_gbases_s": round(st["gbases_per_s"], 3), "batches": st["batches_launched"],
        "overflow_batches": st["overflow_batches"],
        "warmup_s": warm_s,
    }


# ------------------------------------------ pattern-file split comparison


def run_partition(args, steps: int = 3) -> dict:
    """The paper's approach 2 (one machine per chunk of the keyword list, every
    machine scanning the whole text; here each machine sized for shared
    memory) against the single autotuned machine, on the 256 Mbase Markov
    chromosome, for keyword sets of 1,000 .. 100,000 (length 12-30)."""
    import ctypes

    import paper_1403_7294_gb300 as acg
    from paper_1403_7294_gb300 import _native as N
    from paper_1403_7294_gb300 import synth

    lib = acg.lib()
    sp = torch.cuda.current_stream().cuda_stream
    w = synth.plain_chromosome(device="cuda")
    n = int(w.text.ascii.numel())
    packed = acg.pack(w.text.ascii)
    sets = synth.serve_sets(w.text.ascii, sizes=[1000, 3728, 13895, 51795, 100000])
    desc = N.Text(packed.data_ptr(), n, N.AC_TEXT_PACKED2, 1)
    out = []
    for pats in sets:
        d = acg.build(pats)
        acg.autotune(d, packed, n)
        ps = acg.build_partitioned(pats)
        row = {"patterns": len(pats), "states": d.info["n_states"], "parts": ps.n_parts,
               "part_max_states": ps.max_states}
        for name, fn, h in (("single", lib.ac_scan, d.h), ("partitioned", lib.ac_scan_partitioned, ps.h)):
            r0 = N.Result(None, 0, 0, None, 1, 0, 0)
            o = N.ScanOpts()
            o.hot_states = -1
            fn(h, ctypes.byref(desc), ctypes.byref(r0), ctypes.byref(o), sp, None)
            cap = int(r0.n_matches) + 16
            raw = torch.empty((cap, 2), dtype=torch.int64, device="cuda")
            r = N.Result(raw.data_ptr(), cap, 0, None, 1, 0, 0)
            st = N.ScanStats()
            ms = []
            for _ in range(steps + 1):
                assert fn(h, ctypes.byref(desc), ctypes.byref(r), ctypes.byref(o), sp, ctypes.byref(st)) == 0
                ms.append(st.scan_ms)
            t = float(np.median(ms[1:]))
            row[name] = {"kernel_ms": round(t, 4), "gbases_s": round(n / t / 1e6, 2), "occurrences": int(r.n_matches)}
        assert row["single"]["occurrences"] == row["partitioned"]["occurrences"]
        out.append(row)
        ps.close()
        d.close()
    return {"workload": f"partition-{n}b-markov", "rows": out}


# -------------------------------------------- failure-less comparison


def run_failureless(args, steps: int = 3) -> dict:
    """Failure-less matching (one thread per start position over the trie
    edges, the scheme cited in Sec. II) against the failure-folded walk, on the
    1 Mbase / 100-keyword, 256 Mbase / 10,000-keyword and a 1 Gbase slice of
    the genome / 100,000-keyword workloads."""
    import ctypes

    import paper_1403_7294_gb300 as acg
    from paper_1403_7294_gb300 import _native as N

    lib = acg.lib()
    sp = torch.cuda.current_stream().cuda_stream
    rows = []
    for name, nb in (("small", None), ("chromosome", None), ("genome", 1_000_000_000)):
        w = make_workload(name, nb, "cuda", 0)
        n = int(w.text.ascii.numel())
        packed = acg.pack(w.text.ascii)
        del w.text.ascii
        d = acg.build(w.patterns, failureless=True)
        acg.autotune(d, packed, n)
        desc = N.Text(packed.data_ptr(), n, N.AC_TEXT_PACKED2, 1)
        row = {"workload": w.name, "states": d.info["n_states"]}
        for kind, fn in (("ac_walk", lib.ac_scan), ("failureless", lib.ac_scan_failureless)):
            o = N.ScanOpts()
            o.hot_states = -1
            r0 = N.Result(None, 0, 0, None, 1, 0, 0)
            fn(d.h, ctypes.byref(desc), ctypes.byref(r0), ctypes.byref(o), sp, None)
            cap = int(r0.n_matches) + 16
            raw = torch.empty((cap, 2), dtype=torch.int64, device="cuda")
            r = N.Result(raw.data_ptr(), cap, 0, None, 1, 0, 0)
            st = N.ScanStats()
            ms = []
            for _ in range(steps + 1):
                assert fn(d.h, ctypes.byref(desc), ctypes.byref(r), ctypes.byref(o), sp, ctypes.byref(st)) == 0
                ms.append(st.scan_ms)
            t = float(np.median(ms[1:]))
            row[kind] = {"kernel_ms": round(t, 4), "gbases_s": round(n / t / 1e6, 2), "occurrences": int(r.n_matches)}
        assert row["ac_walk"]["occurrences"] == row["failureless"]["occurrences"]
        rows.append(row)
        d.close()
        del packed
        torch.cuda.empty_cache()
    return {"rows": rows}


def run_stream(args, steps: int = 3) -> dict:
    """A long text delivered in consecutive device-resident pieces through
    ac_stream_scan (carried L_max-1 bases, global positions) against one
    ac_scan of the whole text, at several piece sizes; both wall-clock timed
    per pass (every call returns its exact occurrence count)."""
    import ctypes

    import paper_1403_7294_gb300 as acg
    from paper_1403_7294_gb300 import _native as N

    lib = acg.lib()
    sp = torch.cuda.current_stream().cuda_stream
    w = make_workload("genome", args.n_bases, "cuda", 0)
    n = int(w.text.ascii.numel())
    packed = acg.pack(w.text.ascii)
    del w.text.ascii
    torch.cuda.empty_cache()
    d = acg.build(w.patterns)
    acg.autotune(d, packed, n)
    o = N.ScanOpts()
    o.hot_states = -1
    whole = N.Text(packed.data_ptr(), n, N.AC_TEXT_PACKED2, 1)
    r0 = N.Result(None, 0, 0, None, 1, 0, 0)
    lib.ac_scan(d.h, ctypes.byref(whole), ctypes.byref(r0), ctypes.byref(o), sp, None)
    k = int(r0.n_matches)
    raw = torch.empty((k + 16, 2), dtype=torch.int64, device="cuda")
    cnt = torch.empty(len(w.patterns), dtype=torch.int64, device="cuda")

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            t0 = time.perf_counter()
            got = fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            assert got == k, (got, k)
        return float(np.median(ts))

    def one_shot():
        r = N.Result(raw.data_ptr(), k + 16, 0, cnt.data_ptr(), 1, 0, 0)
        assert lib.ac_scan(d.h, ctypes.byref(whole), ctypes.byref(r), ctypes.byref(o), sp, None) == 0
        return int(r.n_matches)

    t_one = timed(one_shot)
    rows = []
    s = acg.Stream(d)
    for piece in (1 << 24, 1 << 26, 1 << 28):
        spans = [(a, min(piece, n - a)) for a in range(0, n, piece)]

        def streamed():
            assert lib.ac_stream_reset(s.h) == 0
            got = 0
            for a, ln in spans:  # a is a multiple of 16 bases: the piece starts on a word
                desc = N.Text(packed.data_ptr() + a // 4, ln, N.AC_TEXT_PACKED2, 1)
                r = N.Result(raw.data_ptr() + 16 * got, k + 16 - got, 0, cnt.data_ptr(), 1, 0, 0)
                assert lib.ac_stream_scan(s.h, ctypes.byref(desc), ctypes.byref(r), ctypes.byref(o), sp, None) == 0
                got += int(r.n_matches)
            return got

        t = timed(streamed)
        rows.append({"piece_bases": piece, "pieces": len(spans), "wall_ms": round(t * 1e3, 3),
                     "gbases_s": round(n / t / 1e9, 2)})
        log(f"[bench/stream] piece {piece}: {t * 1e3:.2f} ms")
    s.close()
    return {"workload": f"stream-{w.name}", "occurrences": k,
            "one_shot": {"wall_ms": round(t_one * 1e3, 3), "gbases_s": round(n / t_one / 1e9, 2)}, "rows": rows}


# ------------------------------------------------------- reference arm


def run_reference(args, world, rank):
    if rank != 0:
        return None
    from paper_1403_7294_gb300 import synth

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t0 = time.time()
    if dev == "cuda":
        w = make_workload(args.workload, args.n_bases, dev, 0)
        text = w.text.ascii[: min(w.text.ascii.numel(), 400_000_000)].cpu().numpy()
        n_full = int(w.text.ascii.numel())
        del w.text.ascii
    else:  # no GPU to draw the full text: draw a sample-sized text of the same model
        w = make_workload(args.workload, min(args.n_bases or 1 << 26, 1 << 26), dev, 0)
        text = w.text.ascii.numpy()
        n_full = int(text.size)
    log(f"[bench/ref] workload ready in {time.time() - t0:.1f}s")
    import oracle

    m = oracle.Machine(w.patterns)
    # size the per-step sample so the whole run ends within a few minutes
    probe = min(text.size, 1_000_000)
    t1 = time.perf_counter()
    m.scan(text[:probe])
    rate = probe / max(time.perf_counter() - t1, 1e-6)
    per_step_s = max(0.5, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    k = int(min(text.size, max(probe, rate * per_step_s)))
    for _ in range(args.warmup):
        m.scan(text[:k])
    times = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        m.scan(text[:k])
        times.append(time.perf_counter() - t1)
    total = sum(times)
    value = args.steps * k / total / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": w.name, "n_bases": n_full, "patterns": len(w.patterns)},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {k} bases of the workload text per step"},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# -------------------------------------------------------------------- main


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload",
                    choices=["genome", "chromosome", "small", "batch", "serve", "partition", "failureless",
                             "stream", "cpu-sweep"],
                    default="genome")
    ap.add_argument("--sweep-bases", type=int, default=32_000_000,
                    help="cpu-sweep: bases of the genome text each thread count scans")
    ap.add_argument("--n-bases", type=int, default=None)
    ap.add_argument("--minimal", action="store_true",
                    help="scan timing only (no e2e, CPU baseline or extras; batch: no per-text loop or ceiling)")
    ap.add_argument("--shape", default=None,
                    help="plain workloads: fixed launch shape 'stride,threads,interleave,hot_states' instead of autotuning")
    ap.add_argument("--serve-seconds", type=float, default=None)
    ap.add_argument("--uniform-patterns", action="store_true",
                    help="replace the keywords by uniform random ones of the same shape (walk-only ceiling)")
    args = ap.parse_args()
    if args.warmup < 3 and not args.minimal:
        log("[bench] warmup raised to 3")
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.workload == "cpu-sweep":  # the oracle only (host threads), either --impl
        out = run_cpu_sweep(args, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, world, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for --impl ours")
    import paper_1403_7294_gb300 as acg

    acg.lib()  # fail loudly if the library is missing
    if args.workload == "batch":
        out = {"metric": METRIC, "unit": UNIT}
        b = run_batched(args, args.steps)
        out.update({"value": b["graph_replay_gbases_s"], "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                    "ms_per_step": b["graph_replay_ms"], "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": {"workload": b["workload"]},
                    "batched": b})
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.workload == "failureless":
        fl = run_failureless(args)
        out = {"metric": METRIC, "value": fl["rows"][-1]["ac_walk"]["gbases_s"], "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "u32", "data": "synthetic",
               "config": {"workload": "failureless-comparison"}, "failureless": fl}
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.workload == "stream":
        sm = run_stream(args)
        best = max(r["gbases_s"] for r in sm["rows"])
        out = {"metric": METRIC, "value": best, "unit": UNIT, "n_gpus": world, "steps": 3, "warmup": 1,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
               "data": "synthetic", "config": {"workload": sm["workload"]}, "stream": sm}
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.workload == "partition":
        pt = run_partition(args)
        best = max(r["single"]["gbases_s"] for r in pt["rows"])
        out = {"metric": METRIC, "value": best, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
               "data": "synthetic", "config": {"workload": pt["workload"]}, "partition": pt}
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.workload == "serve":
        s = run_serving(args, args.serve_seconds or 60.0, 5.0)
        out = {"metric": METRIC, "value": s["sustained_gbases_s"], "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": {"workload": s["workload"]},
               "serving": s}
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    out, keep = run_plain(args, world, rank, local)
    if keep is not None and rank == 0 and world == 1:
        dfa, w, ascii_prefix = keep
        del dfa
        torch.cuda.empty_cache()
        try:
            out["cpu_baseline"] = cpu_baseline(w.patterns, ascii_prefix)
        except Exception as e:  # noqa: BLE001
            out["cpu_baseline"] = {"value": None, "error": repr(e)}
        if args.workload == "genome" and world == 1:
            out["batched"] = run_batched(args, max(3, args.steps))
            out["serving"] = run_serving(args, args.serve_seconds or 60.0, 5.0)
            out["plain_configs"] = run_plain_configs(args, world, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
