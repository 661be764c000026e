#!/usr/bin/env python3
"""Benchmark of the GB300 Parquet scan: decoded GB/s and % of HBM roofline.

Workload (default): the eight-column synthetic table of 2^26 rows (seeded,
shaped like the paper's scan workloads; it stands in for TPC-H lineitem),
row groups of 2^23 rows, 1 MiB pages, uncompressed, written by the engine's
own writer and staged in device memory before timing.

A step is one pass of the whole scan path over the table:
  pq_index_chunks (footer read + page-header index) -> pq_plan_scan ->
  pq_scan_columns -> pq_scan_wait (device status checked).
`value` = decoded bytes (values + validity + offsets + chars) / step time,
summed over ranks (weak scaling: each rank scans its own table).

Extra keys: `roofline` for one scan launch (all stages of pq_scan_columns,
replayed from a CUDA graph): (stored bytes read + decoded bytes written) /
scan time vs the measured HBM copy bandwidth; `stages` (ms per stage);
`e2e` through pq_scan_host from pinned host buffers; `cpu_baseline` (the
CPU oracle decoding a bounded sample on the host cores); `clocks` sampled by
nvidia-smi during the timed region; `gpu_launches` kernels launched in it.

`--impl reference` times the CPU oracle (the reference arm of this project)
on the same workload, a bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

MiB = 1 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rows", type=int, default=1 << 26)
    ap.add_argument("--table", default="eight", choices=["eight", "v2"],
                    help="scan: the eight-column table, or the six-column table of the other V2 encodings "
                         "(BYTE_STREAM_SPLIT, DELTA_LENGTH_BYTE_ARRAY, DELTA_BYTE_ARRAY)")
    ap.add_argument("--rg-rows", type=int, default=1 << 23)
    ap.add_argument("--page-bytes", type=int, default=MiB)
    ap.add_argument("--codec", default="UNCOMPRESSED", choices=["UNCOMPRESSED", "SNAPPY", "ZSTD"])
    ap.add_argument("--page-version", type=int, default=1)
    ap.add_argument("--mode", default="batched", choices=["batched", "plain"])
    ap.add_argument("--no-offset-index", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scan-reps", type=int, default=10, help="graph replays for the roofline")
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--workload", default="scan", choices=["scan", "serve", "batched", "single"],
                    help="scan: one table, index+plan+scan per step; serve: Poisson requests through pq_serve_*; "
                         "batched: many uneven single-column files in one graph launch vs plain launches; "
                         "single: one dictionary INT32 column, plain one-page-per-block vs batched")
    ap.add_argument("--c4-files", type=int, default=256)
    ap.add_argument("--c4-chunks-per-file", type=int, default=4)
    ap.add_argument("--c4-rows-lo", type=float, default=1e4)
    ap.add_argument("--c4-rows-hi", type=float, default=1e6)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serve-files", type=int, default=4, help="serve: tables in the catalog index")
    ap.add_argument("--serve-requests", type=int, default=10000, help="serve: requests per offered-load point")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="serve: arrivals stop after this many seconds at a load point")
    ap.add_argument("--serve-max-pending", type=int, default=256,
                    help="serve: arrivals while this many requests are pending are shed (counted, not sent)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="serve: mean arrivals per second at 1x")
    ap.add_argument("--serve-loads", default="0.125,0.25,0.5,1", help="serve: offered-load multipliers")
    ap.add_argument("--serve-budget-gib", type=float, default=64.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    return ap.parse_args()


def workload_name(a):
    table = "six-column V2-encoding table" if getattr(a, "table", "eight") == "v2" else "eight-column table"
    return (f"{table}, {a.rows} rows, row groups of {a.rg_rows} rows, "
            f"{a.page_bytes // 1024} KiB pages, {a.codec.lower()}, V{a.page_version} pages")


def table_and_spec(a, rank):
    if getattr(a, "table", "eight") == "v2":
        tab = synth.v2_encodings_table(a.rows, a.rg_rows, file=rank)
        spec = synth.v2_encodings_spec(a.rg_rows, a.page_bytes, a.codec, a.page_version,
                                       offset_index=not a.no_offset_index)
    else:
        tab = synth.config2_table(a.rows, a.rg_rows, file=rank)
        spec = synth.config2_spec(a.rg_rows, a.page_bytes, a.codec, a.page_version,
                                  offset_index=not a.no_offset_index)
    return tab, spec


def make_files(a, rank):
    """The table of this rank, written by the engine's native writer."""
    from paper_2602_17335_gb300.tables import write_table
    tab, spec = table_and_spec(a, rank)
    return write_table(tab, spec)


def make_first_row_group_with_oracle(a):
    """Row group 0 of rank 0's table (the part the CPU sample decodes),
    written by the CPU oracle's writer: the same chunk bytes as in the full
    file, and the reference arm never loads the engine library."""
    from oracle import writer as W
    tab, spec = table_and_spec(a, 0)
    hi = min(a.rg_rows, tab.n_rows)
    first = synth.Table([synth.slice_column(c, 0, hi) for c in tab.columns])
    return W.write_file(first, spec)


# ----------------------------------------------------------------- CPU oracle sample

def oracle_sample(data, max_seconds=20.0, pages_per_chunk=1):
    """Decodes, with the CPU oracle, the dictionary page and the first
    `pages_per_chunk` data pages of each chunk of the first row group;
    returns (decoded bytes, seconds, description)."""
    from oracle import reader as R
    data = bytes(data)
    info = R.parse_footer(data)
    chunks = [c for c in info.chunks if c.rg == 0]
    decoded = 0
    pages = 0
    t0 = time.perf_counter()
    for ch in chunks:
        plist = R.chunk_pages(data, ch)
        dictionary = None
        n = 0
        for p in plist:
            if p.page_type == 2:
                dictionary = R.decode_dictionary(data, p, ch)
                continue
            vals, valid = R.decode_data_page(data, p, ch, dictionary)
            rows = p.num_values
            if ch.ptype == "BYTE_ARRAY":
                decoded += 8 * rows + sum(len(v) for v in vals)
            else:
                decoded += vals.nbytes
            if valid is not None:
                decoded += rows / 8
            pages += 1
            n += 1
            if n >= pages_per_chunk or time.perf_counter() - t0 > max_seconds:
                break
    dt = time.perf_counter() - t0
    return decoded, dt, f"first {pages_per_chunk} data page(s) + dictionary of each of the {len(chunks)} chunks of row group 0 ({pages} pages)"


def cpu_count_used():
    return 1  # the oracle is single-threaded Python + numpy


def _oracle_unit(args):
    """One chunk's part of the sample (dictionary page + first data page),
    decoded by the oracle in a worker process; returns decoded bytes."""
    from oracle import reader as R
    blob, pages, ch = args
    dictionary = None
    decoded = 0
    for p in pages:
        if p.page_type == 2:
            dictionary = R.decode_dictionary(blob, p, ch)
            continue
        vals, valid = R.decode_data_page(blob, p, ch, dictionary)
        rows = p.num_values
        decoded += 8 * rows + sum(len(v) for v in vals) if ch.ptype == "BYTE_ARRAY" else vals.nbytes
        if valid is not None:
            decoded += rows / 8
    return decoded


def pyarrow_context(data, decoded_bytes, reps=2):
    """Context point, not the oracle: pyarrow's multithreaded reader on the
    same file bytes in host memory, as decoded GB/s (best of `reps`)."""
    try:
        import pyarrow as pa
        import pyarrow.parquet as pq
    except ImportError:
        return {"unavailable": "pyarrow is not installed on this host"}
    buf = pa.py_buffer(bytes(data))
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        pq.read_table(pa.BufferReader(buf), use_threads=True)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return {"value": decoded_bytes / best / 1e9, "unit": "GB/s", "cores": os.cpu_count(),
            "kind": "pyarrow read_table, all threads (context, not the oracle)", "seconds": best}


def oracle_sample_all_cores(data):
    """The oracle_sample workload with the chunks as independent units over a
    process pool (spawn), one worker per unit up to the host's cores; each
    worker gets only its chunk's dictionary and first data page bytes.
    Returns (decoded bytes, seconds, workers)."""
    import dataclasses
    import multiprocessing as mp
    from oracle import reader as R
    data = bytes(data)
    info = R.parse_footer(data)
    units = []
    for ch in (c for c in info.chunks if c.rg == 0):
        plist = R.chunk_pages(data, ch)
        keep = [p for p in plist if p.page_type == 2][:1] + [p for p in plist if p.page_type != 2][:1]
        base = min(p.offset for p in keep)
        end = max(p.offset + p.header_len + p.compressed for p in keep)
        units.append((bytes(data[base:end]), [dataclasses.replace(p, offset=p.offset - base) for p in keep], ch))
    workers = max(1, min(len(units), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        pool.map_async(_oracle_unit, units[:workers]).get(timeout=300)  # workers started and warm
        t0 = time.perf_counter()
        decoded = sum(pool.map_async(_oracle_unit, units, chunksize=1).get(timeout=300))
        dt = time.perf_counter() - t0
    return decoded, dt, workers


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region, plus the
    sample delivered just before it starts and one taken synchronously as
    soon as it ends, so a region shorter than the sampling period still has
    a record."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            # the raw samples go to $PQ_CLOCKS_CSV when set (the summary is in the JSON line)
            self.out = open(os.environ.get("PQ_CLOCKS_CSV") or os.devnull, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.lines = []
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the timed region starts once the sampler has delivered a sample
            # (taken just after the warm-up, so the clocks are those under load)
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.n_before = len(self.lines)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _one_sample(self):
        try:
            r = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            return [ln.strip() for ln in r.stdout.splitlines() if ln.strip()]
        except (OSError, subprocess.TimeoutExpired):
            return []

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            if self.out:
                self.out.write(line)

    def __exit__(self, *exc):
        if self.proc:
            self.n_during = len(self.lines) - getattr(self, "n_before", 0)
            after = self._one_sample()
            self.lines.extend(after)
            self.n_after = len(after)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)
        if self.out:
            self.out.close()

    def summary(self):
        if not self.proc or not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "samples_before_during_after": [getattr(self, "n_before", 0),
                                                                    getattr(self, "n_during", 0),
                                                                    getattr(self, "n_after", 0)]}


# ----------------------------------------------------------------- arms

# DRAM traffic of one scan launch, from one ncu capture of the NVTX range
# "roofline_scan" (dram__bytes_read.sum + dram__bytes_write.sum summed over
# the launch's kernels).  Keyed by the layout; the capture's row count scales
# the figure to the bench's rows (traffic grows with rows at a fixed layout).
# `sources` is the digest of the kernel sources the counters were taken on
# (the decompression kernels only for the codec that the layout uses, as the
# others do not run): once they change, the stored figure no longer describes
# the kernels and the bench reports null.
TRAFFIC_CAPTURES = {
    # profiles/traffic_eight_column_2p24_1MiB.md
    "8388608/1048576/UNCOMPRESSED/V1/batched/oi1": {"rows": 16777216, "bytes": 1349122816, "sources": "bad20e27c405ef12"},
}

KERNEL_SOURCES = ("k_decode.cu", "k_transcode.cu", "dev_util.cuh", "thrift_dev.cuh", "decode_job.h",
                  "pq_internal.h", "snappy_job.h", "engine.cpp")
CODEC_SOURCES = {"SNAPPY": ("k_snappy.cu",), "ZSTD": ("k_zstd.cu", "zstd_dec.cuh")}


def kernel_sources_digest(codec="UNCOMPRESSED"):
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES + CODEC_SOURCES.get(codec, ()):
        with open(os.path.join(ROOT, "paper_2602_17335_gb300", "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def traffic_key(a):
    table = "v2/" if getattr(a, "table", "eight") == "v2" else ""
    return f"{table}{a.rg_rows}/{a.page_bytes}/{a.codec}/V{a.page_version}/{a.mode}/oi{int(not a.no_offset_index)}"


def stored_traffic(a):
    """(bytes per scan launch at a.rows, note) or (None, why)."""
    cap = TRAFFIC_CAPTURES.get(traffic_key(a))
    if cap is None:
        return None, "no capture for this layout"
    if cap["sources"] != kernel_sources_digest(a.codec):
        return None, "kernels changed since the capture"
    return cap["bytes"] * a.rows / cap["rows"], f"ncu capture at {cap['rows']} rows, scaled by rows"


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def run_reference(a, rank, world):
    """The CPU oracle on the same workload (bounded sample per step)."""
    if rank != 0:
        return
    data = bytes(make_first_row_group_with_oracle(a))
    # each step a bounded sample, sized so that the whole run stays within a
    # few minutes
    per_step = max(0.3, min(20.0, 90.0 / max(1, a.steps + a.warmup)))
    for _ in range(a.warmup):
        oracle_sample(data, max_seconds=per_step)
    tot_b, tot_s = 0.0, 0.0
    desc = ""
    for _ in range(a.steps):
        b, s, desc = oracle_sample(data, max_seconds=per_step)
        tot_b += b
        tot_s += s
    value = tot_b / tot_s / 1e9
    line = {"impl": "reference", "metric": "decoded GB/s", "value": value, "unit": "GB/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot_s / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": workload_name(a), "rows": a.rows, "rg_rows": a.rg_rows,
                       "page_bytes": a.page_bytes, "codec": a.codec},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cpu_count_used(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x, world):
    """The largest x over the ranks: a multi-GPU step is as slow as its
    slowest rank.  NCCL groups reduce on the rank's GPU, gloo on the host."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    """The sum of x over the ranks (bytes every rank decoded)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_gbs(bytes_all_ranks, seconds):
    """Weak scaling: every rank scans its own table of the same shape (the
    ranks' data differ by seed only); the job's rate is the bytes all ranks
    decoded over the slowest rank's time."""
    return bytes_all_ranks / seconds / 1e9


def run_ours(a, rank, world, local_rank):
    import torch
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.scan import Engine, alloc_outputs, stream_handle

    if a.no_offset_index:
        os.environ["PQ_NO_OFFSET_INDEX"] = "1"
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    t0 = time.time()
    data = make_files(a, rank)
    gen_s = time.time() - t0
    files = [torch.from_numpy(data).to(dev)]
    stream = torch.cuda.current_stream(dev)
    sh = stream_handle(stream)
    eng = Engine(local_rank)
    base_flags = N.PQ_SCAN_PLAIN if a.mode == "plain" else N.PQ_SCAN_BATCHED

    # sizes and outputs (allocated once, reused by every step)
    idx = eng.index(files)
    iinfo = N.pq_index_get_info(idx)
    plan, sizes = eng.plan(idx, flags=base_flags)
    pinfo = N.pq_plan_get_info(plan)
    outs = alloc_outputs(sizes, dev)
    N.pq_free_plan(plan)
    N.pq_free_index(idx)
    index_launches = 3 if iinfo.used_offset_index else 2

    host_s = [0.0] * 6  # index, plan, scan enqueue, wait, free plan, free index (host seconds)

    def step():
        tp = [time.perf_counter()]
        ix = N.pq_index_chunks(eng.ctx, [(f.data_ptr(), f.numel()) for f in files], sh)
        tp.append(time.perf_counter())
        pl, _ = N.pq_plan_scan(eng.ctx, ix, None, 0, -1, base_flags)
        tp.append(time.perf_counter())
        N.pq_scan_columns(eng.ctx, pl, [o.desc() for o in outs], sh)
        tp.append(time.perf_counter())
        st, _ = N.pq_scan_wait(eng.ctx, pl, len(outs), sh)
        tp.append(time.perf_counter())
        N.pq_free_plan(pl)
        tp.append(time.perf_counter())
        N.pq_free_index(ix)
        tp.append(time.perf_counter())
        for i in range(6):
            host_s[i] += tp[i + 1] - tp[i]
        if st != N.PQ_OK:
            raise N.PqError(st, N.pq_last_error(eng.ctx))

    for _ in range(max(a.warmup, 1)):
        step()
    torch.cuda.synchronize(dev)
    host_s[:] = [0.0] * 6
    if world > 1:
        torch.distributed.barrier()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize(dev)
        start.record(stream)
        for _ in range(a.steps):
            step()
        end.record(stream)
        torch.cuda.synchronize(dev)
    step_ms = max_over_ranks(start.elapsed_time(end) / a.steps, world)
    decoded = float(pinfo.decoded_bytes)
    read = float(pinfo.read_bytes)
    decoded_all = sum_over_ranks(decoded, world)
    value = whole_job_gbs(decoded_all, step_ms * 1e-3)

    # roofline: one scan launch = all stages of pq_scan_columns, replayed from a graph
    idx = eng.index(files)
    plan, _ = eng.plan(idx, flags=base_flags | (0 if a.mode == "plain" else N.PQ_SCAN_GRAPH))
    for _ in range(3):
        eng.scan(plan, outs, stream)
    torch.cuda.synchronize(dev)
    # one scan launch inside an NVTX range: the launch an ncu capture of the
    # range measures (traffic), outside the timed replays
    try:
        torch.cuda.nvtx.range_push("roofline_scan")
        eng.scan(plan, outs, stream)
    finally:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(a.scan_reps):
        eng.scan(plan, outs, stream)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    st, chars = eng.wait(plan, len(outs))
    assert st == N.PQ_OK, N.pq_last_error(eng.ctx)
    scan_ms = s0.elapsed_time(s1) / a.scan_reps
    N.pq_free_plan(plan)
    # per-stage breakdown
    plan, _ = eng.plan(idx, flags=base_flags | N.PQ_SCAN_TIMING)
    for _ in range(2):
        eng.scan(plan, outs, stream)
        eng.wait(plan, len(outs))
    stages = N.pq_plan_stage_ms(plan)
    N.pq_free_plan(plan)
    N.pq_free_index(idx)
    peak, peak_kind = measured_peak()
    achieved = (read + decoded) / (scan_ms * 1e-3) / 1e9
    traffic, traffic_note = stored_traffic(a)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_note": traffic_note, "peak_kind": peak_kind,
                "kernel": "one scan launch (prepare, snappy, dict, walk, expand, strings; CUDA graph)",
                "algorithmic_bytes": read + decoded, "scan_ms": scan_ms,
                "scan_decoded_gbs": decoded / (scan_ms * 1e-3) / 1e9}

    # end to end through pq_scan_host (pinned host buffers, copies timed)
    e2e = None
    if not a.no_e2e:
        host_file = torch.from_numpy(data).pin_memory()
        hfiles = [(host_file.data_ptr(), host_file.numel())]
        hsizes = N.pq_scan_host(eng.ctx, hfiles)
        houts, keep = [], []
        for s in sizes:
            c = N.pq_column()
            v = torch.empty(int(s.values_bytes), dtype=torch.uint8).pin_memory()
            keep.append(v)
            c.values = v.data_ptr()
            if s.validity_bytes:
                m = torch.empty(int(s.validity_bytes), dtype=torch.uint8).pin_memory()
                keep.append(m)
                c.validity = m.data_ptr()
            if s.chars_bytes:
                ch = torch.empty(int(s.chars_bytes), dtype=torch.uint8).pin_memory()
                keep.append(ch)
                c.chars = ch.data_ptr()
                c.chars_capacity = int(s.chars_bytes)
            houts.append(c)
        del hsizes
        d2h = int(sum(s.values_bytes + s.validity_bytes for s in sizes) + sum(
            int(s.chars_bytes) for s in sizes))
        # the same call without the row-group pipeline (PQ_HOST_NO_PIPELINE):
        # the whole file copied in, then indexed and scanned, then the columns
        # copied out, one after another (the blocking reading that Section 4
        # sets against overlap).  The two alternate call by call, so that both
        # see the same host link (other jobs on the node share its memory
        # bandwidth), and each reports the median over its calls.
        def one(blocking):
            if blocking:
                os.environ["PQ_HOST_NO_PIPELINE"] = "1"
            try:
                t0 = time.perf_counter()
                N.pq_scan_host(eng.ctx, hfiles, outs=houts)
                return time.perf_counter() - t0
            finally:
                os.environ.pop("PQ_HOST_NO_PIPELINE", None)
        one(False)
        one(True)
        reps = max(3, min(a.steps, 7))
        t_pipe, t_blk = [], []
        for _ in range(reps):
            t_pipe.append(one(False))
            t_blk.append(one(True))
        e2e_s = max_over_ranks(float(np.median(t_pipe)), world)
        blk_s = max_over_ranks(float(np.median(t_blk)), world)
        e2e = {"value": whole_job_gbs(decoded_all, e2e_s), "unit": "GB/s", "h2d_bytes_per_step": int(data.nbytes),
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3, "statistic": f"median of {reps} calls",
               "calls_ms": [round(t * 1e3, 2) for t in t_pipe],
               "blocking": {"value": whole_job_gbs(decoded_all, blk_s), "unit": "GB/s", "ms_per_step": blk_s * 1e3,
                            "calls_ms": [round(t * 1e3, 2) for t in t_blk],
                            "overlapped_speedup": blk_s / e2e_s}}
        del keep

    cpu = cpu_all = ctx_pa = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        ctx_pa = pyarrow_context(data, decoded)
        b, s, desc = oracle_sample(bytes(data), max_seconds=25.0)
        cpu = {"value": b / s / 1e9, "unit": "GB/s", "cores": cpu_count_used(), "kind": "oracle", "sample": desc,
               "seconds": s}
        try:
            b2, s2, w = oracle_sample_all_cores(data)
            cpu_all = {"value": b2 / s2 / 1e9, "unit": "GB/s", "cores": w, "kind": "oracle", "sample": desc +
                       ", one process per chunk", "seconds": s2}
        except Exception as exc:  # a host without process pools still reports the one-core figure
            cpu_all = {"unavailable": repr(exc)[:200]}

    line = {"metric": "decoded GB/s", "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": workload_name(a), "rows": a.rows, "rg_rows": a.rg_rows,
                       "page_bytes": a.page_bytes, "codec": a.codec, "page_version": a.page_version,
                       "mode": a.mode, "offset_index": not a.no_offset_index,
                       "l2": "inputs larger than L2 (files %.2f GB, outputs %.2f GB per step)" % (
                           data.nbytes / 1e9, decoded / 1e9),
                       "step": "index + plan + scan + wait"},
            "roofline": roofline, "stages_ms": stages,
            "step_host_ms": dict(zip(("index", "plan", "scan_enqueue", "wait", "free_plan", "free_index"),
                                     (1e3 * x / a.steps for x in host_s))), "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "cpu_context_pyarrow": ctx_pa, "e2e": e2e,
            "gpu_launches": a.steps * (index_launches + pinfo.launches_per_scan),
            "clocks": clk.summary(),
            "detail": {"decoded_bytes": decoded, "read_bytes": read, "pages": pinfo.n_pages,
                       "items": pinfo.n_items, "data_pages_indexed": iinfo.n_data_pages,
                       "write_seconds": gen_s}}
    eng.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
        if a.json_out:
            with open(a.json_out, "w") as f:
                json.dump(line, f, indent=1)


# ----------------------------------------------------------------- serving (Poisson requests)

def serve_catalog(a):
    """Tables sharing the eight-column schema, one per layout: row groups of
    2^23 rows with 64 KiB and 1 MiB pages, uncompressed and Snappy."""
    from paper_2602_17335_gb300.tables import write_table
    layouts = [(64 * 1024, "UNCOMPRESSED"), (MiB, "UNCOMPRESSED"), (64 * 1024, "SNAPPY"), (MiB, "SNAPPY")]
    files = []
    for f in range(a.serve_files):
        pb, codec = layouts[f % len(layouts)]
        tab = synth.config2_table(a.rows, a.rg_rows, file=f)
        spec = synth.config2_spec(a.rg_rows, pb, codec, 1)
        if codec == "SNAPPY":
            for c in spec.columns:
                c.compress_threshold = -1.0
        files.append((write_table(tab, spec), f"{pb // 1024} KiB pages, {codec.lower()}"))
    return files


def request_stream(a, n, rate, seed, total_rows):
    """Open-loop Poisson arrivals; columns log-uniform over 1..8 (a random
    subset), rows log-uniform over [2^20, 2^28), start uniform (ranges wrap)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    out = []
    for i in range(n):
        k = int(np.clip(np.floor(np.exp(rng.uniform(0, np.log(9)))), 1, 8))
        cols = sorted(rng.choice(8, k, replace=False).tolist())
        rows = int(np.exp(rng.uniform(np.log(2 ** 20), np.log(2 ** 28))))
        start = int(rng.integers(0, total_rows))
        out.append((float(t[i]), cols, start, rows))
    return out


def run_serve(a):
    import torch
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.scan import Engine
    t0 = time.time()
    files = serve_catalog(a)
    gen_s = time.time() - t0
    dev_files = [torch.from_numpy(d).cuda() for d, _ in files]
    eng = Engine(0)
    idx = eng.index(dev_files)
    info = N.pq_index_get_info(idx)
    srv = N.pq_serve_create(eng.ctx, idx, int(a.serve_budget_gib * (1 << 30)), a.serve_slots)
    points = []
    with ClockSampler(0) as clk:
        for li, mult in enumerate(float(x) for x in a.serve_loads.split(",")):
            rate = a.serve_rate * mult
            reqs = request_stream(a, a.serve_requests, rate, 1000 + li, info.num_rows)
            reqs = [r for r in reqs if r[0] <= a.serve_seconds]
            pending, lat, qms, rejected, shed, decoded = {}, [], [], 0, 0, 0
            overlap_max, on_device = 0, []
            start = time.perf_counter()
            i = 0
            while i < len(reqs) or pending:
                now = time.perf_counter() - start
                while i < len(reqs) and reqs[i][0] <= now:
                    _, cols, rb, rc = reqs[i]
                    i += 1
                    if len(pending) >= a.serve_max_pending:
                        shed += 1  # open loop: the client sheds what the server cannot queue
                        continue
                    st, tk = N.pq_serve_submit(srv, cols, rb, rc)
                    if st == N.PQ_OK:
                        pending[tk] = i
                    else:
                        rejected += 1
                for tk in list(pending):
                    res = N.pq_serve_poll(srv, tk)
                    if res is None:
                        continue
                    if res.status == N.PQ_OK:
                        lat.append(res.latency_ms)
                        qms.append(res.queue_ms)
                        decoded += res.decoded_bytes
                        on_device.append((res.admit_ms, res.done_ms))
                    else:
                        rejected += 1
                    N.pq_serve_release(srv, tk)
                    del pending[tk]
                time.sleep(0.0002)
            wall = time.perf_counter() - start
            lat_sorted = sorted(lat)

            def pct(p):
                return lat_sorted[min(len(lat_sorted) - 1, int(np.ceil(p / 100 * len(lat_sorted))) - 1)] if lat_sorted else None
            # most requests on the device at once (admitted, not yet completed)
            ev = sorted([(t0, 1) for t0, _ in on_device] + [(t1, -1) for _, t1 in on_device])
            cur = 0
            for _, d in ev:
                cur += d
                overlap_max = max(overlap_max, cur)
            points.append({"offered_rps": rate, "achieved_rps": len(lat) / wall, "completed": len(lat),
                           "arrivals": len(reqs), "shed": shed, "max_on_device": overlap_max,
                           "refused_or_failed": rejected, "p50_ms": pct(50), "p99_ms": pct(99),
                           "mean_queue_ms": float(np.mean(qms)) if qms else None, "decoded_gbs": decoded / wall / 1e9,
                           "wall_s": wall})
    N.pq_serve_destroy(srv)
    N.pq_free_index(idx)
    eng.close()
    knee = max(points, key=lambda p: p["decoded_gbs"])
    line = {"metric": "p50/p99 served scan latency", "value": knee["p99_ms"], "unit": "ms",
            "n_gpus": 1, "steps": sum(p["completed"] for p in points), "warmup": 0, "ms_per_step": None,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": "serving: Poisson requests over %d eight-column tables of %d rows "
                                   "(%s), budget %.0f GiB, %d slots" % (
                                       len(files), a.rows, "; ".join(d for _, d in files), a.serve_budget_gib,
                                       a.serve_slots),
                       "rows_per_request": "log-uniform 2^20..2^28, wrapping", "columns_per_request": "1..8",
                       "arrivals": "Poisson, up to %d requests or %g s per load point; arrivals while %d requests "
                                   "are pending are shed and counted" % (a.serve_requests, a.serve_seconds,
                                                                         a.serve_max_pending),
                       "l2": "inputs larger than L2"},
            "serving": points, "clocks": clk.summary(),
            "detail": {"catalog_rows": info.num_rows, "write_seconds": gen_s,
                       "value_is": "p99 latency at the offered load with the highest decoded GB/s"}}
    print(json.dumps(line), flush=True)
    if a.json_out:
        with open(a.json_out, "w") as f:
            json.dump(line, f, indent=1)


# ----------------------------------------------------------------- batched (uneven chunks, one graph)

def _pack_files(datas, torch):
    """One device buffer holding every file at a 256-byte aligned offset."""
    offs, tot = [], 0
    for d in datas:
        offs.append(tot)
        tot += (d.nbytes + 255) // 256 * 256
    host = np.zeros(tot, np.uint8)
    for d, o in zip(datas, offs):
        host[o:o + d.nbytes] = d
    dev = torch.from_numpy(host).cuda()
    return dev, [(dev.data_ptr() + o, d.nbytes) for d, o in zip(datas, offs)]


def _time_batch(N, ctx, batch, stream, reps, torch):
    for _ in range(3):
        N.pq_batch_launch(ctx, batch, stream)
    assert N.pq_batch_wait(batch) == N.PQ_OK, N.pq_last_error(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        N.pq_batch_launch(ctx, batch, stream)
    e1.record()
    torch.cuda.synchronize()
    assert N.pq_batch_wait(batch) == N.PQ_OK, N.pq_last_error(ctx)
    return e0.elapsed_time(e1) / reps


def run_batched(a):
    import torch
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.autotune import autotune
    from paper_2602_17335_gb300.scan import Engine, alloc_outputs, stream_handle
    from paper_2602_17335_gb300.tables import write_table
    t0 = time.time()
    draws = synth.config4_draws(n_files=a.c4_files, chunks_per_file=a.c4_chunks_per_file, rows_lo=a.c4_rows_lo,
                                rows_hi=a.c4_rows_hi)
    groups = {}
    for d in draws:
        col, cspec = synth.config4_column(d)
        data = write_table(synth.Table([col]), synth.TableSpec(rg_rows=d.n_rows, page_bytes=d.page_bytes,
                                                               columns=[cspec]))
        groups.setdefault(d.kind, []).append(data)
    gen_s = time.time() - t0
    eng = Engine(0)
    sh = stream_handle(torch.cuda.current_stream())
    keep, idxs = [], []
    for kind, datas in groups.items():
        dev, files = _pack_files(datas, torch)
        keep.append(dev)
        idxs.append(N.pq_index_chunks(eng.ctx, files, sh))
    pages = sum(N.pq_index_get_info(ix).n_data_pages for ix in idxs)
    stored = sum(d.nbytes for ds in groups.values() for d in ds)

    def build(flags):
        plans, outs, dec, rd = [], [], 0, 0
        for ix in idxs:
            pl, sizes = N.pq_plan_scan(eng.ctx, ix, None, 0, -1, flags)
            info = N.pq_plan_get_info(pl)
            dec += info.decoded_bytes
            rd += info.read_bytes
            plans.append(pl)
            outs.append(alloc_outputs(sizes))
        return plans, outs, dec, rd

    def free(plans):
        for pl in plans:
            N.pq_free_plan(pl)

    def time_mode(flags, graph, reps):
        plans, outs, dec, rd = build(flags)
        b = N.pq_batch_create(eng.ctx, plans, [[o.desc() for o in oo] for oo in outs],
                              N.PQ_SCAN_GRAPH if graph else 0)
        ms = _time_batch(N, eng.ctx, b, sh, reps, torch)
        launches = sum(N.pq_plan_get_info(pl).launches_per_scan for pl in plans)
        N.pq_batch_free(b)
        free(plans)
        del outs
        return ms, dec, rd, launches

    tuned, trials = None, []
    if not a.no_autotune:
        tuned, _, trials = autotune(eng.ctx, lambda t: time_mode(N.PQ_SCAN_BATCHED, True, 3)[0])
    with ClockSampler(0) as clk:
        ms_graph, dec, rd, launches = time_mode(N.PQ_SCAN_BATCHED, True, a.steps)
    ms_stream, _, _, _ = time_mode(N.PQ_SCAN_BATCHED, False, a.steps)
    ms_plain, _, _, plain_launches = time_mode(N.PQ_SCAN_PLAIN, False, max(2, a.steps // 2))
    value = dec / (ms_graph * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    achieved = (rd + dec) / (ms_graph * 1e-3) / 1e9
    line = {"metric": "decoded GB/s", "value": value, "unit": "GB/s", "n_gpus": 1, "steps": a.steps,
            "warmup": 3, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "batched: %d single-column files, rows log-uniform [%g, %g], pages log-uniform "
                                   "4 KiB-2 MiB, kinds dict INT32 / dict string / PLAIN FP64 / DELTA INT64 / "
                                   "OPTIONAL PLAIN INT64, half Snappy, V1/V2 half each" % (
                                       len(draws), a.c4_rows_lo, a.c4_rows_hi),
                       "step": "one batch launch (all chunks' kernels in one CUDA graph)",
                       "l2": "inputs larger than L2 (%.2f GB stored, %.2f GB decoded)" % (stored / 1e9, dec / 1e9)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "one batch graph launch"},
            "compare": {"graph_ms": ms_graph, "streams_no_graph_ms": ms_stream, "plain_per_page_ms": ms_plain,
                        "plain_vs_graph": ms_plain / ms_graph, "graph_launches_inside": launches,
                        "plain_launches": plain_launches},
            "autotune": {"chosen": tuned, "trials": [{"tuning": t, "ms": m} for t, m in trials]},
            "gpu_launches": a.steps * launches, "clocks": clk.summary(),
            "detail": {"chunks": len(draws), "data_pages": pages, "decoded_bytes": dec, "read_bytes": rd,
                       "write_seconds": gen_s}}
    for ix in idxs:
        N.pq_free_index(ix)
    eng.close()
    print(json.dumps(line), flush=True)
    if a.json_out:
        with open(a.json_out, "w") as f:
            json.dump(line, f, indent=1)


def run_single(a):
    """One REQUIRED INT32 column, 2^20 rows uniform in [0, 1024), dictionary
    encoded (bit width 10), one row group, 1 MiB pages, uncompressed: the
    plain one-page-per-block decode against the batched scan."""
    import torch
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.scan import Engine, alloc_outputs, stream_handle
    from paper_2602_17335_gb300.tables import write_table
    tab = synth.config1_table()
    data = write_table(tab, synth.config1_spec())
    dev = torch.from_numpy(data).cuda()
    eng = Engine(0)
    sh = stream_handle(torch.cuda.current_stream())
    idx = eng.index([dev])
    res = {}
    with ClockSampler(0) as clk:
        for name, flags in (("plain", N.PQ_SCAN_PLAIN), ("batched", N.PQ_SCAN_BATCHED | N.PQ_SCAN_GRAPH)):
            pl, sizes = eng.plan(idx, flags=flags)
            info = N.pq_plan_get_info(pl)
            outs = alloc_outputs(sizes)
            for _ in range(3):
                eng.scan(pl, outs, torch.cuda.current_stream())
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(a.steps):
                eng.scan(pl, outs, torch.cuda.current_stream())
            e1.record()
            torch.cuda.synchronize()
            st, _ = eng.wait(pl, len(outs))
            assert st == N.PQ_OK, N.pq_last_error(eng.ctx)
            ms = e0.elapsed_time(e1) / a.steps
            res[name] = {"ms": ms, "decoded_gbs": info.decoded_bytes / (ms * 1e-3) / 1e9,
                         "launches_per_scan": info.launches_per_scan, "pages": info.n_pages}
            N.pq_free_plan(pl)
    N.pq_free_index(idx)
    eng.close()
    line = {"metric": "decoded GB/s", "value": res["batched"]["decoded_gbs"], "unit": "GB/s", "n_gpus": 1,
            "steps": a.steps, "warmup": 3, "ms_per_step": res["batched"]["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "one dictionary INT32 column, 2^20 rows U[0,1024), bit width 10, one row group, "
                                   "1 MiB pages, uncompressed", "step": "one scan launch",
                       "l2": "inputs smaller than L2 (4 MiB out); scan replayed back to back"},
            "compare": res, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    if a.json_out:
        with open(a.json_out, "w") as f:
            json.dump(line, f, indent=1)


def main():
    a = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if a.impl == "reference":
            if rank != 0:
                return
        else:
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if a.workload in ("serve", "batched", "single"):
        if rank == 0:
            {"serve": run_serve, "batched": run_batched, "single": run_single}[a.workload](a)
        return
    run_ours(a, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
