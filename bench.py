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
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rows", type=int, default=1 << 26)
    ap.add_argument("--rg-rows", type=int, default=1 << 23)
    ap.add_argument("--page-bytes", type=int, default=MiB)
    ap.add_argument("--codec", default="UNCOMPRESSED", choices=["UNCOMPRESSED", "SNAPPY"])
    ap.add_argument("--page-version", type=int, default=1)
    ap.add_argument("--mode", default="batched", choices=["batched", "plain"])
    ap.add_argument("--no-offset-index", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scan-reps", type=int, default=10, help="graph replays for the roofline")
    ap.add_argument("--json-out", default=None)
    return ap.parse_args()


def workload_name(a):
    return (f"eight-column table, {a.rows} rows, row groups of {a.rg_rows} rows, "
            f"{a.page_bytes // 1024} KiB pages, {a.codec.lower()}, V{a.page_version} pages")


def make_files(a, rank):
    """The table of this rank, written by the engine's native writer."""
    from paper_2602_17335_gb300.tables import write_table
    tab = synth.config2_table(a.rows, a.rg_rows, file=rank)
    spec = synth.config2_spec(a.rg_rows, a.page_bytes, a.codec, a.page_version, offset_index=not a.no_offset_index)
    data = write_table(tab, spec)
    return data


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


# ----------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = open(os.path.join(ROOT, "gpurun_out", "clocks.csv") if os.path.isdir(os.path.join(ROOT, "gpurun_out"))
                            else os.devnull, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.lines = []
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            if self.out:
                self.out.write(line)

    def __exit__(self, *exc):
        if self.proc:
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
                "samples": len(sm)}


# ----------------------------------------------------------------- arms

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
    data = make_files(a, 0)
    for _ in range(a.warmup):
        oracle_sample(data, max_seconds=5.0)
    tot_b, tot_s = 0.0, 0.0
    desc = ""
    for _ in range(a.steps):
        b, s, desc = oracle_sample(data, max_seconds=20.0)
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

    def step():
        ix = N.pq_index_chunks(eng.ctx, [(t.data_ptr(), t.numel()) for t in files], sh)
        pl, _ = N.pq_plan_scan(eng.ctx, ix, None, 0, -1, base_flags)
        N.pq_scan_columns(eng.ctx, pl, [o.desc() for o in outs], sh)
        st, _ = N.pq_scan_wait(eng.ctx, pl, len(outs), sh)
        N.pq_free_plan(pl)
        N.pq_free_index(ix)
        if st != N.PQ_OK:
            raise N.PqError(st, N.pq_last_error(eng.ctx))

    for _ in range(max(a.warmup, 1)):
        step()
    torch.cuda.synchronize(dev)
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
    step_ms = start.elapsed_time(end) / a.steps
    if world > 1:
        t = torch.tensor([step_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        step_ms = float(t.item())
    decoded = float(pinfo.decoded_bytes)
    read = float(pinfo.read_bytes)
    value = world * decoded / (step_ms * 1e-3) / 1e9

    # roofline: one scan launch = all stages of pq_scan_columns, replayed from a graph
    idx = eng.index(files)
    plan, _ = eng.plan(idx, flags=base_flags | (0 if a.mode == "plain" else N.PQ_SCAN_GRAPH))
    for _ in range(3):
        eng.scan(plan, outs, stream)
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
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_kind": peak_kind,
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
        N.pq_scan_host(eng.ctx, hfiles, outs=houts)
        reps = max(2, min(a.steps, 5))
        t0 = time.perf_counter()
        for _ in range(reps):
            N.pq_scan_host(eng.ctx, hfiles, outs=houts)
        e2e_s = (time.perf_counter() - t0) / reps
        d2h = int(sum(s.values_bytes + s.validity_bytes for s in sizes) + sum(
            int(s.chars_bytes) for s in sizes))
        e2e = {"value": world * decoded / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": int(data.nbytes),
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3}
        del keep

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        b, s, desc = oracle_sample(data, max_seconds=25.0)
        cpu = {"value": b / s / 1e9, "unit": "GB/s", "cores": cpu_count_used(), "kind": "oracle", "sample": desc,
               "seconds": s}

    line = {"metric": "decoded GB/s", "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": workload_name(a), "rows": a.rows, "rg_rows": a.rg_rows,
                       "page_bytes": a.page_bytes, "codec": a.codec, "page_version": a.page_version,
                       "mode": a.mode, "offset_index": not a.no_offset_index,
                       "l2": "inputs larger than L2 (files %.2f GB, outputs %.2f GB per step)" % (
                           data.nbytes / 1e9, decoded / 1e9),
                       "step": "index + plan + scan + wait"},
            "roofline": roofline, "stages_ms": stages, "cpu_baseline": cpu, "e2e": e2e,
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
    run_ours(a, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
