"""GPU scan vs CPU oracle at the benchmark's full sizes, bit for bit.

* The eight-column table of 2^26 rows in row groups of 2^23 rows with 1 MiB
  pages, uncompressed, V1 pages with an OffsetIndex, written by the engine's
  writer exactly as the benchmark writes it, scanned in the launch
  configuration the benchmark times (index + plan + batched scan + wait).
  Every one of its 64 chunks is decoded by the oracle (a spawn-started
  process pool over chunks) and compared element by element: this covers
  column 1's dictionaries of about 2^20 entries at bit width 20, the string
  chunks of about 170 MB of chars each, and every page and work item.  The
  graph-replayed scan (the roofline measurement) and the plain one-page-per-
  block scan must give the same bytes.
* The single dictionary column of 2^20 rows (values in [0, 1024), bit width
  10, 1 MiB pages), plain per-page scan and batched scan.

The 2^26-row check holds about 15 GB of device memory; it runs in a process
of its own (a fresh CUDA context, like the benchmark's), so that the memory
it leaves behind in the allocators cannot change what later tests see.
"""
import multiprocessing as mp
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from oracle import reader as R
from oracle import writer as W

from gpu_util import assert_columns_equal, bitmap_words, engine, to_dev
from oracle_chunks import cut_chunk, expected_chunk

pytestmark = pytest.mark.gpu

ROWS = 1 << 26
RG_ROWS = 1 << 23
PAGE = 1 << 20


@pytest.fixture(scope="module")
def eng():
    e = engine()
    yield e
    e.close()


def _host(t):
    return t.cpu().numpy()


def test_bench_table_every_chunk():
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([root, here, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-c", "import test_gpu_full_size as t; t.bench_table_every_chunk()"],
                       cwd=here, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, (r.stdout[-4000:] + r.stderr[-4000:])
    assert "every chunk equal" in r.stdout


def bench_table_every_chunk():
    """The 2^26-row check (run in a child process, see the module docstring)."""
    import torch
    workers = max(2, min(16, os.cpu_count() or 2))
    pool = mp.get_context("spawn").Pool(workers)
    eng = engine()
    try:
        _bench_table_every_chunk(pool, eng)
    finally:
        pool.terminate()
        pool.join()
        eng.close()
    print("every chunk equal")


def _bench_table_every_chunk(pool, eng):
    import torch
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.scan import alloc_outputs, stream_handle
    from paper_2602_17335_gb300.tables import write_table

    tab = synth.config2_table(ROWS, RG_ROWS)
    data = write_table(tab, synth.config2_spec(RG_ROWS, PAGE, "UNCOMPRESSED", 1, offset_index=True))
    del tab
    info = R.parse_footer(data.tobytes())
    assert len(info.chunks) == 64 and info.num_rows == ROWS
    # the oracle starts on every chunk while the GPU scans
    pending = pool.imap_unordered(expected_chunk, (cut_chunk(data, ch) for ch in info.chunks), chunksize=1)

    dev = torch.from_numpy(data).to("cuda")
    sh = stream_handle()
    idx = N.pq_index_chunks(eng.ctx, [(dev.data_ptr(), dev.numel())], sh)
    plan, sizes = N.pq_plan_scan(eng.ctx, idx, None, 0, -1, N.PQ_SCAN_BATCHED)
    outs = alloc_outputs(sizes)
    N.pq_scan_columns(eng.ctx, plan, [o.desc() for o in outs], sh)
    st, chars = N.pq_scan_wait(eng.ctx, plan, len(outs), sh)
    assert st == N.PQ_OK, N.pq_last_error(eng.ctx)
    N.pq_free_plan(plan)
    assert [int(s.n_rows) for s in sizes] == [ROWS] * 8

    # the other two launch configurations, same bytes on the device
    for flags in (N.PQ_SCAN_BATCHED | N.PQ_SCAN_GRAPH, N.PQ_SCAN_PLAIN):
        pl, _ = N.pq_plan_scan(eng.ctx, idx, None, 0, -1, flags)
        other = alloc_outputs(sizes)
        for _ in range(2 if flags & N.PQ_SCAN_GRAPH else 1):
            N.pq_scan_columns(eng.ctx, pl, [o.desc() for o in other], sh)
            st2, chars2 = N.pq_scan_wait(eng.ctx, pl, len(other), sh)
            assert st2 == N.PQ_OK, N.pq_last_error(eng.ctx)
        assert list(chars2) == list(chars)
        for o, q, c in zip(outs, other, chars):
            assert torch.equal(o.values, q.values)
            if o.validity is not None:
                assert torch.equal(o.validity, q.validity)
            if o.chars is not None:
                assert torch.equal(o.chars[:c], q.chars[:c])
        N.pq_free_plan(pl)
        del other
    N.pq_free_index(idx)

    host = []
    for o, c in zip(outs, chars):
        host.append((_host(o.values), None if o.chars is None else _host(o.chars[:c]),
                     None if o.validity is None else _host(o.validity).view(np.uint8)))
    del outs, dev
    torch.cuda.empty_cache()

    seen = set()
    for rg, col, vals, ch_chars, valid in pending:
        lo, hi = rg * RG_ROWS, (rg + 1) * RG_ROWS
        got_vals, got_chars, got_valid = host[col]
        name = f"row group {rg}, column {col + 1}"
        if ch_chars is not None:
            off = got_vals[lo:hi + 1] - got_vals[lo]
            assert np.array_equal(off, vals), f"{name}: offsets differ"
            assert np.array_equal(got_chars[got_vals[lo]:got_vals[hi]], ch_chars), f"{name}: chars differ"
        else:
            g = got_vals[lo:hi]
            assert g.dtype.itemsize == vals.dtype.itemsize
            if not np.array_equal(g.view(np.uint8), vals.view(np.uint8)):
                bad = np.nonzero(g.view(np.uint8).reshape(len(g), -1) != vals.view(np.uint8).reshape(len(g), -1))[0]
                raise AssertionError(f"{name}: values differ, first rows {np.unique(bad)[:10] + lo}")
        if valid is None:
            assert got_valid is None
        else:
            words = bitmap_words(valid)
            assert np.array_equal(got_valid[lo // 8: lo // 8 + len(words)], words), f"{name}: validity differs"
        seen.add((rg, col))
    assert len(seen) == 64


def test_single_dictionary_column_full_size(eng):
    from paper_2602_17335_gb300 import native as N
    n = 1 << 20
    tab = synth.config1_table(n)
    data = W.write_file(tab, synth.config1_spec(PAGE, n))
    expect = R.read_file(data)
    dev = to_dev(data)
    for flags in (N.PQ_SCAN_PLAIN, N.PQ_SCAN_BATCHED):
        outs = eng.read([dev], flags=flags)
        assert_columns_equal(outs, expect)
