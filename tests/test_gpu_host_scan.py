"""pq_scan_host (files in host memory, columns back in host memory) against
the oracle, bit for bit: the row-group pipeline (several row groups whose
output rows start on 32-row boundaries), the whole-file path (a row range
whose row groups do not), and both paths on the same request."""
import os

import numpy as np
import pytest

import synth
from oracle import reader as R
from oracle import writer as W

from gpu_util import slice_result

pytestmark = pytest.mark.gpu

SMALL = dict(string_pool_size=700, zipf_k=2000)


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2602_17335_gb300 import native as N
    c = N.pq_ctx_create(0)
    yield c
    N.pq_ctx_destroy(c)


def _zeros(n, pinned):
    """n zero bytes: a numpy array, or a numpy view of pinned host memory
    (which the scan writes back by a copy kernel rather than by copies)."""
    if not pinned:
        return np.zeros(n, np.uint8)
    import torch
    return torch.zeros(max(n, 1), dtype=torch.uint8).pin_memory().numpy()[:n]


def _host_scan(N, ctx, datas, columns, rb, rc, pinned=False):
    import ctypes as C
    bufs = [np.frombuffer(bytes(d), dtype=np.uint8).copy() for d in datas]
    files = [(b.ctypes.data, b.nbytes) for b in bufs]
    sizes = N.pq_scan_host(ctx, files, columns, rb, rc)
    n = len(columns)
    outs, keep = [], []
    for i in range(n):
        s = sizes[i]
        c = N.pq_column()
        v = _zeros(int(s.values_bytes), pinned)
        keep.append(v)
        c.values = v.ctypes.data
        m = None
        if s.validity_bytes:
            m = _zeros(int(s.validity_bytes), pinned)
            keep.append(m)
            c.validity = m.ctypes.data
        ch = None
        if s.chars_bytes:
            ch = _zeros(int(s.chars_bytes), pinned)
            keep.append(ch)
            c.chars = ch.ctypes.data
            c.chars_capacity = int(s.chars_bytes)
        outs.append(c)
    N.pq_scan_host(ctx, files, columns, rb, rc, outs=outs)
    return sizes, keep, outs


def _check(sizes, keep, expect_cols, columns):
    from gpu_util import bitmap_words
    k = 0
    for i, e in enumerate(expect_cols):
        s = sizes[i]
        v = keep[k]
        k += 1
        m = None
        if s.validity_bytes:
            m = keep[k]
            k += 1
        ch = None
        if s.chars_bytes:
            ch = keep[k]
            k += 1
        if e.ptype == "BYTE_ARRAY":
            offs = v.view(np.int64)
            assert np.array_equal(offs, e.offsets), f"{e.name}: offsets differ"
            assert np.array_equal(ch[:int(offs[-1])], e.chars), f"{e.name}: chars differ"
        else:
            assert np.array_equal(v.view(e.values.dtype), e.values), f"{e.name}: values differ"
        if e.valid is not None:
            words = bitmap_words(e.valid)
            assert np.array_equal(m[:len(words)], words), f"{e.name}: validity differs"


@pytest.mark.parametrize("rb,rc", [(0, -1), (8192, 24576), (100, 30_001), (32, 30_000)])
@pytest.mark.parametrize("pipeline,pinned", [(True, False), (False, False), (True, True)])
def test_host_scan_matches_oracle(ctx, rb, rc, pipeline, pinned, monkeypatch):
    """(32, 30000): the pipeline with a partial first and last row group
    (their string chars are waited for; the whole ones are planned exactly);
    (100, 30001): row groups off the 32-row grid, the whole-file path."""
    from paper_2602_17335_gb300 import native as N
    if not pipeline:
        monkeypatch.setenv("PQ_HOST_NO_PIPELINE", "1")
    tab = synth.config2_table(40_000, 8192, **SMALL)
    data = W.write_file(tab, synth.config2_spec(8192, 16 * 1024, "SNAPPY", 2))
    expect = R.read_file(data)
    columns = list(range(8))
    sizes, keep, _ = _host_scan(N, ctx, [data], columns, rb, rc, pinned)
    hi = 40_000 if rc < 0 else rb + rc
    _check(sizes, keep, [slice_result(expect[c], rb, hi) for c in columns], columns)


@pytest.mark.parametrize("offset_index", [True, False])
def test_host_scan_pipeline_offset_index(ctx, offset_index):
    """The pipeline walks each row group's page headers on the host, with or
    without OffsetIndex structures in the file (which it does not read);
    both give the oracle's columns."""
    from paper_2602_17335_gb300 import native as N
    tab = synth.config2_table(30_000, 4096, **SMALL)
    data = W.write_file(tab, synth.config2_spec(4096, 8 * 1024, "UNCOMPRESSED", 1, offset_index=offset_index))
    expect = R.read_file(data)
    columns = [0, 1, 5, 6]
    sizes, keep, _ = _host_scan(N, ctx, [data], columns, 0, -1)
    _check(sizes, keep, [expect[c] for c in columns], columns)
