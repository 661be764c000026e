"""Serving loop (pq_serve_*) through the C ABI: requests of different sizes
over an indexed table, row ranges that wrap around the table, results
compared bit for bit with the oracle, each request alone and in a mix of
concurrent requests (continuous batching); budget refusal and release."""
import time

import numpy as np
import pytest

import synth
from oracle import reader as R
from oracle import writer as W

from gpu_util import assert_columns_equal, engine, server_result_outs, slice_result, to_dev

pytestmark = pytest.mark.gpu

SMALL = dict(string_pool_size=700, zipf_k=2000)
N_ROWS = 30_000


@pytest.fixture(scope="module")
def setup():
    e = engine()
    tab = synth.config2_table(N_ROWS, 10_000, **SMALL)
    data = W.write_file(tab, synth.config2_spec(10_000, 8192))
    expect = R.read_file(data)
    dev = to_dev(data)
    idx = e.index([dev])
    yield e, idx, expect
    from paper_2602_17335_gb300 import native as N
    N.pq_free_index(idx)
    e.close()


def _expected(expect, cols, rb, rc):
    """Rows (rb + i) mod N, i < rc: slices of the oracle's columns joined."""
    from oracle.reader import ColumnResult
    out = []
    for c in cols:
        parts, r, left = [], rb % N_ROWS, rc
        while left > 0:
            take = min(N_ROWS - r, left)
            parts.append(slice_result(expect[c], r, r + take))
            left -= take
            r = 0
        p0 = parts[0]
        valid = None if p0.valid is None else np.concatenate([p.valid for p in parts])
        if p0.ptype == "BYTE_ARRAY":
            offs, base = [np.zeros(1, np.int64)], 0
            for p in parts:
                offs.append(p.offsets[1:] + base)
                base += int(p.offsets[-1])
            out.append(ColumnResult(p0.name, p0.ptype, None, valid, np.concatenate(offs),
                                    np.concatenate([p.chars for p in parts])))
        else:
            out.append(ColumnResult(p0.name, p0.ptype, np.concatenate([p.values for p in parts]), valid))
    return out


REQUESTS = [
    (list(range(8)), 0, N_ROWS),          # whole table
    ([5], 12_345, 50_000),                # strings, wraps once
    ([4, 2], 29_000, 3_000),              # OPTIONAL + PLAIN across the end
    ([1], 7, 1),                          # one DELTA row
    ([6, 7, 0], 100, 65_000),             # wraps twice
    ([3, 5, 4], 9_999, 10_002),           # across row-group boundaries
]


def _wait(N, srv, ticket, timeout=60.0):
    t0 = time.time()
    while True:
        res = N.pq_serve_poll(srv, ticket)
        if res is not None:
            return res
        assert time.time() - t0 < timeout, "serving request did not finish"
        time.sleep(0.0005)


def test_serving_alone_and_in_mix(setup):
    from paper_2602_17335_gb300 import native as N
    e, idx, expect = setup
    srv = N.pq_serve_create(e.ctx, idx, budget_bytes=1 << 30, slots=3)
    try:
        # alone: one request at a time
        for cols, rb, rc in REQUESTS:
            st, t = N.pq_serve_submit(srv, cols, rb, rc)
            assert st == N.PQ_OK
            res = _wait(N, srv, t)
            assert res.status == N.PQ_OK
            assert_columns_equal(server_result_outs(res), _expected(expect, cols, rb, rc))
            assert res.latency_ms >= res.queue_ms >= 0
            assert N.pq_serve_release(srv, t) == N.PQ_OK
        # in the mix: all submitted at once, three slots, results identical
        tickets = []
        for cols, rb, rc in REQUESTS * 3:
            st, t = N.pq_serve_submit(srv, cols, rb, rc)
            assert st == N.PQ_OK
            tickets.append((t, cols, rb, rc))
        spans = []
        for t, cols, rb, rc in tickets:
            res = _wait(N, srv, t)
            assert res.status == N.PQ_OK
            assert_columns_equal(server_result_outs(res), _expected(expect, cols, rb, rc))
            assert res.done_ms >= res.admit_ms >= 0
            spans.append((res.admit_ms, res.done_ms))
            assert N.pq_serve_release(srv, t) == N.PQ_OK
        # continuous batching: some request was admitted while another was
        # still on the device (their device intervals overlap)
        overlapping = sum(1 for i, (a0, d0) in enumerate(spans) for (a1, d1) in spans[i + 1:]
                          if a0 < d1 and a1 < d0)
        assert overlapping > 0, spans
    finally:
        N.pq_serve_destroy(srv)


def _one_request_budget(N, e, idx, cols, rb, rc):
    """The smallest power of two (bytes) that admits the request alone: at
    least its device bytes and less than twice them."""
    b = 1 << 16
    while True:
        srv = N.pq_serve_create(e.ctx, idx, budget_bytes=b, slots=1)
        try:
            st, t = N.pq_serve_submit(srv, cols, rb, rc)
            if st == N.PQ_OK:
                assert _wait(N, srv, t).status == N.PQ_OK
                N.pq_serve_release(srv, t)
                return b
            assert st == N.PQ_ERR_BUDGET
        finally:
            N.pq_serve_destroy(srv)
        b *= 2


def test_serving_budget(setup):
    """A request larger than the whole budget is refused at submit; requests
    that fit about one at a time still all finish (admission waits for
    released outputs)."""
    from paper_2602_17335_gb300 import native as N
    e, idx, expect = setup
    one = _one_request_budget(N, e, idx, [2, 4], 0, 20_000)
    srv = N.pq_serve_create(e.ctx, idx, budget_bytes=one + one // 4, slots=4)
    try:
        st, _ = N.pq_serve_submit(srv, list(range(8)), 0, 40 * N_ROWS)
        assert st == N.PQ_ERR_BUDGET
        tickets = []
        for k in range(6):
            st, t = N.pq_serve_submit(srv, [2, 4], 1000 * k, 20_000)
            assert st == N.PQ_OK
            tickets.append((t, 1000 * k))
        for t, rb in tickets:
            res = _wait(N, srv, t)
            assert res.status == N.PQ_OK
            assert_columns_equal(server_result_outs(res), _expected(expect, [2, 4], rb, 20_000))
            assert N.pq_serve_release(srv, t) == N.PQ_OK
    finally:
        N.pq_serve_destroy(srv)


def test_serving_queue_timeout(setup):
    """With the budget held by an unreleased result, a queued request ages
    past its timeout and fails with PQ_ERR_TIMEOUT; the server keeps working."""
    from paper_2602_17335_gb300 import native as N
    e, idx, expect = setup
    one = _one_request_budget(N, e, idx, [2], 0, 20_000)  # admits one such request, not two
    srv = N.pq_serve_create(e.ctx, idx, budget_bytes=one, slots=2, timeout_ms=50)
    try:
        st, t1 = N.pq_serve_submit(srv, [2], 0, 20_000)
        assert st == N.PQ_OK
        r1 = _wait(N, srv, t1)
        assert r1.status == N.PQ_OK
        st, t2 = N.pq_serve_submit(srv, [2], 0, 20_000)  # cannot fit until t1 is released
        assert st == N.PQ_OK
        r2 = _wait(N, srv, t2)
        assert r2.status == N.PQ_ERR_TIMEOUT
        assert N.pq_serve_release(srv, t2) == N.PQ_OK
        assert N.pq_serve_release(srv, t1) == N.PQ_OK
        st, t3 = N.pq_serve_submit(srv, [2], 0, 20_000)
        r3 = _wait(N, srv, t3)
        assert r3.status == N.PQ_OK
        assert_columns_equal(server_result_outs(r3), _expected(expect, [2], 0, 20_000))
        N.pq_serve_release(srv, t3)
    finally:
        N.pq_serve_destroy(srv)
