"""pq_delta_decode_static (allocation-free DELTA stream decode) through the
C ABI, bit for bit against the CPU oracle's decoding of the same stream
bytes (oracle.delta.decode) and against the DELTA path of pq_scan_columns.

The file is named to be collected last: it must pass alone in a fresh
process and after every other GPU test.  Each stream is decoded twice in a
row into two buffers; both must equal the oracle's values and the scan's
column."""
import numpy as np
import pytest

import synth
from oracle import delta as D
from oracle import reader as R
from oracle import writer as W

from gpu_util import engine, to_dev

pytestmark = pytest.mark.gpu

DATA_PAGE = 0
DELTA_BINARY_PACKED = 5


@pytest.fixture(scope="module")
def eng():
    e = engine()
    yield e
    e.close()


def _value_streams(data):
    """(column, stream bytes, value count) of each DELTA data page; with a
    REQUIRED column, V1 pages and no codec the page body is the stream."""
    out = []
    for ch in R.parse_footer(data).chunks:
        for p in R.chunk_pages(data, ch):
            if p.page_type == DATA_PAGE and p.encoding == DELTA_BINARY_PACKED:
                b = p.offset + p.header_len
                out.append((ch.column, bytes(data[b:b + p.compressed]), p.num_values))
    return out


def _padded(stream):
    import torch
    t = torch.zeros(len(stream) + 32, dtype=torch.uint8, device="cuda")
    t[:len(stream)] = torch.frombuffer(bytearray(stream), dtype=torch.uint8).cuda()
    return t


def _decode_twice_and_compare(eng, cols):
    import torch
    from paper_2602_17335_gb300 import native as N
    n = len(cols[0].values)
    spec = synth.TableSpec(n, 64 << 20, [synth.ColumnSpec("DELTA_BINARY_PACKED") for _ in cols])
    data = W.write_file(synth.Table(cols), spec)
    scanned = eng.read([to_dev(data)])
    streams = _value_streams(data)
    assert len(streams) == len(cols)  # one page per column
    for col, stream, nv in streams:
        ref = scanned[col].values
        assert nv == ref.numel()
        ptype = N.PQ_TYPE_INT32 if ref.dtype == torch.int32 else N.PQ_TYPE_INT64
        s = _padded(stream)
        got = [torch.full_like(ref, -7) for _ in range(2)]
        for g in got:
            st = N.pq_delta_decode_static(eng.ctx, s.data_ptr(), len(stream), ptype, nv, g.data_ptr())
            assert st == N.PQ_OK, N.pq_last_error(eng.ctx)
        bits = 32 if ptype == N.PQ_TYPE_INT32 else 64
        vals, end = D.decode(stream, 0, len(stream), bits)
        assert len(vals) == nv and end <= len(stream)
        expect = np.array(vals, dtype=np.int32 if bits == 32 else np.int64)
        for g in got:
            assert np.array_equal(g.cpu().numpy(), expect), f"column {col}: static decode differs from the oracle"
            assert torch.equal(g, ref), f"column {col}: static decode differs from the scan"


def test_static_decode_matches_scan_many_regions(eng):
    """Long streams: the block chain spans many 8 KB regions."""
    rng = np.random.default_rng(11)
    n = 1_000_001
    i64 = np.iinfo(np.int64)
    cols = [
        synth.ColumnData("steps", "INT64", np.cumsum(rng.integers(0, 8, n)).astype(np.int64)),
        synth.ColumnData("mixed32", "INT32", np.cumsum(np.where((np.arange(n) // 4096) % 2 == 0, 1,
                                                                rng.integers(-1000, 1000, n))).astype(np.int32)),
        synth.ColumnData("const", "INT64", np.full(n, -5, np.int64)),
    ]
    _decode_twice_and_compare(eng, cols)
    m = 8000
    _decode_twice_and_compare(eng, [synth.ColumnData("rand64", "INT64",
                                                     rng.integers(i64.min, i64.max, m, dtype=np.int64,
                                                                  endpoint=True))])


@pytest.mark.parametrize("n", [1, 2, 129, 130, 4097])
def test_static_decode_matches_scan_small(eng, n):
    rng = np.random.default_rng(n)
    _decode_twice_and_compare(eng, [synth.ColumnData("v", "INT32", rng.integers(-50, 50, n).astype(np.int32))])


def test_static_decode_rejections(eng):
    """Over the limits: refused on the host before any launch.  A value count
    that disagrees with the stream header: refused by the device check."""
    import torch
    from paper_2602_17335_gb300 import native as N
    n = 1000
    vals = np.arange(n, dtype=np.int64) * 3
    data = W.write_file(synth.Table([synth.ColumnData("v", "INT64", vals)]),
                        synth.TableSpec(n, 1 << 20, [synth.ColumnSpec("DELTA_BINARY_PACKED")]))
    (_, stream, nv), = _value_streams(data)
    s = _padded(stream)
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    assert N.pq_delta_decode_static(eng.ctx, s.data_ptr(), (1 << 20) + 1, N.PQ_TYPE_INT64, nv,
                                    out.data_ptr()) == N.PQ_ERR_CAPACITY
    assert N.pq_delta_decode_static(eng.ctx, s.data_ptr(), len(stream), N.PQ_TYPE_INT64, 4194306,
                                    out.data_ptr()) == N.PQ_ERR_CAPACITY
    assert N.pq_delta_decode_static(eng.ctx, s.data_ptr(), len(stream), N.PQ_TYPE_DOUBLE, nv,
                                    out.data_ptr()) == N.PQ_ERR_INVALID_ARG
    assert N.pq_delta_decode_static(eng.ctx, s.data_ptr(), len(stream), N.PQ_TYPE_INT64, nv - 1,
                                    out.data_ptr()) == N.PQ_ERR_CORRUPT
    # still usable afterwards
    assert N.pq_delta_decode_static(eng.ctx, s.data_ptr(), len(stream), N.PQ_TYPE_INT64, nv,
                                    out.data_ptr()) == N.PQ_OK
    assert np.array_equal(out.cpu().numpy(), vals)
