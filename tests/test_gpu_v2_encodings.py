"""GPU scan of the V2 encodings BYTE_STREAM_SPLIT, DELTA_LENGTH_BYTE_ARRAY
and DELTA_BYTE_ARRAY (the paper's Section 3, Insight 3) vs the CPU oracle,
bit for bit, through the C ABI.

The pages are rewritten into PLAIN bodies on the device before the walk;
the cases cover V1 and V2 pages, Snappy, nulls, pages cut small enough to
hold a handful of values, prefix chains longer than one 256-value batch,
row ranges, the three scan modes, and corrupt pages (an error status, the
same pages the oracle rejects)."""
import numpy as np
import pytest

import synth
from oracle import delta as D
from oracle import delta_strings as DS
from oracle import reader as R
from oracle import writer as W

from gpu_util import assert_columns_equal, engine, slice_result, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    e = engine()
    yield e
    e.close()


def _roundtrip(eng, data, **kw):
    expect = R.read_file(data)
    outs = eng.read([to_dev(data)], **kw)
    cols = kw.get("columns")
    rb = kw.get("row_begin", 0)
    rc = kw.get("row_count", -1)
    e0 = expect[0]
    rows = len(e0.values) if e0.values is not None else len(e0.offsets) - 1
    hi = rows if rc < 0 else rb + rc
    exp = [slice_result(expect[c], rb, hi) for c in (cols if cols is not None else range(len(expect)))]
    assert_columns_equal(outs, exp)


@pytest.mark.parametrize("rg_rows,page_bytes", [(20_000, 1 << 20), (7000, 700)])
@pytest.mark.parametrize("codec,version", [("UNCOMPRESSED", 1), ("UNCOMPRESSED", 2), ("SNAPPY", 1),
                                           ("SNAPPY", 2)])
def test_v2_encodings_table(eng, rg_rows, page_bytes, codec, version):
    tab = synth.v2_encodings_table(20_000, rg_rows)
    _roundtrip(eng, W.write_file(tab, synth.v2_encodings_spec(rg_rows, page_bytes, codec, version)))


@pytest.mark.parametrize("rb,rc,cols", [(0, 1, None), (8191, 2, [0, 4, 5]), (12345, 9000, [3, 4]),
                                        (29_999, 1, [5, 2]), (4000, 0, [4])])
def test_v2_encodings_row_ranges(eng, rb, rc, cols):
    tab = synth.v2_encodings_table(30_000, 11_000)
    data = W.write_file(tab, synth.v2_encodings_spec(11_000, 8192, "SNAPPY", 1))
    _roundtrip(eng, data, columns=cols, row_begin=rb, row_count=rc)


@pytest.mark.parametrize("mode", ["plain", "graph", "timing"])
def test_v2_encodings_scan_modes(eng, mode):
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.scan import alloc_outputs
    tab = synth.v2_encodings_table(20_000, 8000)
    data = W.write_file(tab, synth.v2_encodings_spec(8000, 16 * 1024, "SNAPPY", 2))
    expect = R.read_file(data)
    flags = {"plain": N.PQ_SCAN_PLAIN, "graph": N.PQ_SCAN_GRAPH, "timing": N.PQ_SCAN_TIMING}[mode]
    idx = eng.index([to_dev(data)])
    plan, sizes = eng.plan(idx, flags=flags)
    for _ in range(3):  # replays rewrite the same plan pages
        outs = alloc_outputs(sizes)
        eng.scan(plan, outs)
        st, chars = eng.wait(plan, len(outs))
        assert st == N.PQ_OK, N.pq_last_error(eng.ctx)
        for o, c in zip(outs, chars):
            if o.chars is not None:
                o.chars = o.chars[:c]
        assert_columns_equal(outs, expect)
    N.pq_free_plan(plan)
    N.pq_free_index(idx)


def _string_column(name, rows, valid=None):
    lens = np.array([len(x) for x in rows], dtype=np.int64)
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    chars = np.frombuffer(b"".join(rows), dtype=np.uint8).copy()
    return synth.ColumnData(name, "BYTE_ARRAY",
                            synth.StringData(off, chars, np.arange(len(rows), dtype=np.int32)), valid)


def test_delta_byte_array_prefix_chains(eng):
    """Front-coded pages whose prefixes reach back across batches: one long
    stem shared by every row, identical rows (prefix = whole value), rows
    that grow one byte at a time, empty rows, strings of 0-500 bytes, and
    nulls in between."""
    rng = np.random.default_rng(5)
    n = 6000
    stem = bytes(rng.integers(97, 123, size=600, dtype=np.uint8))
    shared = sorted(stem[:int(rng.integers(0, 601))] + bytes(rng.integers(65, 70, size=int(rng.integers(0, 6)),
                                                                           dtype=np.uint8)) for _ in range(n))
    same = [b"identical-row-" * 3] * n
    grow = [b"g" * (i % 500) for i in range(n)]
    empty = [b"" if i % 3 else b"x%d" % i for i in range(n)]
    cols = [_string_column("shared", shared), _string_column("same", same), _string_column("grow", grow),
            _string_column("empty", empty), _string_column("shared_opt", shared, rng.random(n) > 0.4)]
    tab = synth.Table(cols)
    for enc in ("DELTA_BYTE_ARRAY", "DELTA_LENGTH_BYTE_ARRAY"):
        for rg, page, version in ((n, 1 << 20, 1), (2500, 2048, 2), (n, 64, 1)):
            spec = synth.TableSpec(rg, page, [synth.ColumnSpec(enc, page_version=version) for _ in cols])
            _roundtrip(eng, W.write_file(tab, spec))


def test_byte_stream_split_types_and_nulls(eng):
    """BYTE_STREAM_SPLIT over INT32, INT64 and DOUBLE, REQUIRED (copy path)
    and OPTIONAL (walk path), all-null and all-valid pages, one-row pages."""
    rng = np.random.default_rng(8)
    n = 20_011
    cols = [
        synth.ColumnData("i32", "INT32", rng.integers(-2**31, 2**31, n, dtype=np.int64).astype(np.int32)),
        synth.ColumnData("i64", "INT64", rng.integers(-2**63, 2**63 - 1, n, dtype=np.int64)),
        synth.ColumnData("f64", "DOUBLE", rng.standard_normal(n)),
        synth.ColumnData("opt_f64", "DOUBLE", rng.standard_normal(n), rng.random(n) > 0.5),
        synth.ColumnData("allnull", "INT32", np.zeros(n, np.int32), np.zeros(n, bool)),
        synth.ColumnData("allvalid", "INT64", rng.integers(0, 9, n, dtype=np.int64), np.ones(n, bool)),
    ]
    cols[3].values[~cols[3].valid] = 0
    tab = synth.Table(cols)
    for rg, page, version, codec in ((n, 1 << 20, 1, "UNCOMPRESSED"), (5000, 999, 2, "SNAPPY"), (n, 8, 1, "SNAPPY")):
        spec = synth.TableSpec(rg, page, [synth.ColumnSpec("BYTE_STREAM_SPLIT", codec, version) for _ in cols])
        _roundtrip(eng, W.write_file(tab, spec))


def _bad_prefix(items):
    """DELTA_BYTE_ARRAY whose second prefix is longer than the first value."""
    items = [bytes(s) for s in items]
    prefix = [0, len(items[0]) + 1] + [0] * (len(items) - 2)
    return D.encode(prefix, 32) + DS.encode_length_byte_array(items)


@pytest.mark.parametrize("case", ["bss_ragged", "dlba_short", "dba_prefix"])
def test_v2_encodings_corrupt_pages(eng, case, monkeypatch):
    """Pages the oracle rejects give PQ_ERR_CORRUPT (no fault, no partial
    success): stream bytes that are not a whole number of values, value
    bytes that run past the page, a prefix longer than the value before."""
    from paper_2602_17335_gb300 import native as N
    rng = np.random.default_rng(3)
    n = 3000
    if case == "bss_ragged":
        orig = W._bss.encode
        monkeypatch.setattr(W._bss, "encode", lambda v, t: orig(v, t) + b"\x00")
        col, enc = synth.ColumnData("f", "DOUBLE", rng.standard_normal(n)), "BYTE_STREAM_SPLIT"
    elif case == "dlba_short":
        orig = W._dstr.encode_length_byte_array
        monkeypatch.setattr(W._dstr, "encode_length_byte_array", lambda items: orig(items)[:-1])
        col, enc = _string_column("s", [b"v%05d" % i for i in range(n)]), "DELTA_LENGTH_BYTE_ARRAY"
    else:
        monkeypatch.setattr(W._dstr, "encode_byte_array", _bad_prefix)
        col, enc = _string_column("s", [b"v%05d" % i for i in range(n)]), "DELTA_BYTE_ARRAY"
    data = W.write_file(synth.Table([col]), synth.TableSpec(n, 4096, [synth.ColumnSpec(enc)]))
    with pytest.raises(ValueError):
        R.read_file(data)
    with pytest.raises(N.PqError) as ei:
        eng.read([to_dev(data)])
    assert ei.value.status == N.PQ_ERR_CORRUPT


@pytest.mark.parametrize("writer", ["oracle", "native"])
def test_files_with_chosen_encodings(eng, writer):
    """Files whose every chunk carries the smallest valid encoding of its type
    (Section 3, "Encoding Flexibility"): encodings differ from chunk to chunk
    of one column, V1 and V2 pages, with and without Snappy."""
    from paper_2602_17335_gb300.tables import write_table
    for tab, rg in ((synth.config2_table(20_000, 6000, string_pool_size=700, zipf_k=2000), 6000),
                    (synth.v2_encodings_table(20_000, 7000), 7000)):
        for codec, version in (("UNCOMPRESSED", 1), ("SNAPPY", 2)):
            spec = synth.TableSpec(rg, 4096, [synth.ColumnSpec("AUTO", codec, version) for _ in tab.columns])
            data = W.write_file(tab, spec) if writer == "oracle" else bytes(write_table(tab, spec))
            _roundtrip(eng, data)
