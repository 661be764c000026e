"""File-level pins of the oracle writer/reader: round trips against the
seeded generator's arrays across encodings, page versions, codecs and
layouts, page-walk structure, and (where pyarrow is installed) reads of
oracle files by pyarrow and of pyarrow files by the oracle."""
import io

import numpy as np
import pytest

import synth
from oracle import reader as R
from oracle import writer as W
from oracle.parquet_meta import DATA_PAGE, DATA_PAGE_V2, DICTIONARY_PAGE


def expected_rows(col):
    if col.ptype == "BYTE_ARRAY":
        off, ch = col.values.materialize()
        return off, ch
    return np.asarray(col.values), None


def assert_matches(table, results):
    for col, r in zip(table.columns, results):
        if col.ptype == "BYTE_ARRAY":
            off, ch = col.values.materialize()
            assert np.array_equal(off, r.offsets), col.name
            assert np.array_equal(ch, r.chars), col.name
        else:
            v = np.asarray(col.values)
            assert r.values.dtype.itemsize == v.dtype.itemsize
            assert np.array_equal(v.view(np.uint8), r.values.view(np.uint8)), col.name
        if col.valid is None:
            assert r.valid is None
        else:
            assert np.array_equal(col.valid, r.valid)


SMALL = dict(string_pool_size=200, zipf_k=300)


def string_rows(col):
    """Row values of a BYTE_ARRAY column, b'' for a null row."""
    off, ch = col.values.materialize()
    rows = [bytes(ch[off[j]:off[j + 1]]) for j in range(len(off) - 1)]
    return rows if col.valid is None else [x if v else b"" for x, v in zip(rows, col.valid)]


def assert_rows_match(table, results):
    for col, r in zip(table.columns, results):
        if col.ptype == "BYTE_ARRAY":
            got = [bytes(r.chars[r.offsets[j]:r.offsets[j + 1]]) for j in range(len(r.offsets) - 1)]
            assert got == string_rows(col), col.name
        else:
            v = np.asarray(col.values)
            assert np.array_equal(v.view(np.uint8), r.values.view(np.uint8)), col.name
        assert (r.valid is None) if col.valid is None else np.array_equal(col.valid, r.valid)


@pytest.mark.parametrize("rg_rows,page_bytes", [(4096, 512), (1500, 2048), (10_000, 64 * 1024), (777, 8)])
@pytest.mark.parametrize("codec,version", [("UNCOMPRESSED", 1), ("SNAPPY", 1), ("UNCOMPRESSED", 2), ("SNAPPY", 2)])
def test_roundtrip_eight_column_table(rg_rows, page_bytes, codec, version):
    tab = synth.config2_table(6000, rg_rows, **SMALL)
    data = W.write_file(tab, synth.config2_spec(rg_rows, page_bytes, codec, version))
    assert_matches(tab, R.read_file(data))


@pytest.mark.parametrize("policy", ["rle", "packed", "mixed"])
def test_roundtrip_hybrid_policies(policy):
    tab = synth.config2_table(3000, 1024, **SMALL)
    spec = synth.config2_spec(1024, 777)
    for c in spec.columns:
        c.hybrid_policy = policy
    assert_matches(tab, R.read_file(W.write_file(tab, spec)))


def test_page_walk_structure_and_offset_index():
    tab = synth.config2_table(5000, 2000, **SMALL)
    data = W.write_file(tab, synth.config2_spec(2000, 1000))
    info = R.parse_footer(data)
    assert info.num_rows == 5000 and info.rg_rows == [2000, 2000, 1000]
    for ch in info.chunks:
        pages = R.chunk_pages(data, ch)
        data_pages = [p for p in pages if p.page_type in (DATA_PAGE, DATA_PAGE_V2)]
        dict_pages = [p for p in pages if p.page_type == DICTIONARY_PAGE]
        assert sum(p.num_values for p in data_pages) == ch.num_values
        assert len(dict_pages) == (1 if ch.column in (0, 3, 5, 6, 7) else 0)
        oi = R.read_offset_index(data, ch)
        assert [o for o, _, _ in oi] == [p.offset for p in data_pages]
        assert [s for _, s, _ in oi] == [p.header_len + p.compressed for p in data_pages]
        firsts = np.cumsum([0] + [p.num_values for p in data_pages])[:-1].tolist()
        assert [f for _, _, f in oi] == firsts
        assert pages[-1].offset + pages[-1].header_len + pages[-1].compressed == ch.start + ch.total_compressed


def test_page_size_rule_fixed_width():
    # 8 KiB pages of DOUBLE: floor(8192*8/64) = 1024 rows; OPTIONAL INT64: floor(65536/65)//8*8 = 1008
    tab = synth.config2_table(5000, 5000, **SMALL)
    data = W.write_file(tab, synth.config2_spec(5000, 8192))
    info = R.parse_footer(data)
    counts = {c: [p.num_values for p in R.chunk_pages(data, info.chunks[c]) if p.page_type == DATA_PAGE]
              for c in (2, 4, 0)}
    assert counts[2] == [1024] * 4 + [904]
    assert counts[4] == [1008] * 4 + [968]
    bw = int(np.unique(np.asarray(tab.columns[0].values)).size - 1).bit_length()
    per = (8192 * 8 // bw) // 8 * 8
    assert counts[0][0] == min(per, 5000)


def test_selective_compression_threshold():
    """A chunk of random doubles does not shrink under Snappy by 10%: with the
    threshold the chunk is written uncompressed (paper Section 3, Insight 4);
    the low-cardinality sorted column shrinks and keeps SNAPPY."""
    tab = synth.config2_table(4000, 4000, **SMALL)
    spec = synth.config2_spec(4000, 4096, codec="SNAPPY")
    for c in spec.columns:
        c.compress_threshold = 0.10
    data = W.write_file(tab, spec)
    info = R.parse_footer(data)
    assert info.chunks[2].codec == 0
    assert_matches(tab, R.read_file(data))


def test_config4_style_chunks_roundtrip():
    draws = synth.config4_draws(n_files=2, chunks_per_file=5, rows_lo=50, rows_hi=3000, page_lo=256, page_hi=8192)
    for d in draws:
        col, cspec = synth.config4_column(d)
        tab = synth.Table([col])
        data = W.write_file(tab, synth.TableSpec(rg_rows=1000, page_bytes=d.page_bytes, columns=[cspec]))
        assert_matches(tab, R.read_file(data))


def test_corrupt_files_raise():
    tab = synth.config2_table(500, 500, **SMALL)
    data = bytearray(W.write_file(tab, synth.config2_spec(500, 256)))
    with pytest.raises(ValueError):
        R.read_file(bytes(data[:-1]))
    info = R.parse_footer(bytes(data))
    ch = info.chunks[1]
    bad = bytearray(data)
    bad[ch.start + 2] ^= 0x7F    # damage the first page header of the DELTA chunk
    with pytest.raises(Exception):
        R.decode_chunk(bytes(bad), ch)


# ------------------------------------------------------------- pyarrow cross-check

def test_pyarrow_reads_oracle_files():
    pq = pytest.importorskip("pyarrow.parquet")
    tab = synth.config2_table(3000, 1000, **SMALL)
    for codec, version in (("UNCOMPRESSED", 1), ("SNAPPY", 2)):
        data = W.write_file(tab, synth.config2_spec(1000, 700, codec, version))
        t = pq.read_table(io.BytesIO(data))
        for i, col in enumerate(tab.columns):
            got = t.column(i).to_pylist()
            if col.ptype == "BYTE_ARRAY":
                off, ch = col.values.materialize()
                assert got == [bytes(ch[off[j]:off[j + 1]]) for j in range(len(off) - 1)]
            else:
                v = np.asarray(col.values).tolist()
                exp = v if col.valid is None else [x if m else None for x, m in zip(v, col.valid)]
                assert got == exp


@pytest.mark.parametrize("version,compression,dict_,delta", [
    ("1.0", "snappy", True, False), ("2.6", "snappy", True, False), ("2.6", "none", False, True),
    ("2.6", "snappy", False, True)])
def test_oracle_reads_pyarrow_files(version, compression, dict_, delta):
    pa = pytest.importorskip("pyarrow")
    pq = pytest.importorskip("pyarrow.parquet")
    rng = np.random.default_rng(11)
    n = 5000
    i32 = rng.integers(-1000, 1000, size=n).astype(np.int32)
    i64 = np.cumsum(rng.integers(0, 5, size=n)).astype(np.int64)
    f64 = rng.standard_normal(n)
    valid = rng.random(n) > 0.1
    strs = [b"s%d" % (x % 37) for x in rng.integers(0, 1000, size=n)]
    t = pa.table({"a": pa.array(i32), "b": pa.array(i64), "c": pa.array(f64),
                  "d": pa.array(i64, mask=~valid), "e": pa.array(strs, pa.binary())})
    kw = dict(version=version, compression=compression, use_dictionary=dict_, data_page_size=2048,
              row_group_size=2100, data_page_version="2.0" if version != "1.0" else "1.0")
    if delta:
        kw["column_encoding"] = {"a": "DELTA_BINARY_PACKED", "b": "DELTA_BINARY_PACKED"}
    buf = io.BytesIO()
    pq.write_table(t, buf, **kw)
    res = R.read_file(buf.getvalue())
    assert np.array_equal(res[0].values, i32)
    assert np.array_equal(res[1].values, i64)
    assert np.array_equal(res[2].values.view(np.int64), f64.view(np.int64))
    assert np.array_equal(res[3].valid, valid) and np.array_equal(res[3].values[valid], i64[valid])
    assert np.all(res[3].values[~valid] == 0)
    assert [bytes(res[4].chars[res[4].offsets[j]:res[4].offsets[j + 1]]) for j in range(n)] == strs


# ------------------------------------------------------------- V2 encodings (Insight 3)

@pytest.mark.parametrize("rg_rows,page_bytes", [(2500, 700), (6000, 64 * 1024), (999, 8)])
@pytest.mark.parametrize("codec,version", [("UNCOMPRESSED", 1), ("SNAPPY", 1), ("UNCOMPRESSED", 2), ("SNAPPY", 2)])
def test_roundtrip_v2_encodings(rg_rows, page_bytes, codec, version):
    tab = synth.v2_encodings_table(6000, rg_rows)
    data = W.write_file(tab, synth.v2_encodings_spec(rg_rows, page_bytes, codec, version))
    info = R.parse_footer(data)
    encs = {p.encoding for ch in info.chunks for p in R.chunk_pages(data, ch)}
    assert encs == {6, 7, 9}
    assert_rows_match(tab, R.read_file(data))


def test_pyarrow_reads_oracle_v2_encodings():
    pq = pytest.importorskip("pyarrow.parquet")
    tab = synth.v2_encodings_table(3000, 1100)
    for codec, version in (("UNCOMPRESSED", 1), ("SNAPPY", 2)):
        data = W.write_file(tab, synth.v2_encodings_spec(1100, 900, codec, version))
        t = pq.read_table(io.BytesIO(data))
        for i, col in enumerate(tab.columns):
            got = t.column(i).to_pylist()
            if col.ptype == "BYTE_ARRAY":
                rows = string_rows(col)
                exp = rows if col.valid is None else [x if v else None for x, v in zip(rows, col.valid)]
            else:
                v = np.asarray(col.values).tolist()
                exp = v if col.valid is None else [x if m else None for x, m in zip(v, col.valid)]
            assert got == exp, col.name


@pytest.mark.parametrize("page_version", ["1.0", "2.0"])
def test_oracle_reads_pyarrow_v2_encodings(page_version):
    pa = pytest.importorskip("pyarrow")
    pq = pytest.importorskip("pyarrow.parquet")
    rng = np.random.default_rng(5)
    n = 5000
    f64 = rng.standard_normal(n)
    i32 = rng.integers(-1000, 1000, size=n).astype(np.int32)
    i64 = rng.integers(-2**62, 2**62, size=n)
    valid = rng.random(n) > 0.1
    strs = [b"key%06d" % x for x in np.sort(rng.integers(0, 10**6, size=n))]
    t = pa.table({"a": pa.array(f64), "b": pa.array(i32), "c": pa.array(i64, mask=~valid),
                  "d": pa.array(strs, pa.binary()), "e": pa.array(strs, pa.binary(), mask=~valid)})
    buf = io.BytesIO()
    pq.write_table(t, buf, use_dictionary=False, data_page_size=2048, row_group_size=2100,
                   data_page_version=page_version,
                   column_encoding={"a": "BYTE_STREAM_SPLIT", "b": "BYTE_STREAM_SPLIT", "c": "BYTE_STREAM_SPLIT",
                                    "d": "DELTA_LENGTH_BYTE_ARRAY", "e": "DELTA_BYTE_ARRAY"})
    res = R.read_file(buf.getvalue())
    assert np.array_equal(res[0].values.view(np.int64), f64.view(np.int64))
    assert np.array_equal(res[1].values, i32)
    assert np.array_equal(res[2].valid, valid) and np.array_equal(res[2].values[valid], i64[valid])
    assert [bytes(res[3].chars[res[3].offsets[j]:res[3].offsets[j + 1]]) for j in range(n)] == strs
    assert [bytes(res[4].chars[res[4].offsets[j]:res[4].offsets[j + 1]]) for j in range(n)] == \
        [x if v else b"" for x, v in zip(strs, valid)]


# ------------------------------------------------------------- Zstandard (Section 2's codecs)

@pytest.mark.parametrize("page_version", ["1.0", "2.0"])
@pytest.mark.parametrize("level", [1, 9])
def test_oracle_reads_pyarrow_zstd_files(page_version, level):
    pa = pytest.importorskip("pyarrow")
    pq = pytest.importorskip("pyarrow.parquet")
    rng = np.random.default_rng(21)
    n = 6000
    i64 = np.cumsum(rng.integers(0, 5, size=n)).astype(np.int64)
    f64 = rng.standard_normal(n)
    valid = rng.random(n) > 0.1
    strs = [b"s%d" % (x % 97) for x in rng.integers(0, 1000, size=n)]
    t = pa.table({"a": pa.array(i64), "b": pa.array(f64), "c": pa.array(i64, mask=~valid),
                  "d": pa.array(strs, pa.binary()), "e": pa.array(strs, pa.binary(), mask=~valid)})
    buf = io.BytesIO()
    pq.write_table(t, buf, compression="zstd", compression_level=level, data_page_size=4096, row_group_size=2500,
                   data_page_version=page_version, use_dictionary=["d", "e"],
                   column_encoding={"a": "DELTA_BINARY_PACKED", "b": "BYTE_STREAM_SPLIT"})
    data = buf.getvalue()
    assert {ch.codec for ch in R.parse_footer(data).chunks} == {6}
    res = R.read_file(data)
    assert np.array_equal(res[0].values, i64)
    assert np.array_equal(res[1].values.view(np.int64), f64.view(np.int64))
    assert np.array_equal(res[2].valid, valid) and np.array_equal(res[2].values[valid], i64[valid])
    assert [bytes(res[3].chars[res[3].offsets[j]:res[3].offsets[j + 1]]) for j in range(n)] == strs
    assert [bytes(res[4].chars[res[4].offsets[j]:res[4].offsets[j + 1]]) for j in range(n)] == \
        [x if v else b"" for x, v in zip(strs, valid)]


def test_oracle_zstd_files_round_trip_and_pyarrow_reads_them():
    tab = synth.config2_table(4000, 1500, **SMALL)
    for version in (1, 2):
        spec = synth.config2_spec(1500, 2048, "ZSTD", version)
        data = W.write_file(tab, spec)
        assert {ch.codec for ch in R.parse_footer(data).chunks} == {6}
        assert_rows_match(tab, R.read_file(data))
    pq = pytest.importorskip("pyarrow.parquet")
    t = pq.read_table(io.BytesIO(data))
    for i, col in enumerate(tab.columns):
        got = t.column(i).to_pylist()
        if col.ptype == "BYTE_ARRAY":
            assert got == string_rows(col)
        else:
            v = np.asarray(col.values).tolist()
            assert got == (v if col.valid is None else [x if m else None for x, m in zip(v, col.valid)])


@pytest.mark.parametrize("name", ["zstd_eight_column_v1.parquet", "zstd_eight_column_v2.parquet"])
def test_zstd_fixtures_decode_to_their_table(name):
    """The committed Zstandard fixtures (libzstd pages, written by
    tests/golden/make_zstd_fixtures.py) decode, with the oracle, to the
    seeded table they were made from."""
    import importlib.util
    import os
    golden = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_zstd_fixtures", os.path.join(golden, "make_zstd_fixtures.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    rows, rg, _, _, _ = mod.FIXTURES[name]
    data = open(os.path.join(golden, name), "rb").read()
    assert {ch.codec for ch in R.parse_footer(data).chunks} == {6}
    tab = synth.config2_table(rows, rg, string_pool_size=700, zipf_k=2000)
    assert_rows_match(tab, R.read_file(data))
