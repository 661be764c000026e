"""The engine's native writer (`pq_write_table`, the rewriter of the paper's
Sections 3 and 5) against the oracle writer, on the CPU (no GPU needed).

Both follow the same deterministic layout rules, so on uncompressed data
they must write the same bytes (only the footer's created_by differs);
with Snappy the compressors differ, so the file must read back to the table
and keep the same page structure; its Zstandard pages (LZ77 sequences under
fitted or predefined FSE tables) read back through the oracle and libzstd.  The
per-chunk encoding choice ("AUTO", Section 3's "Encoding Flexibility") is
pinned to the smallest explicit encoding of each chunk and to the obvious
winners of shaped data."""
import io

import numpy as np
import pytest

import synth
from oracle import reader as R
from oracle import thrift as T
from oracle import writer as W
from oracle import zstd as Z


def _native():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.tables import write_table
    return N, write_table


def _split(data):
    """(bytes before the footer, footer fields without created_by)."""
    flen = int.from_bytes(data[-8:-4], "little")
    fs = len(data) - 8 - flen
    meta, _ = T.decode_struct(data, fs, len(data) - 8)
    meta.pop(6, None)
    return data[:fs], meta


def _tables():
    return {"eight_column": (synth.config2_table(12_000, 5000, string_pool_size=300, zipf_k=500),
                             lambda v: synth.config2_spec(5000, 3000, "UNCOMPRESSED", v)),
            "v2_encodings": (synth.v2_encodings_table(12_000, 5000),
                             lambda v: synth.v2_encodings_spec(5000, 3000, "UNCOMPRESSED", v))}


def _string_rows(col):
    off, ch = col.values.materialize()
    rows = [bytes(ch[off[j]:off[j + 1]]) for j in range(len(off) - 1)]
    return rows if col.valid is None else [x if v else b"" for x, v in zip(rows, col.valid)]


@pytest.mark.parametrize("table", ["eight_column", "v2_encodings"])
@pytest.mark.parametrize("version", [1, 2])
@pytest.mark.parametrize("auto", [False, True])
def test_native_writer_matches_oracle_bytes(table, version, auto):
    _, write_table = _native()
    tab, spec_of = _tables()[table]
    spec = spec_of(version)
    if auto:
        for c in spec.columns:
            c.encoding = "AUTO"
    native = bytes(write_table(tab, spec))
    oracle = W.write_file(tab, spec)
    assert _split(native) == _split(oracle)


@pytest.mark.parametrize("version", [1, 2])
def test_native_writer_snappy_reads_back(version):
    _, write_table = _native()
    tab = synth.v2_encodings_table(9000, 4000)
    spec = synth.v2_encodings_spec(4000, 2048, "SNAPPY", version)
    native = bytes(write_table(tab, spec))
    res = R.read_file(native)
    for col, r in zip(tab.columns, res):
        if col.ptype == "BYTE_ARRAY":
            got = [bytes(r.chars[r.offsets[j]:r.offsets[j + 1]]) for j in range(len(r.offsets) - 1)]
            assert got == _string_rows(col), col.name
        else:
            assert np.array_equal(np.asarray(col.values).view(np.uint8), r.values.view(np.uint8)), col.name
    # same pages (row counts, encodings) as the oracle writer's file
    oracle = W.write_file(tab, spec)

    def pages(data):
        info = R.parse_footer(data)
        return [[(p.page_type, p.num_values, p.encoding) for p in R.chunk_pages(data, ch)] for ch in info.chunks]

    assert pages(native) == pages(oracle)


def test_selective_compression_decisions():
    """Insight 4's threshold: incompressible doubles drop Snappy, sorted
    low-cardinality values keep it, in both writers."""
    _, write_table = _native()
    rng = np.random.default_rng(4)
    n = 20_000
    cols = [synth.ColumnData("noise", "DOUBLE", rng.standard_normal(n)),
            synth.ColumnData("sorted", "INT32", np.sort(rng.integers(0, 40, n)).astype(np.int32))]
    tab = synth.Table(cols)
    spec = synth.TableSpec(n, 1 << 16, [synth.ColumnSpec("PLAIN", "SNAPPY", 1, compress_threshold=0.10)
                                        for _ in cols])
    for data in (bytes(write_table(tab, spec)), W.write_file(tab, spec)):
        codecs = [ch.codec for ch in R.parse_footer(data).chunks]
        assert codecs == [0, 1]


def test_auto_is_the_smallest_candidate():
    """AUTO's chunk equals the smallest explicit candidate of its type."""
    tab = synth.v2_encodings_table(6000, 6000)
    tab2 = synth.config2_table(6000, 6000, string_pool_size=300, zipf_k=500)
    for col in tab.columns + tab2.columns:
        sizes = {}
        for enc in W.CANDIDATES[col.ptype]:
            _, meta, _, _ = W.write_chunk(col, synth.ColumnSpec(enc), 4096, 0)
            sizes[enc] = dict((f, v) for f, _, v in meta)[6]
        _, meta, _, _ = W.write_chunk(col, synth.ColumnSpec("AUTO"), 4096, 0)
        assert dict((f, v) for f, _, v in meta)[6] == min(sizes.values()), col.name
        assert W.choose_encoding(col, synth.ColumnSpec("AUTO"), 4096) == min(sizes, key=lambda e: (
            sizes[e], W.CANDIDATES[col.ptype].index(e)))


def test_auto_obvious_winners():
    """Shaped data whose best encoding follows from the definitions:
    sorted keys with small steps -> DELTA_BINARY_PACKED (about 3 bits per
    value); 16 distinct values -> RLE_DICTIONARY (4-bit indices); sorted
    strings with long shared stems -> DELTA_BYTE_ARRAY; distinct random
    strings -> DELTA_LENGTH_BYTE_ARRAY (packed lengths beat 4-byte ones);
    random doubles -> PLAIN (BYTE_STREAM_SPLIT has the same size; the tie
    goes to PLAIN)."""
    rng = np.random.default_rng(12)
    n = 8000
    cases = [
        (synth.ColumnData("keys", "INT64", synth.sorted_keys_int64(rng, n)), "DELTA_BINARY_PACKED"),
        (synth.ColumnData("card16", "INT32", synth.lowcard_int32(rng, n, 16)), "RLE_DICTIONARY"),
        (synth.ColumnData("stems", "BYTE_ARRAY", synth.strings_sorted(rng, n, n)), "DELTA_BYTE_ARRAY"),
        (synth.ColumnData("distinct", "BYTE_ARRAY", synth.strings_uniform(rng, n, k=10 * n)), "DELTA_LENGTH_BYTE_ARRAY"),
        (synth.ColumnData("noise", "DOUBLE", rng.standard_normal(n)), "PLAIN"),
    ]
    for col, want in cases:
        assert W.choose_encoding(col, synth.ColumnSpec("AUTO"), 1 << 16) == want, col.name


def test_native_writer_rejects_invalid_encodings():
    N, _ = _native()
    v = np.arange(16, dtype=np.int32)
    for enc, status in ((6, N.PQ_ERR_INVALID_ARG), (7, N.PQ_ERR_INVALID_ARG), (3, N.PQ_ERR_UNSUPPORTED)):
        w = N.pq_write_column()
        w.name = b"x"
        w.type = N.PQ_TYPE_INT32
        w.encoding = enc
        w.page_version = 1
        w.compress_threshold = -1.0
        w.values = v.ctypes.data
        with pytest.raises(N.PqError) as ei:
            N.pq_write_table([w], 16, 16, 1024)
        assert ei.value.status == status
    off = np.array([0, 1, 2], dtype=np.int64)
    chars = np.frombuffer(b"ab", dtype=np.uint8).copy()
    w = N.pq_write_column()
    w.name = b"s"
    w.type = N.PQ_TYPE_BYTE_ARRAY
    w.encoding = 9
    w.page_version = 1
    w.compress_threshold = -1.0
    w.values = off.ctypes.data
    w.chars = chars.ctypes.data
    with pytest.raises(N.PqError) as ei:
        N.pq_write_table([w], 2, 2, 1024)
    assert ei.value.status == N.PQ_ERR_INVALID_ARG


def _frame_block_types(frame):
    """Block types of one Zstandard frame (0 raw, 1 RLE, 2 compressed)."""
    pos = 4
    fhd = frame[pos]
    pos += 1
    single, fcs = (fhd >> 5) & 1, fhd >> 6
    pos += 0 if single else 1
    pos += single if fcs == 0 else {1: 2, 2: 4, 3: 8}[fcs]
    out = []
    while True:
        h = int.from_bytes(frame[pos:pos + 3], "little")
        pos += 3
        t = (h >> 1) & 3
        out.append(t)
        pos += 1 if t == 1 else h >> 3
        if h & 1:
            return out


def zstd_pages(data):
    """(column, frame, uncompressed bytes) of every compressed page."""
    for ch in R.parse_footer(data).chunks:
        for p in R.chunk_pages(data, ch):
            body = data[p.offset + p.header_len:p.offset + p.header_len + p.compressed]
            if p.page_type == 3:
                if not p.is_compressed:
                    continue
                yield ch.column, body[p.def_len + p.rep_len:], p.uncompressed - p.def_len - p.rep_len
            else:
                yield ch.column, body, p.uncompressed


@pytest.mark.parametrize("version", [1, 2])
def test_native_writer_zstd_pages(version):
    """Zstandard pages of the native writer: the oracle reads them back to
    the table, compressible columns get compressed blocks (LZ77 sequences
    under FSE tables), uniformly random bytes raw blocks,
    and libzstd (through pyarrow) reads the same file."""
    _, write_table = _native()
    rng = np.random.default_rng(3)
    n = 30_000
    cols = [synth.ColumnData("sorted", "INT64", np.cumsum(rng.integers(0, 3, n)).astype(np.int64)),
            synth.ColumnData("strs", "BYTE_ARRAY", synth.strings_uniform(rng, n, k=200)),
            synth.ColumnData("lowcard", "INT32", rng.integers(0, 5, n).astype(np.int32), rng.random(n) > 0.2),
            synth.ColumnData("noise", "INT64", rng.integers(-2**63, 2**63 - 1, n, dtype=np.int64))]
    cols[2].values[~cols[2].valid] = 0
    tab = synth.Table(cols)
    spec = synth.TableSpec(12_000, 1 << 16, [synth.ColumnSpec("PLAIN", "ZSTD", version) for _ in cols])
    data = bytes(write_table(tab, spec))
    res = R.read_file(data)
    for col, r in zip(tab.columns, res):
        if col.ptype == "BYTE_ARRAY":
            off, ch = col.values.materialize()
            assert np.array_equal(off, r.offsets) and np.array_equal(ch, r.chars)
        else:
            assert np.array_equal(np.asarray(col.values).view(np.uint8), r.values.view(np.uint8))
    kinds = {}
    for c, frame, _ in zstd_pages(data):
        kinds.setdefault(c, set()).update(_frame_block_types(frame))
    assert 2 in kinds[0] and 2 in kinds[1] and 2 in kinds[2]
    assert kinds[3] == {0}
    pq = pytest.importorskip("pyarrow.parquet")
    t = pq.read_table(io.BytesIO(data))
    assert t.column(0).to_pylist() == cols[0].values.tolist()
    assert t.column(3).to_pylist() == cols[3].values.tolist()
    assert t.column(2).to_pylist() == [int(v) if m else None for v, m in zip(cols[2].values, cols[2].valid)]


def test_native_zstd_frames_decode_with_libzstd():
    """Every page frame the native writer makes decodes with libzstd to the
    oracle's bytes (frames with up to several 128 KB blocks)."""
    pa = pytest.importorskip("pyarrow")
    _, write_table = _native()
    tab = synth.config2_table(200_000, 200_000, string_pool_size=300, zipf_k=500)
    data = bytes(write_table(tab, synth.config2_spec(200_000, 1 << 20, "ZSTD", 1)))
    n = 0
    for _, frame, size in zstd_pages(data):
        want = Z.decompress(frame)
        assert len(want) == size
        assert pa.Codec("zstd").decompress(frame, decompressed_size=size, asbytes=True) == want
        n += 1
    assert n > 10


def test_native_zstd_huffman_literals(monkeypatch):
    """Literal bytes below 128 come out Huffman-coded in 1- and 4-stream
    sections, and libzstd reads them."""
    pa = pytest.importorskip("pyarrow")
    _, write_table = _native()
    rng = np.random.default_rng(8)
    rows = [(65 + np.minimum(rng.geometric(0.5, 100 if k % 2 else 1100) - 1, 60)).astype(np.uint8).tobytes()
            for k in range(400)]   # lengths 100 and 1100: their bytes are below 128 too
    lens = np.array([len(r) for r in rows], dtype=np.int64)
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    col = synth.ColumnData("geo", "BYTE_ARRAY", synth.StringData(off, np.frombuffer(b"".join(rows), np.uint8).copy(),
                                                                 np.arange(len(rows), dtype=np.int32)))
    data = bytes(write_table(synth.Table([col]), synth.TableSpec(len(rows), 1 << 20,
                                                                 [synth.ColumnSpec("PLAIN", "ZSTD", 1)])))
    kinds = set()
    orig = Z.decode_literals

    def spy(buf, pos, end, st):
        kinds.add((buf[pos] & 3, (buf[pos] >> 2) & 3))
        return orig(buf, pos, end, st)
    monkeypatch.setattr(Z, "decode_literals", spy)
    r = R.read_file(data)[0]
    assert [bytes(r.chars[r.offsets[j]:r.offsets[j + 1]]) for j in range(len(rows))] == rows
    assert (2, 0) in kinds and ((2, 2) in kinds or (2, 3) in kinds)
    for _, frame, size in zstd_pages(data):
        assert pa.Codec("zstd").decompress(frame, decompressed_size=size, asbytes=True) == Z.decompress(frame)


def test_huffman_length_limit():
    """The writer's code lengths: at most 11 bits, a complete prefix code
    (Kraft sum exactly 1), never shorter for a rarer symbol; Fibonacci counts
    (19 bits deep unrestricted) force the limit."""
    import ctypes
    import os
    import shutil
    import subprocess
    import tempfile
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = os.path.join(tempfile.mkdtemp(), "huf.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                    os.path.join(root, "paper_2602_17335_gb300", "csrc"),
                    os.path.join(root, "tests", "huf_lengths_harness.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    fib = [1, 1]
    while len(fib) < 20:
        fib.append(fib[-1] + fib[-2])
    rng = np.random.default_rng(2)
    cases = [fib, fib[::-1], [1] * 128, [5] + [0] * 50 + [7], list(rng.integers(0, 1000, 128)),
             list((2.0 ** -np.arange(40) * 2 ** 30).astype(np.int64) + 1)]
    for counts in cases:
        cnt = np.array(counts, dtype=np.uint32)
        ln = np.zeros(len(cnt), dtype=np.int32)
        ok = lib.huf_lengths_host(cnt.ctypes.data, len(cnt), ln.ctypes.data)
        assert ok
        used = ln[cnt > 0]
        assert np.all(ln[cnt == 0] == 0) and used.min() >= 1 and used.max() <= 11
        assert sum(2.0 ** -int(l) for l in used) == 1.0
        order = np.argsort(-cnt[cnt > 0], kind="stable")
        assert np.all(np.diff(used[order]) >= 0) or len(used) < 2
    ln = np.zeros(20, dtype=np.int32)
    lib.huf_lengths_host(np.array(fib, np.uint32).ctypes.data, 20, ln.ctypes.data)
    assert ln.max() == 11


def test_native_zstd_fse_compressed_weights(monkeypatch):
    """Binary pages (literal bytes of 128 and above) get Huffman literals
    whose weights are FSE-compressed (normalized counts, table description,
    two interleaved states); libzstd reads every frame."""
    pa = pytest.importorskip("pyarrow")
    _, write_table = _native()
    rng = np.random.default_rng(3)
    n = 40_000
    cols = [synth.ColumnData("sorted", "INT64", np.cumsum(rng.integers(0, 1000, n)).astype(np.int64)),
            synth.ColumnData("rounded", "DOUBLE", np.round(rng.standard_normal(n), 2))]
    data = bytes(write_table(synth.Table(cols), synth.TableSpec(n, 1 << 20, [synth.ColumnSpec("PLAIN", "ZSTD", 1)
                                                                            for _ in cols])))
    forms = []
    orig = Z.read_huffman_description

    def spy(buf, pos, end):
        forms.append("direct" if buf[pos] >= 128 else "fse")
        return orig(buf, pos, end)
    monkeypatch.setattr(Z, "read_huffman_description", spy)
    res = R.read_file(data)
    for c, r in zip(cols, res):
        assert np.array_equal(np.asarray(c.values).view(np.uint8), r.values.view(np.uint8))
    assert "fse" in forms
    for _, frame, size in zstd_pages(data):
        assert pa.Codec("zstd").decompress(frame, decompressed_size=size, asbytes=True) == Z.decompress(frame)


def test_native_zstd_fitted_sequence_tables(monkeypatch):
    """Blocks whose sequence codes pay for their own FSE tables carry them
    (transmitted tables; an RLE table where one code is used), and libzstd
    reads every frame."""
    pa = pytest.importorskip("pyarrow")
    _, write_table = _native()
    rng = np.random.default_rng(5)
    n = 60_000
    cols = [synth.ColumnData("sorted", "INT64", np.cumsum(rng.integers(0, 1000, n)).astype(np.int64)),
            synth.ColumnData("lowcard", "INT32", rng.integers(0, 3, n).astype(np.int32))]
    data = bytes(write_table(synth.Table(cols), synth.TableSpec(n, 1 << 20, [synth.ColumnSpec("PLAIN", "ZSTD", 2)
                                                                            for _ in cols])))
    modes = set()
    orig = Z._table

    def spy(buf, pos, end, mode, name, st):
        modes.add(mode)
        return orig(buf, pos, end, mode, name, st)
    monkeypatch.setattr(Z, "_table", spy)
    for c, r in zip(cols, R.read_file(data)):
        assert np.array_equal(np.asarray(c.values).view(np.uint8), r.values.view(np.uint8))
    assert {1, 2} <= modes
    for _, frame, size in zstd_pages(data):
        assert pa.Codec("zstd").decompress(frame, decompressed_size=size, asbytes=True) == Z.decompress(frame)


_WRITER_FUZZ = r'''
import ctypes, pickle, sys
sys.path.insert(0, sys.argv[3])
from paper_2602_17335_gb300 import native as N
lib = ctypes.CDLL(sys.argv[1])
lib.pq_write_table.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                               ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
lib.pq_write_free.argtypes = [ctypes.c_void_p]
out = []
for blob, page, kind in pickle.load(open(sys.argv[2], "rb")):
    if kind == "bytes":
        offs = (ctypes.c_int64 * 2)(0, len(blob))
        chars = ctypes.create_string_buffer(blob, max(len(blob), 1))
        col = N.pq_write_column(b"b", N.PQ_TYPE_BYTE_ARRAY, 0, 6, 1, -1.0, ctypes.cast(offs, ctypes.c_void_p),
                                ctypes.cast(chars, ctypes.c_void_p), None)
        n_rows = 1
    else:
        vals = ctypes.create_string_buffer(blob, max(len(blob), 8))
        col = N.pq_write_column(b"i", N.PQ_TYPE_INT64, 0, 6, 2, -1.0, ctypes.cast(vals, ctypes.c_void_p), None, None)
        n_rows = len(blob) // 8
    arr = (N.pq_write_column * 1)(col)
    p = ctypes.c_void_p()
    size = ctypes.c_uint64()
    rc = lib.pq_write_table(ctypes.cast(arr, ctypes.c_void_p), 1, n_rows, max(n_rows, 1), page, 1, 1,
                            ctypes.byref(p), ctypes.byref(size))
    assert rc == 0, rc
    out.append(ctypes.string_at(p, size.value))
    lib.pq_write_free(p)
pickle.dump(out, open(sys.argv[2] + ".out", "wb"))
'''


def test_native_zstd_writer_under_asan(tmp_path):
    """The writer (its Zstandard encoder: matching, Huffman literals with
    both weight forms, fitted and predefined FSE tables) compiled with
    AddressSanitizer/UBSan on inputs of many shapes and sizes: no invalid
    access, and every page decodes with libzstd and the oracle."""
    import os
    import pickle
    import shutil
    import subprocess
    import sys
    pa = pytest.importorskip("pyarrow")
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    asan = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    ubsan = subprocess.run(["g++", "-print-file-name=libubsan.so"], capture_output=True, text=True).stdout.strip()
    if not (os.path.isabs(asan) and os.path.exists(asan) and os.path.isabs(ubsan) and os.path.exists(ubsan)):
        pytest.skip("no sanitizer runtime")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = str(tmp_path / "writer_asan.so")
    subprocess.run(["g++", "-O1", "-g", "-std=c++17", "-shared", "-fPIC", "-fsanitize=address,undefined",
                    "-fno-omit-frame-pointer", "-I", os.path.join(root, "include"), "-I",
                    os.path.join(root, "paper_2602_17335_gb300", "csrc"),
                    os.path.join(root, "paper_2602_17335_gb300", "csrc", "writer.cpp"), "-o", so, "-lpthread"],
                   check=True)
    rng = np.random.default_rng(6)
    from test_oracle_pins import _zstd_inputs
    cases = []
    for i, x in enumerate(_zstd_inputs(np.random.default_rng(4))[:60]):
        page = [700, 1 << 16, 1 << 20][i % 3]
        if i % 2:
            cases.append((x, page, "bytes"))
        else:
            cases.append((x[:len(x) // 8 * 8] or bytes(8), page, "int64"))
    cases.append((bytes(rng.integers(0, 2, 400_000, dtype=np.uint8)), 1 << 20, "bytes"))
    pk = str(tmp_path / "cases.pkl")
    pickle.dump(cases, open(pk, "wb"))
    env = dict(os.environ, LD_PRELOAD=asan + ":" + ubsan, ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", _WRITER_FUZZ, so, pk, root], capture_output=True, text=True, env=env,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "Sanitizer" not in r.stderr and "runtime error" not in r.stderr, r.stderr[-3000:]
    files = pickle.load(open(pk + ".out", "rb"))
    assert len(files) == len(cases)
    for (blob, _, kind), data in zip(cases, files):
        res = R.read_file(data)[0]
        if kind == "bytes":
            assert res.chars.tobytes() == blob
        else:
            assert res.values.tobytes() == (blob[:len(blob) // 8 * 8])
        for _, frame, size in zstd_pages(data):
            assert pa.Codec("zstd").decompress(frame, decompressed_size=size, asbytes=True) == Z.decompress(frame)


@pytest.mark.parametrize("writer", ["oracle", "native"])
def test_pyarrow_reads_chosen_encodings_with_codecs(writer):
    """Files whose chunks carry their chosen encodings (every valid encoding
    of each type can win) under each codec, V1 and V2 pages: pyarrow reads
    the same values."""
    pq = pytest.importorskip("pyarrow.parquet")
    _, write_table = _native()
    tabs = [synth.config2_table(6000, 2500, string_pool_size=300, zipf_k=500), synth.v2_encodings_table(6000, 2500)]
    for tab in tabs:
        for codec, version in (("UNCOMPRESSED", 2), ("SNAPPY", 1), ("ZSTD", 2)):
            spec = synth.TableSpec(2500, 2048, [synth.ColumnSpec("AUTO", codec, version) for _ in tab.columns])
            data = W.write_file(tab, spec) if writer == "oracle" else bytes(write_table(tab, spec))
            t = pq.read_table(io.BytesIO(data))
            for i, col in enumerate(tab.columns):
                got = t.column(i).to_pylist()
                if col.ptype == "BYTE_ARRAY":
                    rows = _string_rows(col)
                    exp = rows if col.valid is None else [x if v else None for x, v in zip(rows, col.valid)]
                else:
                    v = np.asarray(col.values).tolist()
                    exp = v if col.valid is None else [x if m else None for x, m in zip(v, col.valid)]
                assert got == exp, (writer, codec, version, col.name)


def _snappy_elements(b):
    """(declared length, [(kind, output offset, length, copy offset)]) of a raw
    Snappy block, parsed here on its own."""
    i, x, sh = 0, 0, 0
    while True:
        y = b[i]
        i += 1
        x |= (y & 0x7F) << sh
        sh += 7
        if not y & 0x80:
            break
    out, els = 0, []
    while i < len(b):
        t = b[i]
        kind = t & 3
        if kind == 0:
            n = t >> 2
            i += 1
            if n >= 60:
                nb = n - 59
                n = int.from_bytes(b[i:i + nb], "little")
                i += nb
            els.append((0, out, n + 1, 0))
            i += n + 1
            out += n + 1
            continue
        if kind == 1:
            n, off = 4 + ((t >> 2) & 7), ((t >> 5) << 8) | b[i + 1]
            i += 2
        elif kind == 2:
            n, off = (t >> 2) + 1, int.from_bytes(b[i + 1:i + 3], "little")
            i += 3
        else:
            n, off = (t >> 2) + 1, int.from_bytes(b[i + 1:i + 5], "little")
            i += 5
        els.append((kind, out, n, off))
        out += n
    return x, els


def test_native_snappy_fragments():
    """The native writer frames Snappy pages as the reference compressor does:
    64 KiB fragments compressed on their own, so that every multiple of 65536
    in a page's output starts an element and no copy reads before the start
    of its own fragment (the GPU reader decompresses large pages fragment by
    fragment on that basis); the pages still read back to the table."""
    _, write_table = _native()
    tab = synth.config2_table(200_000, 200_000, string_pool_size=3000, zipf_k=5000)
    spec = synth.config2_spec(200_000, 1 << 20, "SNAPPY", 1)
    for c in spec.columns:
        c.compress_threshold = -1.0
    native = bytes(write_table(tab, spec))
    info = R.parse_footer(native)
    big = 0
    for ch in info.chunks:
        for p in R.chunk_pages(native, ch):
            body = native[p.offset + p.header_len:p.offset + p.header_len + p.compressed]
            n, els = _snappy_elements(body)
            assert n == p.uncompressed
            starts = {o for _, o, _, _ in els}
            for f in range(65536, n, 65536):
                assert f in starts, (ch.column, f)
            for kind, o, ln, off in els:
                if kind:
                    assert o - off >= (o // 65536) * 65536, (ch.column, o, off)
                assert (o + ln - 1) // 65536 == o // 65536, (ch.column, o, ln)
            big += n > 2 * 65536
    assert big >= 8  # dictionary and data pages of several fragments
    res = R.read_file(native)
    for col, r in zip(tab.columns, res):
        if col.ptype == "BYTE_ARRAY":
            got = [bytes(r.chars[r.offsets[j]:r.offsets[j + 1]]) for j in range(len(r.offsets) - 1)]
            assert got == _string_rows(col), col.name
        else:
            assert np.array_equal(np.asarray(col.values).view(np.uint8), r.values.view(np.uint8)), col.name
