"""GPU scan vs CPU oracle, bit for bit, through the C ABI.

Inputs are files the oracle writer produced from seeded synthetic tables
shaped like the scan workloads (eight-column table, single dictionary
column); sizes span several 8192-row work items and 2048-row tiles with
ragged tails.  Expected values always come from the oracle reader."""
import numpy as np
import pytest

import synth
from oracle import reader as R
from oracle import writer as W

from gpu_util import assert_columns_equal, engine, slice_result, to_dev

pytestmark = pytest.mark.gpu

SMALL = dict(string_pool_size=700, zipf_k=2000)


@pytest.fixture(scope="module")
def eng():
    e = engine()
    yield e
    e.close()


def _roundtrip(eng, data, **kw):
    from paper_2602_17335_gb300 import native as N
    expect = R.read_file(data)
    outs = eng.read([to_dev(data)], **kw)
    cols = kw.get("columns")
    rb = kw.get("row_begin", 0)
    rc = kw.get("row_count", -1)
    rows = len(expect[0].values) if expect[0].values is not None else len(expect[0].offsets) - 1
    hi = rows if rc < 0 else rb + rc
    exp = [slice_result(expect[c], rb, hi) for c in (cols if cols is not None else range(len(expect)))]
    assert_columns_equal(outs, exp)
    return N


@pytest.mark.parametrize("rg_rows,page_bytes", [(16384, 2048), (25000, 64 * 1024), (40000, 1 << 20),
                                                (7000, 700)])
@pytest.mark.parametrize("codec,version", [("UNCOMPRESSED", 1), ("UNCOMPRESSED", 2), ("SNAPPY", 1),
                                           ("SNAPPY", 2)])
def test_eight_column_table(eng, rg_rows, page_bytes, codec, version):
    tab = synth.config2_table(40_000, rg_rows, **SMALL)
    data = W.write_file(tab, synth.config2_spec(rg_rows, page_bytes, codec, version))
    _roundtrip(eng, data)


@pytest.mark.parametrize("policy", ["rle", "packed", "mixed"])
def test_hybrid_writer_policies(eng, policy):
    tab = synth.config2_table(30_000, 30_000, **SMALL)
    spec = synth.config2_spec(30_000, 4096)
    spec.seed = 5
    for c in spec.columns:
        c.hybrid_policy = policy
    _roundtrip(eng, W.write_file(tab, spec))


def test_single_dictionary_column(eng):
    n = 1 << 18
    tab = synth.config1_table(n)
    _roundtrip(eng, W.write_file(tab, synth.config1_spec(1 << 20, n)))


@pytest.mark.parametrize("rb,rc,cols", [(0, 1, None), (8191, 2, [0, 4, 5]), (12345, 20000, [1, 2, 3]),
                                        (39999, 1, [4, 5, 6, 7]), (5000, 0, [0]), (0, -1, [7, 5]),
                                        (16383, 8194, None)])
def test_row_ranges_and_column_subsets(eng, rb, rc, cols):
    tab = synth.config2_table(40_000, 16384, **SMALL)
    data = W.write_file(tab, synth.config2_spec(16384, 8192, "SNAPPY", 1))
    _roundtrip(eng, data, columns=cols, row_begin=rb, row_count=rc)


@pytest.mark.parametrize("mode", ["plain", "graph", "resident"])
def test_scan_modes(eng, mode):
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.scan import alloc_outputs
    tab = synth.config2_table(30_000, 12_000, **SMALL)
    data = W.write_file(tab, synth.config2_spec(12_000, 16 * 1024, "SNAPPY", 2))
    expect = R.read_file(data)
    flags = {"plain": N.PQ_SCAN_PLAIN, "graph": N.PQ_SCAN_GRAPH,
             "resident": N.PQ_SCAN_RESIDENT_DICT | N.PQ_SCAN_GRAPH}[mode]
    dev = to_dev(data)
    idx = eng.index([dev])
    plan, sizes = eng.plan(idx, flags=flags)
    for rep in range(3):  # replays reuse the plan (and the captured graph)
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


def test_page_table_matches_oracle_walk(eng):
    from paper_2602_17335_gb300 import native as N
    tab = synth.config2_table(20_000, 8000, **SMALL)
    for oi in (True, False):
        spec = synth.config2_spec(8000, 3000, "SNAPPY", 2, offset_index=oi)
        data = W.write_file(tab, spec)
        info = R.parse_footer(data)
        idx = eng.index([to_dev(data)])
        pages = N.pq_index_copy_pages(idx)
        ii = N.pq_index_get_info(idx)
        assert ii.used_offset_index == (1 if oi else 0)
        exp = []
        for ci, ch in enumerate(info.chunks):
            row = 0
            for p in R.chunk_pages(data, ch):
                first = 0 if p.page_type == 2 else row
                if p.page_type != 2:
                    row += p.num_values
                exp.append((p.offset, ci, p.page_type, p.encoding, p.header_len, p.uncompressed,
                            p.compressed, p.num_values, p.num_nulls, p.def_len, first))
        got = [(g.header_offset, g.chunk, g.page_type, g.encoding, g.header_len, g.uncompressed_size,
                g.compressed_size, g.num_values, g.num_nulls, g.def_len, g.first_row) for g in pages]
        assert got == exp
        assert ii.num_rows == 20_000 and ii.n_chunks == len(info.chunks)
        N.pq_free_index(idx)


def test_multiple_files(eng):
    from oracle.reader import ColumnResult
    datas, expects = [], []
    for f in range(3):
        tab = synth.config2_table(9000 + 1000 * f, 4096, file=f, **SMALL)
        d = W.write_file(tab, synth.config2_spec(4096, 4096, "SNAPPY" if f % 2 else "UNCOMPRESSED", 1 + f % 2))
        datas.append(d)
        expects.append(R.read_file(d))
    outs = eng.read([to_dev(d) for d in datas])
    merged = []
    for c in range(8):
        parts = [e[c] for e in expects]
        valid = None if parts[0].valid is None else np.concatenate([p.valid for p in parts])
        if parts[0].ptype == "BYTE_ARRAY":
            offs = [parts[0].offsets]
            base = parts[0].offsets[-1]
            for p in parts[1:]:
                offs.append(p.offsets[1:] + base)
                base += p.offsets[-1]
            merged.append(ColumnResult(parts[0].name, "BYTE_ARRAY", None, valid, np.concatenate(offs),
                                       np.concatenate([p.chars for p in parts])))
        else:
            merged.append(ColumnResult(parts[0].name, parts[0].ptype, np.concatenate([p.values for p in parts]), valid))
    assert_columns_equal(outs, merged)


def test_edge_cases(eng):
    """All-null and all-valid OPTIONAL pages, a one-entry dictionary (bit
    width 0), DELTA with full-width random deltas and wrap-around extremes,
    one-row and single-page chunks."""
    n = 20_000
    rng = np.random.default_rng(1)
    i64 = np.iinfo(np.int64)
    i32 = np.iinfo(np.int32)
    cols = [
        synth.ColumnData("allnull", "INT64", np.zeros(n, np.int64), np.zeros(n, bool)),
        synth.ColumnData("allvalid", "INT32", rng.integers(-5, 5, n).astype(np.int32), np.ones(n, bool)),
        synth.ColumnData("onedict", "INT64", np.full(n, 77, np.int64)),
        synth.ColumnData("delta_rand64", "INT64", rng.integers(i64.min, i64.max, n, dtype=np.int64, endpoint=True)),
        synth.ColumnData("delta_rand32", "INT32", rng.integers(i32.min, i32.max, n, dtype=np.int64).astype(np.int32)),
        synth.ColumnData("delta_wrap", "INT64", np.tile(np.array([i64.min, i64.max, 0, -1], np.int64), n // 4)),
        synth.ColumnData("opt_dict", "DOUBLE", np.where(rng.random(n) < 0.5, rng.integers(0, 3, n) * 1.5, 0.0),
                         None),
        synth.ColumnData("opt_delta", "INT32", np.cumsum(rng.integers(0, 3, n)).astype(np.int32),
                         rng.random(n) > 0.3),
    ]
    cols[7].values[~cols[7].valid] = 0
    encs = ["PLAIN", "RLE_DICTIONARY", "RLE_DICTIONARY", "DELTA_BINARY_PACKED", "DELTA_BINARY_PACKED",
            "DELTA_BINARY_PACKED", "RLE_DICTIONARY", "DELTA_BINARY_PACKED"]
    tab = synth.Table(cols)
    for rg, page in ((n, 1 << 20), (5000, 1500), (1, 64)):
        spec = synth.TableSpec(rg, page, [synth.ColumnSpec(e) for e in encs])
        nt = synth.Table([synth.slice_column(c, 0, n if rg > 1 else 40) for c in cols])
        _roundtrip(eng, W.write_file(nt if rg == 1 else tab, spec))


@pytest.mark.parametrize("enc", ["RLE_DICTIONARY", "PLAIN"])
def test_string_lengths_and_nulls(eng, enc):
    """String columns whose rows cover every case of the chunk assembly:
    lengths 0-3 (spans under a word), 4-12, up to 80 bytes (past the source
    slots), nulls, and pools large and small; 64-row chunks end inside
    items and pages."""
    n = 50_003
    rng = np.random.default_rng(99)
    cols = []
    for name, k, lo, hi, null in (("tiny", 50, 0, 3, 0.0), ("short", 400, 4, 12, 0.0), ("wide", 3000, 0, 80, 0.0),
                                  ("opt_mid", 900, 5, 20, 0.3), ("opt_wide", 200, 1, 64, 0.05)):
        sd = synth.strings_uniform(rng, n, k=k, min_len=lo, max_len=hi)
        valid = None if null == 0.0 else rng.random(n) >= null
        cols.append(synth.ColumnData(name, "BYTE_ARRAY", sd, valid))
    tab = synth.Table(cols)
    for page in (1 << 20, 3000):
        spec = synth.TableSpec(20_000, page, [synth.ColumnSpec(enc) for _ in cols])
        _roundtrip(eng, W.write_file(tab, spec))
    spec = synth.TableSpec(n, 1 << 16, [synth.ColumnSpec(enc) for _ in cols])
    _roundtrip(eng, W.write_file(tab, spec), row_begin=777, row_count=40_001)


def test_string_dictionary_chains(eng):
    """Dictionary pages whose (length, bytes) chain is found per region in
    parallel: binary strings (bytes that read as small plausible lengths),
    strings longer than a region, many empty strings, and pools whose
    dictionary page spans dozens of regions; uncompressed and Snappy."""
    rng = np.random.default_rng(4242)
    n = 30_000

    def pool(lens, binary):
        offs = np.zeros(len(lens) + 1, np.int64)
        np.cumsum(lens, out=offs[1:])
        if binary:
            chars = rng.integers(0, 8, int(offs[-1])).astype(np.uint8)  # mostly bytes 0-7
        else:
            chars = rng.integers(65, 91, int(offs[-1])).astype(np.uint8)
        return offs, chars

    cols = []
    for name, lens, binary in (
            ("binary", rng.integers(0, 40, 6000), True),
            ("long", rng.integers(2000, 9000, 60), False),
            ("empties", np.where(rng.random(5000) < 0.5, 0, rng.integers(1, 12, 5000)), True),
            ("mixed", np.where(rng.random(8000) < 0.02, rng.integers(3000, 6000, 8000), rng.integers(0, 20, 8000)),
             True)):
        offs, chars = pool(np.asarray(lens, np.int64), binary)
        k = len(lens)
        idx = rng.integers(0, k, n).astype(np.int32)
        cols.append(synth.ColumnData(name, "BYTE_ARRAY", synth.StringData(offs, chars, idx)))
    tab = synth.Table(cols)
    for codec in ("UNCOMPRESSED", "SNAPPY"):
        spec = synth.TableSpec(n, 1 << 20, [synth.ColumnSpec("RLE_DICTIONARY", codec=codec) for _ in cols])
        _roundtrip(eng, W.write_file(tab, spec))


def test_config4_style_mixed_chunks(eng):
    draws = synth.config4_draws(n_files=3, chunks_per_file=4, rows_lo=500, rows_hi=40_000, page_lo=512,
                                page_hi=64 * 1024)
    for d in draws:
        col, cspec = synth.config4_column(d)
        data = W.write_file(synth.Table([col]), synth.TableSpec(rg_rows=15_000, page_bytes=d.page_bytes,
                                                                columns=[cspec]))
        _roundtrip(eng, data)


def test_delta_block_chains_across_regions(eng):
    """Single-page DELTA chunks long enough that the block chain spans many
    16 KB regions: constant deltas (zero-width miniblocks, 5-byte blocks),
    small random steps, runs that alternate between constant and noisy
    deltas, and full-width random values (1 KB blocks, where a region's
    lead-in holds about one block)."""
    n = 1 << 20
    rng = np.random.default_rng(3)
    i64 = np.iinfo(np.int64)
    cols = [
        synth.ColumnData("const_step", "INT64", np.arange(n, dtype=np.int64) * 3),
        synth.ColumnData("steps07", "INT64", np.cumsum(rng.integers(0, 8, n)).astype(np.int64)),
        synth.ColumnData("mixed32", "INT32", np.cumsum(np.where((np.arange(n) // 4096) % 2 == 0, 1,
                                                                rng.integers(-1000, 1000, n))).astype(np.int32)),
    ]
    spec = synth.TableSpec(n, 64 << 20, [synth.ColumnSpec("DELTA_BINARY_PACKED")] * 3)
    _roundtrip(eng, W.write_file(synth.Table(cols), spec))
    m = 1 << 16
    wide = [synth.ColumnData("rand64", "INT64", rng.integers(i64.min, i64.max, m, dtype=np.int64, endpoint=True)),
            synth.ColumnData("rand32", "INT32", rng.integers(-2**31, 2**31, m, dtype=np.int64).astype(np.int32))]
    spec = synth.TableSpec(m, 64 << 20, [synth.ColumnSpec("DELTA_BINARY_PACKED")] * 2)
    _roundtrip(eng, W.write_file(synth.Table(wide), spec))


@pytest.mark.parametrize("graph", [True, False])
def test_batch_of_heterogeneous_chunks(eng, graph):
    """Batched workload in miniature: single-column files of five kinds,
    grouped by schema into one index and one plan each, all plans run as one
    batch (one CUDA graph launch, or enqueued), launched twice; every column
    equals the oracle's reading of its files; then again under a non-default
    tuning (smaller work items, fewer branches, capped CTAs)."""
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.scan import alloc_outputs
    draws = synth.config4_draws(n_files=6, chunks_per_file=4, rows_lo=300, rows_hi=30_000, page_lo=512,
                                page_hi=32 * 1024)
    groups = {}
    for d in draws:
        col, cspec = synth.config4_column(d)
        data = W.write_file(synth.Table([col]), synth.TableSpec(rg_rows=7_000, page_bytes=d.page_bytes,
                                                                columns=[cspec]))
        groups.setdefault(d.kind, []).append(data)
    expected = {}
    for kind, datas in groups.items():
        parts = [R.read_file(d)[0] for d in datas]
        from oracle.reader import ColumnResult
        p0 = parts[0]
        valid = None if p0.valid is None else np.concatenate([p.valid for p in parts])
        if p0.ptype == "BYTE_ARRAY":
            offs, base = [np.zeros(1, np.int64)], 0
            for p in parts:
                offs.append(p.offsets[1:] + base)
                base += int(p.offsets[-1])
            expected[kind] = ColumnResult(p0.name, p0.ptype, None, valid, np.concatenate(offs),
                                          np.concatenate([p.chars for p in parts]))
        else:
            expected[kind] = ColumnResult(p0.name, p0.ptype, np.concatenate([p.values for p in parts]), valid)
    devs = {k: [to_dev(d) for d in v] for k, v in groups.items()}
    for tuning in (None, dict(item_rows=512, item_rows_opt=64, expand_ctas_per_sm=1, branches=2)):
        if tuning:
            N.pq_ctx_set_tuning(eng.ctx, **tuning)
        try:
            idxs, plans, outs, kinds = [], [], [], []
            for kind, files in devs.items():
                ix = eng.index(files)
                pl, sizes = eng.plan(ix)
                idxs.append(ix)
                plans.append(pl)
                outs.append(alloc_outputs(sizes))
                kinds.append(kind)
            b = N.pq_batch_create(eng.ctx, plans, [[o.desc() for o in oo] for oo in outs],
                                  N.PQ_SCAN_GRAPH if graph else 0)
            for _ in range(2):
                N.pq_batch_launch(eng.ctx, b)
                assert N.pq_batch_wait(b) == N.PQ_OK, N.pq_last_error(eng.ctx)
                for pl, oo, kind in zip(plans, outs, kinds):
                    st, chars = eng.wait(pl, len(oo))
                    assert st == N.PQ_OK
                    if oo[0].chars is not None:
                        oo[0].chars = oo[0].chars[:chars[0]]
                    assert_columns_equal(oo, [expected[kind]])
            N.pq_batch_free(b)
            for pl in plans:
                N.pq_free_plan(pl)
            for ix in idxs:
                N.pq_free_index(ix)
        finally:
            N.pq_ctx_set_tuning(eng.ctx)


def test_maximal_run_stretches(eng):
    """Dictionary-index streams made of stretches of maximal bit-packed runs
    (63 groups, header byte 127) broken by repeated runs at irregular gaps:
    a few runs apart, hundreds apart, and more than a walk batch (1024 runs)
    apart; bit widths 4, 12 and 20; one 8 MiB page per chunk, so a page
    holds thousands of runs; nullable and REQUIRED columns; the "mixed"
    policy adds bit-packed runs shorter than the maximum."""
    n = 1 << 21
    rng = np.random.default_rng(2026)

    def with_repeats(vals, mean_gap_runs):
        out = vals.copy()
        i = 0
        while True:
            i += int(rng.geometric(1.0 / (mean_gap_runs * 504))) // 8 * 8
            if i >= n - 64:
                break
            L = int(rng.integers(8, 40))
            out[i:i + L] = out[i]
            i += L
        return out

    cols = [
        synth.ColumnData("bw4_gap3", "INT32", with_repeats(rng.integers(0, 16, n).astype(np.int32), 3)),
        synth.ColumnData("bw12_gap300", "INT32", with_repeats(rng.integers(0, 4096, n).astype(np.int32), 300)),
        synth.ColumnData("bw20_gap5000", "INT64", with_repeats(rng.integers(0, 1 << 20, n).astype(np.int64), 5000)),
        synth.ColumnData("bw12_none", "INT32", rng.integers(0, 4096, n).astype(np.int32)),
    ]
    valid = rng.random(n) < 0.999
    cols.append(synth.ColumnData("opt_bw12", "INT32", np.where(valid, cols[1].values, 0).astype(np.int32), valid))
    for policy in ("default", "mixed"):
        cs = [synth.ColumnSpec("RLE_DICTIONARY") for _ in cols]
        for c in cs:
            c.hybrid_policy = policy
        data = W.write_file(synth.Table(cols), synth.TableSpec(n, 8 << 20, cs))
        _roundtrip(eng, data)
        _roundtrip(eng, data, row_begin=300_001, row_count=1_500_007)


def test_hybrid_run_chains_across_regions(eng):
    """Level and dictionary-index streams long enough to span many 4 KB run
    regions: nulls with probability 1/2 (short bit-packed runs), long null
    and non-null stretches (long repeated runs), a nullable dictionary column,
    indices of bit width 1 to 18, and a one-entry dictionary (bit width 0)."""
    n = 1 << 20
    rng = np.random.default_rng(7)
    stretch = (np.arange(n) // 5000) % 3 != 0
    coin = rng.random(n) < 0.5
    cols = [
        synth.ColumnData("opt_coin", "INT64", np.where(coin, rng.integers(-9, 9, n), 0).astype(np.int64), coin),
        synth.ColumnData("opt_stretch", "INT32", np.where(stretch, np.arange(n) % 1000, 0).astype(np.int32), stretch),
        synth.ColumnData("opt_dict", "INT32", np.where(coin, rng.integers(0, 300, n), 0).astype(np.int32), coin),
        synth.ColumnData("dict_bw18", "INT32", rng.integers(0, 1 << 18, n).astype(np.int32)),
        synth.ColumnData("dict_bw1", "INT64", rng.integers(0, 2, n).astype(np.int64)),
        synth.ColumnData("dict_one", "INT32", np.full(n, 42, np.int32)),
    ]
    encs = ["PLAIN", "PLAIN", "RLE_DICTIONARY", "RLE_DICTIONARY", "RLE_DICTIONARY", "RLE_DICTIONARY"]
    for policy in ("default", "mixed"):
        cs = [synth.ColumnSpec(e) for e in encs]
        for c in cs:
            c.hybrid_policy = policy
        spec = synth.TableSpec(n, 8 << 20, cs)
        _roundtrip(eng, W.write_file(synth.Table(cols), spec))
    # row ranges that start and end inside runs
    spec = synth.TableSpec(n, 8 << 20, [synth.ColumnSpec(e) for e in encs])
    data = W.write_file(synth.Table(cols), spec)
    _roundtrip(eng, data, row_begin=12_345, row_count=700_001)


def test_snappy_large_pages(eng):
    """Snappy pages far above the size at which a block of warps takes a page
    (hundreds of KB to MB, literals longer than the ring), with Snappy forced
    on every chunk; V1 and V2 pages."""
    tab = synth.config2_table(300_000, 300_000, **SMALL)
    for version in (1, 2):
        spec = synth.config2_spec(300_000, 4 << 20, "SNAPPY", version)
        for c in spec.columns:
            c.compress_threshold = -1.0
        _roundtrip(eng, W.write_file(tab, spec))


@pytest.mark.parametrize("enc", ["RLE_DICTIONARY", "PLAIN", "DELTA_LENGTH_BYTE_ARRAY"])
def test_strings_without_size_statistics(eng, enc):
    """BYTE_ARRAY chunks whose metadata carries no SizeStatistics (as older
    writers leave it out): the planner sizes the chars with a sizing scan;
    REQUIRED and OPTIONAL columns, several row groups, a row range, and a
    second column that does carry the statistics."""
    rng = np.random.default_rng(17)
    n = 30_000
    a = synth.strings_uniform(rng, n, k=500, min_len=0, max_len=40)
    b = synth.strings_uniform(rng, n, k=900, min_len=3, max_len=20)
    valid = rng.random(n) >= 0.2
    cols = [synth.ColumnData("s_req", "BYTE_ARRAY", a), synth.ColumnData("s_opt", "BYTE_ARRAY", b, valid),
            synth.ColumnData("s_stats", "BYTE_ARRAY", a)]
    specs = [synth.ColumnSpec(enc, size_statistics=False), synth.ColumnSpec(enc, size_statistics=False),
             synth.ColumnSpec(enc)]
    for version in (1, 2):
        for s in specs:
            s.page_version = version
        data = W.write_file(synth.Table(cols), synth.TableSpec(12_000, 8192, specs))
        assert R.parse_footer(data).raw is not None
        _roundtrip(eng, data)
        _roundtrip(eng, data, row_begin=5_555, row_count=17_000)


def test_large_offset_index(eng):
    """Chunks of thousands of small pages: their OffsetIndex is larger than
    the index kernel's shared-memory buffer and streams through it in
    windows.  The page table equals the oracle's walk and the scan the
    oracle's reading."""
    from paper_2602_17335_gb300 import native as N
    n = 200_000
    rng = np.random.default_rng(8)
    cols = [synth.ColumnData("a", "INT64", rng.integers(-10**12, 10**12, n).astype(np.int64)),
            synth.ColumnData("b", "INT32", rng.integers(0, 50, n).astype(np.int32))]
    spec = synth.TableSpec(n, 1024, [synth.ColumnSpec("PLAIN"), synth.ColumnSpec("RLE_DICTIONARY")])
    data = W.write_file(synth.Table(cols), spec)
    info = R.parse_footer(data)
    assert any(ch.offset_index[1] > 8192 for ch in info.chunks)
    idx = eng.index([to_dev(data)])
    assert N.pq_index_get_info(idx).used_offset_index == 1
    got = [(g.header_offset, g.page_type, g.num_values, g.first_row) for g in N.pq_index_copy_pages(idx)]
    exp = []
    for ch in info.chunks:
        row = 0
        for p in R.chunk_pages(data, ch):
            exp.append((p.offset, p.page_type, p.num_values, 0 if p.page_type == 2 else row))
            if p.page_type != 2:
                row += p.num_values
    assert got == exp
    N.pq_free_index(idx)
    _roundtrip(eng, data)


def _concat_results(a, b):
    """Rows of oracle ColumnResult a followed by those of b."""
    from oracle.reader import ColumnResult
    valid = None if a.valid is None else np.concatenate([a.valid, b.valid])
    if a.ptype == "BYTE_ARRAY":
        off = np.concatenate([a.offsets, b.offsets[1:] + a.offsets[-1]])
        return ColumnResult(a.name, a.ptype, None, valid, off, np.concatenate([a.chars, b.chars]))
    return ColumnResult(a.name, a.ptype, np.concatenate([a.values, b.values]), valid)


def test_snappy_split_pages(eng):
    """Snappy pages of several 64 KiB fragments from the native writer (framed
    as the reference compressor frames them: data pages of 1 MiB, dictionary
    pages of hundreds of KB), decompressed fragment by fragment; V1 and V2.
    The same table from the oracle writer (whole-page matches, no such
    framing) is read in the same scan, so that its large pages take the
    whole-page path next to the split ones."""
    from paper_2602_17335_gb300.tables import write_table
    tab = synth.config2_table(240_000, 120_000, string_pool_size=20_000, zipf_k=5000)
    for version in (1, 2):
        spec = synth.config2_spec(120_000, 1 << 20, "SNAPPY", version)
        for c in spec.columns:
            c.compress_threshold = -1.0
        native = bytes(write_table(tab, spec))
        _roundtrip(eng, native)
        oracle = W.write_file(tab, spec)
        expect = [_concat_results(a, b) for a, b in zip(R.read_file(native), R.read_file(oracle))]
        assert_columns_equal(eng.read([to_dev(native), to_dev(oracle)]), expect)
