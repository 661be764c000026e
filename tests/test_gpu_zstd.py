"""Zstandard pages on the GPU (the codec list of the paper's Section 2),
bit for bit against the CPU oracle's reading of the same files.

* The two committed fixtures, written with libzstd from the seeded
  eight-column table (V1 and V2 pages): entropy-coded frames with Huffman
  literals (one and four streams), FSE-coded sequences and repeat offsets.
* Files from the engine's own writer with Zstandard pages (V1 and V2).
* A scan over files of three codecs at once (Zstandard, Snappy, none), so
  that the Snappy and Zstandard kernels share job lists."""
import os

import pytest

import synth
from oracle import reader as R
from oracle import writer as W

from gpu_util import assert_columns_equal, engine, to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SMALL = dict(string_pool_size=700, zipf_k=2000)


@pytest.fixture(scope="module")
def eng():
    e = engine()
    yield e
    e.close()


@pytest.mark.parametrize("name", ["zstd_eight_column_v1.parquet", "zstd_eight_column_v2.parquet"])
def test_libzstd_fixtures(eng, name):
    data = open(os.path.join(GOLDEN, name), "rb").read()
    expect = R.read_file(data)
    outs = eng.read([to_dev(data)])
    assert_columns_equal(outs, expect)
    # row ranges and column subsets over the same pages
    outs = eng.read([to_dev(data)], columns=[5, 1], row_begin=1234, row_count=4000)
    from gpu_util import slice_result
    assert_columns_equal(outs, [slice_result(expect[c], 1234, 5234) for c in (5, 1)])


@pytest.mark.parametrize("version", [1, 2])
def test_native_writer_zstd(eng, version):
    from paper_2602_17335_gb300.tables import write_table
    tab = synth.config2_table(30_000, 12_000, **SMALL)
    spec = synth.config2_spec(12_000, 16 * 1024, "ZSTD", version)
    for c in spec.columns:
        c.compress_threshold = -1.0
    data = write_table(tab, spec)
    expect = R.read_file(data.tobytes())
    assert_columns_equal(eng.read([to_dev(data.tobytes())]), expect)


def test_three_codecs_in_one_scan(eng):
    from oracle.reader import ColumnResult
    import numpy as np
    from paper_2602_17335_gb300.tables import write_table
    datas = []
    for f, codec in enumerate(("ZSTD", "SNAPPY", "UNCOMPRESSED")):
        tab = synth.config2_table(9000 + 1000 * f, 4096, file=f, **SMALL)
        spec = synth.config2_spec(4096, 4096, codec, 1 + f % 2)
        for c in spec.columns:
            c.compress_threshold = -1.0
        datas.append(write_table(tab, spec).tobytes())
    expects = [R.read_file(d) for d in datas]
    outs = eng.read([to_dev(d) for d in datas])
    merged = []
    for c in range(8):
        parts = [e[c] for e in expects]
        valid = None if parts[0].valid is None else np.concatenate([p.valid for p in parts])
        if parts[0].ptype == "BYTE_ARRAY":
            offs, base = [parts[0].offsets], parts[0].offsets[-1]
            for p in parts[1:]:
                offs.append(p.offsets[1:] + base)
                base += p.offsets[-1]
            merged.append(ColumnResult(parts[0].name, "BYTE_ARRAY", None, valid, np.concatenate(offs),
                                       np.concatenate([p.chars for p in parts])))
        else:
            merged.append(ColumnResult(parts[0].name, parts[0].ptype, np.concatenate([p.values for p in parts]),
                                       valid))
    assert_columns_equal(outs, merged)
