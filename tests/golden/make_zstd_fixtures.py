"""Writes the Zstandard Parquet fixtures of tests/golden (run it where
pyarrow is installed: the fixtures carry libzstd-made pages to machines that
have no Zstandard library).

Inputs only: seeded synthetic tables from `synth`, compressed by libzstd
through pyarrow at two levels, V1 and V2 pages.  Expected values never come
from these files' writer: the tests decode them with the CPU oracle.

    python tests/golden/make_zstd_fixtures.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402

FIXTURES = {
    # name: (rows, row-group rows, page bytes, page version, level)
    "zstd_eight_column_v1.parquet": (6000, 2500, 8192, "1.0", 3),
    "zstd_eight_column_v2.parquet": (6000, 2500, 8192, "2.0", 19),
}


def arrow_table(tab):
    import pyarrow as pa
    cols = {}
    for c in tab.columns:
        if c.ptype == "BYTE_ARRAY":
            off, ch = c.values.materialize()
            arr = pa.array([bytes(ch[off[i]:off[i + 1]]) for i in range(len(off) - 1)], pa.binary(),
                           mask=None if c.valid is None else ~np.asarray(c.valid))
        else:
            arr = pa.array(np.asarray(c.values), mask=None if c.valid is None else ~np.asarray(c.valid))
        cols[c.name] = arr
    schema = pa.schema([pa.field(c.name, cols[c.name].type, nullable=c.valid is not None) for c in tab.columns])
    return pa.table(cols, schema=schema)


def write(name, rows, rg, page, version, level):
    import pyarrow.parquet as pq
    tab = synth.config2_table(rows, rg, string_pool_size=700, zipf_k=2000)
    t = arrow_table(tab)
    pq.write_table(t, os.path.join(HERE, name), compression="zstd", compression_level=level,
                   row_group_size=rg, data_page_size=page, data_page_version=version,
                   use_dictionary=["c1_dict_i32", "c4_zipf_i32", "c6_dict_str", "c7_card16_i32",
                                   "c8_card5_sorted_i32"],
                   column_encoding={"c2_delta_i64": "DELTA_BINARY_PACKED", "c3_plain_f64": "PLAIN",
                                    "c5_opt_i64": "PLAIN"},
                   write_page_index=True, write_statistics=False, store_schema=False)


if __name__ == "__main__":
    for name, args in FIXTURES.items():
        write(name, *args)
        print(name, os.path.getsize(os.path.join(HERE, name)))
