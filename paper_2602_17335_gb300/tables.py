"""Writes seeded synthetic tables (``synth``) to Parquet with the engine's
native writer (``pq_write_table``) — how benchmarks stage their input files."""
from __future__ import annotations

import ctypes as C

import numpy as np

import synth

from . import native as N

_TYPE = {"INT32": N.PQ_TYPE_INT32, "INT64": N.PQ_TYPE_INT64, "DOUBLE": N.PQ_TYPE_DOUBLE,
         "BYTE_ARRAY": N.PQ_TYPE_BYTE_ARRAY}
_ENC = {"PLAIN": 0, "RLE_DICTIONARY": 8, "DELTA_BINARY_PACKED": 5, "DELTA_LENGTH_BYTE_ARRAY": 6,
        "DELTA_BYTE_ARRAY": 7, "BYTE_STREAM_SPLIT": 9, "AUTO": -1}
_CODEC = {"UNCOMPRESSED": 0, "SNAPPY": 1, "ZSTD": 6}


def write_table(table: synth.Table, spec: synth.TableSpec, n_threads: int = 0) -> np.ndarray:
    cols, keep = [], []
    for col, cs in zip(table.columns, spec.columns):
        w = N.pq_write_column()
        name = col.name.encode()
        keep.append(name)
        w.name = name
        w.type = _TYPE[col.ptype]
        w.encoding = _ENC[cs.encoding]
        w.codec = _CODEC[cs.codec]
        w.page_version = cs.page_version
        w.compress_threshold = -1.0 if cs.compress_threshold is None else cs.compress_threshold
        if col.ptype == "BYTE_ARRAY":
            off, chars = col.values.materialize()
            off = np.ascontiguousarray(off, dtype=np.int64)
            chars = np.ascontiguousarray(chars, dtype=np.uint8)
            keep += [off, chars]
            w.values = off.ctypes.data
            w.chars = chars.ctypes.data if chars.size else None
        else:
            v = np.ascontiguousarray(col.values)
            keep.append(v)
            w.values = v.ctypes.data
        if col.valid is not None:
            m = np.ascontiguousarray(col.valid, dtype=np.uint8)
            keep.append(m)
            w.valid = m.ctypes.data
        cols.append(w)
    return N.pq_write_table(cols, table.n_rows, spec.rg_rows, spec.page_bytes, spec.offset_index, n_threads)
