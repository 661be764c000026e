"""Seeded synthetic inputs for the Parquet scan engine and its CPU oracle.

This module only draws column data and names table layouts.  It holds none
of the format arithmetic (no encoding, no decoding): both the CPU oracle and
the product writer consume what it returns.

The tables stand in for the TPC-H SF300 ``lineitem`` files the paper scans
(Section 3, setup paragraph), which are not available here.  Column
distributions follow the eight-column synthetic table of the scan workloads:

  c1  INT32 uniform in [0, 2^20)                     -> dictionary encoded
  c2  INT64 sorted keys k0 = 1, k_i = k_{i-1} + U{0..7} -> DELTA_BINARY_PACKED
  c3  DOUBLE standard normal                         -> PLAIN
  c4  INT32 Zipf(1.1) over 10^4 distinct values      -> dictionary encoded
  c5  OPTIONAL INT64 uniform over int64, 10% nulls   -> PLAIN + def levels
  c6  BYTE_ARRAY, 10^4 random [A-Za-z0-9] strings of length U[8,32],
      rows uniform over them                         -> dictionary encoded
  c7  INT32 uniform over 16 distinct values          -> dictionary encoded
  c8  INT32 over 5 distinct values, sorted inside each row group -> dictionary

Every generator takes an explicit ``numpy.random.Generator``; ``rng_for``
derives one per (config, column, file) from the master seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np

MASTER_SEED = 2602_17335

# Parquet physical type names used across the repository.
INT32, INT64, DOUBLE, BYTE_ARRAY = "INT32", "INT64", "DOUBLE", "BYTE_ARRAY"
FIXED_WIDTH = {INT32: 4, INT64: 8, DOUBLE: 8}

# Writer-side knobs (names of encodings/codecs; no arithmetic here).
PLAIN, RLE_DICTIONARY, DELTA_BINARY_PACKED = "PLAIN", "RLE_DICTIONARY", "DELTA_BINARY_PACKED"
DELTA_LENGTH_BYTE_ARRAY, DELTA_BYTE_ARRAY = "DELTA_LENGTH_BYTE_ARRAY", "DELTA_BYTE_ARRAY"
BYTE_STREAM_SPLIT = "BYTE_STREAM_SPLIT"
UNCOMPRESSED, SNAPPY, ZSTD = "UNCOMPRESSED", "SNAPPY", "ZSTD"

KiB = 1 << 10
MiB = 1 << 20


def rng_for(config: int, column: int, file: int = 0, seed: int = MASTER_SEED) -> np.random.Generator:
    """A generator per (config, column, file), derived from the master seed."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, config, column, file])))


# --------------------------------------------------------------------------
# Column data
# --------------------------------------------------------------------------

@dataclass
class StringData:
    """A BYTE_ARRAY column given as a small pool of distinct strings plus a
    row -> pool index.  ``materialize`` produces the row values as (int64
    offsets of length n+1, uint8 chars) for a row range."""
    pool_offsets: np.ndarray  # int64, len k+1
    pool_chars: np.ndarray    # uint8
    row_index: np.ndarray     # int32, len n

    def __len__(self) -> int:
        return int(self.row_index.shape[0])

    def materialize(self, lo: int = 0, hi: Optional[int] = None):
        hi = len(self) if hi is None else hi
        idx = self.row_index[lo:hi]
        lens = (self.pool_offsets[1:] - self.pool_offsets[:-1])[idx]
        offsets = np.zeros(idx.shape[0] + 1, dtype=np.int64)
        np.cumsum(lens, out=offsets[1:])
        total = int(offsets[-1])
        chars = np.empty(total, dtype=np.uint8)
        step = 1 << 20
        for a in range(0, idx.shape[0], step):
            b = min(idx.shape[0], a + step)
            l = lens[a:b]
            src0 = np.repeat(self.pool_offsets[idx[a:b]], l)
            within = np.arange(int(l.sum()), dtype=np.int64) - np.repeat(offsets[a:b] - offsets[a], l)
            chars[offsets[a]:offsets[b]] = self.pool_chars[src0 + within]
        return offsets, chars


@dataclass
class ColumnData:
    """One column of a synthetic table.

    ``values``: fixed-width numpy array of n rows (null slots hold 0), or a
    ``StringData`` for BYTE_ARRAY.  ``valid``: bool per row, or None for a
    REQUIRED column."""
    name: str
    ptype: str
    values: object
    valid: Optional[np.ndarray] = None

    @property
    def n_rows(self) -> int:
        return len(self.values)

    @property
    def required(self) -> bool:
        return self.valid is None


def uniform_int32(rng, n, lo, hi):
    return rng.integers(lo, hi, size=n, dtype=np.int64).astype(np.int32)


def sorted_keys_int64(rng, n, start=1, max_step=7):
    steps = rng.integers(0, max_step + 1, size=n, dtype=np.int64)
    steps[0] = 0
    return (np.cumsum(steps) + start).astype(np.int64)


def normal_f64(rng, n):
    return rng.standard_normal(n)


def zipf_int32(rng, n, s=1.1, k=10_000):
    """Ranks 1..k with P(rank) proportional to rank^-s by inverse CDF; each rank
    maps through a seeded permutation onto k distinct uniform int32 values."""
    p = np.arange(1, k + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    ranks = np.searchsorted(cdf, rng.random(n), side="right")
    ranks = np.minimum(ranks, k - 1)
    values = rng.choice(np.iinfo(np.int32).max, size=k, replace=False).astype(np.int64)
    values -= 1 << 30  # spread over negative and positive int32
    values = rng.permutation(values).astype(np.int32)
    return values[ranks]


def uniform_int64_full(rng, n):
    return rng.integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, size=n, dtype=np.int64, endpoint=True)


def bernoulli_valid(rng, n, null_frac=0.1):
    return rng.random(n) >= null_frac


def string_pool(rng, k=10_000, min_len=8, max_len=32):
    alphabet = np.frombuffer(b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789", dtype=np.uint8)
    lens = rng.integers(min_len, max_len + 1, size=k, dtype=np.int64)
    offsets = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    chars = alphabet[rng.integers(0, alphabet.shape[0], size=int(offsets[-1]))]
    return offsets, chars


def strings_uniform(rng, n, k=10_000, min_len=8, max_len=32):
    off, ch = string_pool(rng, k, min_len, max_len)
    idx = rng.integers(0, k, size=n, dtype=np.int64).astype(np.int32)
    return StringData(off, ch, idx)


def strings_sorted(rng, n, rg_rows, k=4096, stems=64):
    """Rows sorted inside each row group over a pool of ``k`` strings that
    share prefixes: each is one of ``stems`` random stems (length U[4,12])
    plus a random tail (length U[0,20]), all over [A-Za-z0-9]."""
    alphabet = np.frombuffer(b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789", dtype=np.uint8)
    stem_len = rng.integers(4, 13, size=stems)
    stem = [bytes(alphabet[rng.integers(0, alphabet.shape[0], size=int(m))]) for m in stem_len]
    pool = sorted(set(stem[int(rng.integers(0, stems))]
                      + bytes(alphabet[rng.integers(0, alphabet.shape[0], size=int(rng.integers(0, 21)))])
                      for _ in range(k)))
    lens = np.array([len(x) for x in pool], dtype=np.int64)
    offsets = np.zeros(len(pool) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    chars = np.frombuffer(b"".join(pool), dtype=np.uint8).copy()
    idx = rng.integers(0, len(pool), size=n, dtype=np.int64).astype(np.int32)
    for a in range(0, n, rg_rows):
        idx[a:a + rg_rows].sort()
    return StringData(offsets, chars, idx)


def lowcard_int32(rng, n, card=16):
    pool = rng.choice(1 << 20, size=card, replace=False).astype(np.int32)
    return pool[rng.integers(0, card, size=n)]


def sorted_lowcard_int32(rng, n, card, rg_rows):
    pool = np.sort(rng.choice(1 << 20, size=card, replace=False).astype(np.int32))
    out = pool[rng.integers(0, card, size=n)]
    for a in range(0, n, rg_rows):
        out[a:a + rg_rows].sort()
    return out


# --------------------------------------------------------------------------
# Writer layout specifications (knob names only)
# --------------------------------------------------------------------------

@dataclass
class ColumnSpec:
    # PLAIN | RLE_DICTIONARY | DELTA_BINARY_PACKED | BYTE_STREAM_SPLIT |
    # DELTA_LENGTH_BYTE_ARRAY | DELTA_BYTE_ARRAY | AUTO (per chunk, the
    # smallest valid encoding of the column's type)
    encoding: str = PLAIN
    codec: str = UNCOMPRESSED        # UNCOMPRESSED | SNAPPY | ZSTD (oracle writer: stored frames)
    page_version: int = 1            # 1 = DATA_PAGE, 2 = DATA_PAGE_V2
    # hybrid run policy for the writer: "default", "rle", "packed", "mixed"
    hybrid_policy: str = "default"
    # compress a chunk only when it shrinks by more than this fraction
    # (None: always keep the codec's output)
    compress_threshold: Optional[float] = None
    # BYTE_ARRAY: write the chunk's SizeStatistics (unencoded byte total);
    # older writers leave it out
    size_statistics: bool = True


@dataclass
class TableSpec:
    rg_rows: int
    page_bytes: int
    columns: List[ColumnSpec]
    offset_index: bool = True
    seed: int = 0  # only for randomised writer policies ("mixed")


@dataclass
class Table:
    columns: List[ColumnData]

    @property
    def n_rows(self) -> int:
        return self.columns[0].n_rows


# --------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------

def config1_table(n_rows: int = 1 << 20, seed: int = MASTER_SEED) -> Table:
    """Single REQUIRED INT32 column, uniform in [0, 1024), dictionary encoded."""
    rng = rng_for(1, 0, 0, seed)
    return Table([ColumnData("c1", INT32, uniform_int32(rng, n_rows, 0, 1024))])


def config1_spec(page_bytes: int = MiB, n_rows: int = 1 << 20) -> TableSpec:
    return TableSpec(rg_rows=n_rows, page_bytes=page_bytes, columns=[ColumnSpec(RLE_DICTIONARY)])


def config2_table(n_rows: int, rg_rows: int, seed: int = MASTER_SEED, file: int = 0,
                  string_pool_size: int = 10_000, zipf_k: int = 10_000) -> Table:
    """The eight-column table (see module docstring)."""
    r = lambda col: rng_for(2, col, file, seed)
    c5_valid = bernoulli_valid(r(50), n_rows, 0.1)
    c5 = uniform_int64_full(r(5), n_rows)
    c5[~c5_valid] = 0
    return Table([
        ColumnData("c1_dict_i32", INT32, uniform_int32(r(1), n_rows, 0, 1 << 20)),
        ColumnData("c2_delta_i64", INT64, sorted_keys_int64(r(2), n_rows)),
        ColumnData("c3_plain_f64", DOUBLE, normal_f64(r(3), n_rows)),
        ColumnData("c4_zipf_i32", INT32, zipf_int32(r(4), n_rows, 1.1, zipf_k)),
        ColumnData("c5_opt_i64", INT64, c5, c5_valid),
        ColumnData("c6_dict_str", BYTE_ARRAY, strings_uniform(r(6), n_rows, string_pool_size)),
        ColumnData("c7_card16_i32", INT32, lowcard_int32(r(7), n_rows, 16)),
        ColumnData("c8_card5_sorted_i32", INT32, sorted_lowcard_int32(r(8), n_rows, 5, rg_rows)),
    ])


def config2_spec(rg_rows: int, page_bytes: int, codec: str = UNCOMPRESSED,
                 page_version: int = 1, offset_index: bool = True) -> TableSpec:
    encs = [RLE_DICTIONARY, DELTA_BINARY_PACKED, PLAIN, RLE_DICTIONARY, PLAIN,
            RLE_DICTIONARY, RLE_DICTIONARY, RLE_DICTIONARY]
    return TableSpec(rg_rows=rg_rows, page_bytes=page_bytes,
                     columns=[ColumnSpec(e, codec, page_version) for e in encs],
                     offset_index=offset_index)


def v2_encodings_table(n_rows: int, rg_rows: int, seed: int = MASTER_SEED, file: int = 0) -> Table:
    """Six columns for the other V2 encodings of the paper's Insight 3:

      e1  DOUBLE standard normal                          -> BYTE_STREAM_SPLIT
      e2  INT32 Zipf(1.1) over 10^4 distinct values       -> BYTE_STREAM_SPLIT
      e3  OPTIONAL INT64 uniform over int64, 10% nulls    -> BYTE_STREAM_SPLIT
      e4  BYTE_ARRAY, 10^4 random strings, rows uniform   -> DELTA_LENGTH_BYTE_ARRAY
      e5  BYTE_ARRAY sorted in each row group, shared stems -> DELTA_BYTE_ARRAY
      e6  OPTIONAL BYTE_ARRAY as e4, 10% nulls            -> DELTA_BYTE_ARRAY
    """
    r = lambda col: rng_for(6, col, file, seed)
    e3_valid = bernoulli_valid(r(30), n_rows, 0.1)
    e3 = uniform_int64_full(r(3), n_rows)
    e3[~e3_valid] = 0
    return Table([
        ColumnData("e1_bss_f64", DOUBLE, normal_f64(r(1), n_rows)),
        ColumnData("e2_bss_i32", INT32, zipf_int32(r(2), n_rows, 1.1, 10_000)),
        ColumnData("e3_bss_opt_i64", INT64, e3, e3_valid),
        ColumnData("e4_dlba_str", BYTE_ARRAY, strings_uniform(r(4), n_rows, 10_000)),
        ColumnData("e5_dba_sorted_str", BYTE_ARRAY, strings_sorted(r(5), n_rows, rg_rows)),
        ColumnData("e6_dba_opt_str", BYTE_ARRAY, strings_uniform(r(6), n_rows, 10_000),
                   bernoulli_valid(r(60), n_rows, 0.1)),
    ])


V2_ENCODINGS = (BYTE_STREAM_SPLIT, BYTE_STREAM_SPLIT, BYTE_STREAM_SPLIT, DELTA_LENGTH_BYTE_ARRAY,
                DELTA_BYTE_ARRAY, DELTA_BYTE_ARRAY)


def v2_encodings_spec(rg_rows: int, page_bytes: int, codec: str = UNCOMPRESSED,
                      page_version: int = 2, offset_index: bool = True) -> TableSpec:
    return TableSpec(rg_rows=rg_rows, page_bytes=page_bytes,
                     columns=[ColumnSpec(e, codec, page_version) for e in V2_ENCODINGS],
                     offset_index=offset_index)


# Layout sweep of the eight-column table: row-group rows x page bytes.
CONFIG2_RG_ROWS = (1 << 20, 1 << 23, 1 << 26)
CONFIG2_PAGE_BYTES = (8 * KiB, 64 * KiB, MiB, 8 * MiB)


def config3_spec(page_bytes: int, rg_rows: int = 1 << 23) -> TableSpec:
    """The eight-column table with every chunk Snappy compressed (forced)."""
    return config2_spec(rg_rows, page_bytes, codec=SNAPPY)


# Batched workload: many uneven chunks from many files.
CONFIG4_KINDS = ("dict_i32", "dict_str", "plain_f64", "delta_i64", "opt_plain_i64")


@dataclass
class ChunkDraw:
    file: int
    index: int
    kind: str
    n_rows: int
    page_bytes: int
    snappy: bool
    page_version: int


def config4_draws(n_files: int = 256, chunks_per_file: int = 16, rows_lo: float = 1e4,
                  rows_hi: float = 1e7, page_lo: int = 4 * KiB, page_hi: int = 2 * MiB,
                  seed: int = MASTER_SEED) -> List[ChunkDraw]:
    """Per-chunk draws of the batched workload: rows and page bytes
    log-uniform, kind uniform over CONFIG4_KINDS, Snappy and page version
    each with probability 1/2."""
    rng = rng_for(4, 0, 0, seed)
    out = []
    for f in range(n_files):
        for c in range(chunks_per_file):
            rows = int(round(np.exp(rng.uniform(np.log(rows_lo), np.log(rows_hi)))))
            page = int(round(np.exp(rng.uniform(np.log(page_lo), np.log(page_hi)))))
            out.append(ChunkDraw(f, c, CONFIG4_KINDS[int(rng.integers(0, len(CONFIG4_KINDS)))], rows, page,
                                 bool(rng.integers(0, 2)), 1 + int(rng.integers(0, 2))))
    return out


def config4_column(draw: ChunkDraw, seed: int = MASTER_SEED):
    """(ColumnData, ColumnSpec) for one draw of the batched workload."""
    rng = rng_for(4, 1 + draw.index, 1 + draw.file, seed)
    n = draw.n_rows
    codec = SNAPPY if draw.snappy else UNCOMPRESSED
    if draw.kind == "dict_i32":
        col, enc = ColumnData("dict_i32", INT32, uniform_int32(rng, n, 0, 1 << 16)), RLE_DICTIONARY
    elif draw.kind == "dict_str":
        col, enc = ColumnData("dict_str", BYTE_ARRAY, strings_uniform(rng, n, 1000)), RLE_DICTIONARY
    elif draw.kind == "plain_f64":
        col, enc = ColumnData("plain_f64", DOUBLE, normal_f64(rng, n)), PLAIN
    elif draw.kind == "delta_i64":
        col, enc = ColumnData("delta_i64", INT64, sorted_keys_int64(rng, n)), DELTA_BINARY_PACKED
    else:
        valid = bernoulli_valid(rng, n, 0.1)
        v = uniform_int64_full(rng, n)
        v[~valid] = 0
        col, enc = ColumnData("opt_plain_i64", INT64, v, valid), PLAIN
    return col, ColumnSpec(enc, codec, draw.page_version)


def slice_column(col: ColumnData, lo: int, hi: int) -> ColumnData:
    """Rows [lo, hi) of a column (used by writers to cut row groups)."""
    v = col.values
    if isinstance(v, StringData):
        v = StringData(v.pool_offsets, v.pool_chars, v.row_index[lo:hi])
    else:
        v = v[lo:hi]
    return replace(col, values=v, valid=None if col.valid is None else col.valid[lo:hi])


def as_fixed(col: ColumnData) -> np.ndarray:
    """Row values of a fixed-width column as a numpy array."""
    assert col.ptype in FIXED_WIDTH
    return np.asarray(col.values)
