"""Parquet writer for the oracle (test infrastructure only).

Writes a flat table into a Parquet file following the paper's Section 2
hierarchy (file -> row groups -> one column chunk per column -> pages) with
the knobs its Section 3 varies: page size, row-group size, encoding per
chunk (V1 PLAIN / dictionary, the V2 set DELTA_BINARY_PACKED,
DELTA_LENGTH_BYTE_ARRAY, DELTA_BYTE_ARRAY and BYTE_STREAM_SPLIT, V1 or V2
data pages)
and per-chunk compression, optionally kept only when it shrinks the chunk by
more than a threshold ("No Unnecessary Compression", 10% in the paper).

Layout rules (deterministic, so that an independent writer can reproduce
them byte for byte on uncompressed data):

* row group k holds rows [k * rg_rows, (k+1) * rg_rows);
* a dictionary chunk starts with one dictionary page (PLAIN entries in order
  of first appearance), followed by its data pages;
* rows per data page, with b = bits per row:
  - fixed-width PLAIN: b = 8 * width (+1 when OPTIONAL);
  - dictionary indices: b = max(index bit width, 1) (+1 when OPTIONAL);
  - rows = max(8, floor(page_bytes * 8 / b) rounded down to a multiple of 8);
  - REQUIRED DELTA_BINARY_PACKED: 1 + 128 k values, k >= 1 the largest count
    of whole 128-value blocks whose encoded stream still fits page_bytes;
    OPTIONAL DELTA uses the fixed-width rule;
  - BYTE_STREAM_SPLIT: as fixed-width PLAIN;
  - BYTE_ARRAY (PLAIN, DELTA_LENGTH_BYTE_ARRAY, DELTA_BYTE_ARRAY): rows are
    added while the page has < 8 rows or the PLAIN-encoded bytes (4 + length
    per non-null value) still fit;
  the last page of a chunk takes the remaining rows;
* hybrid runs follow the chosen policy (``default`` unless the spec says
  otherwise); V1 definition levels carry a 4-byte length prefix;
* V1 pages compress levels and values together, V2 pages compress values
  only; the dictionary page body is compressed with the chunk's codec;
* encoding "AUTO": each chunk is written with the valid encoding of its type
  whose uncompressed chunk is smallest (``CANDIDATES`` order breaks ties);
* an OffsetIndex per chunk (data pages only, first_row_index relative to the
  row group) is written after the last row group when requested.
"""
from __future__ import annotations

import copy
from dataclasses import replace

import numpy as np

from synth import FIXED_WIDTH, ColumnSpec, StringData, Table, TableSpec, slice_column

from . import byte_stream_split as _bss
from . import delta as _delta
from . import delta_strings as _dstr
from . import hybrid as _hybrid
from . import plain as _plain
from . import snappy as _snappy
from . import thrift as T
from . import zstd as _zstd
from .parquet_meta import (CODEC_ID, DATA_PAGE, DATA_PAGE_V2, DICTIONARY_PAGE, ENCODING_ID,
                           OPTIONAL, PLAIN, REQUIRED, RLE, SNAPPY, TYPE_ID, UNCOMPRESSED, ZSTD)

CREATED_BY = "pq-oracle"


def _row_values(col):
    """Non-null values of a column slice as a Python list (fixed width: numpy
    scalars; BYTE_ARRAY: bytes) and the per-row validity (or None)."""
    if isinstance(col.values, StringData):
        off, chars = col.values.materialize()
        rows = [bytes(chars[off[i]:off[i + 1]]) for i in range(len(off) - 1)]
    else:
        rows = np.asarray(col.values)
    if col.valid is None:
        return rows, None
    valid = np.asarray(col.valid, dtype=bool)
    if isinstance(rows, list):
        return [r for r, v in zip(rows, valid) if v], valid
    return rows[valid], valid


def _dictionary(values, ptype):
    """(entries in order of first appearance, index per value)."""
    if ptype == "BYTE_ARRAY":
        pos, entries, idx = {}, [], []
        for v in values:
            if v not in pos:
                pos[v] = len(entries)
                entries.append(v)
            idx.append(pos[v])
        return entries, np.array(idx, dtype=np.uint64)
    arr = np.asarray(values)
    keys = arr.view(np.int64) if ptype == "DOUBLE" else arr.astype(np.int64)
    if keys.size == 0:
        return arr[:0], np.zeros(0, dtype=np.uint64)
    uniq, first, inverse = np.unique(keys, return_index=True, return_inverse=True)
    order = np.argsort(first, kind="stable")
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    return arr[first[order]], rank[inverse].astype(np.uint64)


def _rows_fixed_rule(page_bytes, bits_per_row):
    return max(8, (page_bytes * 8 // bits_per_row) // 8 * 8)


def _delta_page_values(vals, a, bits, page_bytes):
    """Values in the DELTA page starting at value ``a``: 1 + 128 k, the
    largest k >= 1 whose encoded stream fits page_bytes; a shorter tail is
    taken whole when it fits."""
    n = len(vals)
    rem = n - a
    if rem <= 129:
        return rem
    deltas = [_delta.wrap(vals[i] - vals[i - 1], bits) for i in range(a + 1, n)]

    def size(count):
        blocks = sum(len(_delta.encode_block(deltas[j:min(j + 128, count - 1)], bits))
                     for j in range(0, count - 1, 128))
        return len(_delta.encode_header(count, vals[a], bits)) + blocks

    k = 1
    body = len(_delta.encode_block(deltas[0:128], bits))
    while 1 + 128 * (k + 1) <= rem:
        nxt = body + len(_delta.encode_block(deltas[128 * k:128 * (k + 1)], bits))
        if len(_delta.encode_header(1 + 128 * (k + 1), vals[a], bits)) + nxt > page_bytes:
            return 1 + 128 * k
        body = nxt
        k += 1
    if size(rem) <= page_bytes:
        return rem
    return 1 + 128 * k


def _page_row_counts(ptype, encoding, n_rows, valid, vals_all, page_bytes, bw):
    optional = valid is not None
    counts = []
    if ptype == "BYTE_ARRAY" and encoding in ("PLAIN", "DELTA_LENGTH_BYTE_ARRAY", "DELTA_BYTE_ARRAY"):
        # vals_all holds the row values with None for nulls
        r = 0
        while r < n_rows:
            used, rows = 0, 0
            while r + rows < n_rows:
                v = vals_all[r + rows]
                cost = 0 if v is None else 4 + len(v)
                if rows >= 8 and used + cost > page_bytes:
                    break
                used += cost
                rows += 1
            counts.append(rows)
            r += rows
        return counts
    if encoding == "DELTA_BINARY_PACKED" and not optional:
        bits = 32 if ptype == "INT32" else 64
        r = 0
        while r < n_rows:
            c = _delta_page_values(vals_all, r, bits, page_bytes)
            counts.append(c)
            r += c
        return counts
    if encoding == "RLE_DICTIONARY":
        bits_per_row = max(bw, 1) + (1 if optional else 0)
    else:
        width = FIXED_WIDTH[ptype]
        bits_per_row = 8 * width + (1 if optional else 0)
    per = _rows_fixed_rule(page_bytes, bits_per_row)
    r = 0
    while r < n_rows:
        c = min(per, n_rows - r)
        counts.append(c)
        r += c
    return counts


def _levels_v1(levels, policy, rng):
    body = _hybrid.encode(levels, 1, policy, rng)
    return len(body).to_bytes(4, "little") + body


def _page_header(ptype_page, uncompressed, compressed, sub_fid, sub_fields):
    return T.encode_struct([
        (1, T.I32, ptype_page),
        (2, T.I32, uncompressed),
        (3, T.I32, compressed),
        (sub_fid, T.STRUCT, sub_fields),
    ])


def _compress(codec, data):
    if codec == SNAPPY:
        return _snappy.compress(data)
    if codec == ZSTD:
        return _zstd.compress_stored(data)
    return bytes(data)


# Valid encodings per physical type, in the order a tie is broken (the
# paper's Section 3, "Encoding Flexibility": every valid encoding of the
# type is tried per chunk and the smallest one is kept).
CANDIDATES = {"INT32": ("PLAIN", "RLE_DICTIONARY", "DELTA_BINARY_PACKED", "BYTE_STREAM_SPLIT"),
              "INT64": ("PLAIN", "RLE_DICTIONARY", "DELTA_BINARY_PACKED", "BYTE_STREAM_SPLIT"),
              "DOUBLE": ("PLAIN", "RLE_DICTIONARY", "BYTE_STREAM_SPLIT"),
              "BYTE_ARRAY": ("PLAIN", "RLE_DICTIONARY", "DELTA_LENGTH_BYTE_ARRAY", "DELTA_BYTE_ARRAY")}


def choose_encoding(col, cspec: ColumnSpec, page_bytes: int, rng=None):
    """The candidate whose uncompressed chunk (headers + page bodies) is
    smallest; ties go to the earlier candidate."""
    best, best_size = None, None
    for enc in CANDIDATES[col.ptype]:
        trial = replace(cspec, encoding=enc, codec="UNCOMPRESSED", compress_threshold=None)
        _, meta, _, _ = write_chunk(col, trial, page_bytes, 0, copy.deepcopy(rng))
        size = dict((f, v) for f, _, v in meta)[6]
        if best is None or size < best_size:
            best, best_size = enc, size
    return best


def write_chunk(col, cspec: ColumnSpec, page_bytes: int, base: int, rng=None):
    """Encodes one column chunk.  Returns (bytes, ColumnMetaData fields list,
    page locations, codec actually used).  Encoding "AUTO" writes the chunk
    with ``choose_encoding``'s pick."""
    if cspec.encoding == "AUTO":
        cspec = replace(cspec, encoding=choose_encoding(col, cspec, page_bytes, rng))
    ptype = col.ptype
    enc_name = cspec.encoding
    codec = CODEC_ID[cspec.codec]
    optional = col.valid is not None
    nonnull, valid = _row_values(col)
    n_rows = col.n_rows
    if ptype == "BYTE_ARRAY":
        # row view with None for nulls (page cutting needs it)
        it = iter(nonnull)
        rows_view = [next(it) if (valid is None or valid[i]) else None for i in range(n_rows)]
    else:
        rows_view = np.asarray(col.values)
    policy = cspec.hybrid_policy

    dict_entries, dict_idx, bw = None, None, 0
    if enc_name == "RLE_DICTIONARY":
        dict_entries, dict_idx = _dictionary(nonnull, ptype)
        bw = _hybrid.bit_width_for(max(len(dict_entries) - 1, 0))
    elif enc_name == "DELTA_BINARY_PACKED" and ptype not in ("INT32", "INT64"):
        raise ValueError("DELTA_BINARY_PACKED needs an INT32 or INT64 column")
    elif enc_name == "BYTE_STREAM_SPLIT" and ptype == "BYTE_ARRAY":
        raise ValueError("BYTE_STREAM_SPLIT needs a fixed-width column")
    elif enc_name in ("DELTA_LENGTH_BYTE_ARRAY", "DELTA_BYTE_ARRAY") and ptype != "BYTE_ARRAY":
        raise ValueError(f"{enc_name} needs a BYTE_ARRAY column")

    counts = _page_row_counts(ptype, enc_name, n_rows, valid,
                              rows_view if ptype == "BYTE_ARRAY" or enc_name != "DELTA_BINARY_PACKED"
                              else [int(v) for v in rows_view], page_bytes, bw)

    def build(codec_used):
        out = bytearray()
        locations = []
        total_unc = 0
        total_cmp = 0
        dict_off = None
        if dict_entries is not None:
            if ptype == "BYTE_ARRAY":
                body = _plain.encode_byte_array(dict_entries)
            else:
                body = _plain.encode_fixed(dict_entries, ptype)
            cbody = _compress(codec_used, body)
            hdr = _page_header(DICTIONARY_PAGE, len(body), len(cbody), 7,
                               [(1, T.I32, len(dict_entries)), (2, T.I32, PLAIN)])
            dict_off = base + len(out)
            out += hdr + cbody
            total_unc += len(hdr) + len(body)
            total_cmp += len(hdr) + len(cbody)
        data_off = base + len(out)
        row = 0
        vpos = 0  # index into non-null values
        for c in counts:
            lv = None if valid is None else valid[row:row + c]
            nn = c if lv is None else int(lv.sum())
            # values of the page
            if enc_name == "RLE_DICTIONARY":
                vbytes = bytes([bw]) + _hybrid.encode(dict_idx[vpos:vpos + nn], bw, policy, rng)
            elif enc_name == "DELTA_BINARY_PACKED":
                bits = 32 if ptype == "INT32" else 64
                vbytes = _delta.encode([int(v) for v in nonnull[vpos:vpos + nn]], bits)
            elif enc_name == "BYTE_STREAM_SPLIT":
                vbytes = _bss.encode(nonnull[vpos:vpos + nn], ptype)
            elif enc_name == "DELTA_LENGTH_BYTE_ARRAY":
                vbytes = _dstr.encode_length_byte_array(nonnull[vpos:vpos + nn])
            elif enc_name == "DELTA_BYTE_ARRAY":
                vbytes = _dstr.encode_byte_array(nonnull[vpos:vpos + nn])
            elif ptype == "BYTE_ARRAY":
                vbytes = _plain.encode_byte_array(nonnull[vpos:vpos + nn])
            else:
                vbytes = _plain.encode_fixed(nonnull[vpos:vpos + nn], ptype)
            enc_id = ENCODING_ID[enc_name]
            if cspec.page_version == 1:
                levels = b"" if lv is None else _levels_v1(lv.astype(np.uint64), policy, rng)
                body = levels + vbytes
                cbody = _compress(codec_used, body)
                hdr = _page_header(DATA_PAGE, len(body), len(cbody), 5,
                                   [(1, T.I32, c), (2, T.I32, enc_id), (3, T.I32, RLE), (4, T.I32, RLE)])
            else:
                levels = b"" if lv is None else _hybrid.encode(lv.astype(np.uint64), 1, policy, rng)
                cv = _compress(codec_used, vbytes)
                body_len = len(levels) + len(vbytes)
                cbody = levels + cv
                hdr = _page_header(DATA_PAGE_V2, body_len, len(cbody), 8,
                                   [(1, T.I32, c), (2, T.I32, c - nn), (3, T.I32, c), (4, T.I32, enc_id),
                                    (5, T.I32, len(levels)), (6, T.I32, 0),
                                    (7, T.BOOL_TRUE, codec_used != UNCOMPRESSED)])
            locations.append((base + len(out), len(hdr) + len(cbody), row))
            out += hdr + cbody
            total_unc += len(hdr) + (len(levels) + len(vbytes))
            total_cmp += len(hdr) + len(cbody)
            row += c
            vpos += nn
        return bytes(out), locations, total_unc, total_cmp, dict_off, data_off

    res = build(codec)
    if codec != UNCOMPRESSED and cspec.compress_threshold is not None:
        plain_res = build(UNCOMPRESSED)
        # keep compression only when it saves more than the threshold
        if res[3] > plain_res[3] * (1.0 - cspec.compress_threshold):
            res, codec = plain_res, UNCOMPRESSED
    data, locations, total_unc, total_cmp, dict_off, data_off = res

    encs = {ENCODING_ID[enc_name]}
    if dict_entries is not None:
        encs.add(PLAIN)
    if optional:
        encs.add(RLE)
    meta = [
        (1, T.I32, TYPE_ID[ptype]),
        (2, T.LIST, (T.I32, sorted(encs))),
        (3, T.LIST, (T.BINARY, [col.name])),
        (4, T.I32, codec),
        (5, T.I64, n_rows),
        (6, T.I64, total_unc),
        (7, T.I64, total_cmp),
        (9, T.I64, data_off),
        (11, T.I64, dict_off),
    ]
    if ptype == "BYTE_ARRAY" and cspec.size_statistics:
        meta.append((16, T.STRUCT, [(1, T.I64, int(sum(len(v) for v in nonnull)))]))
    return data, meta, locations, codec


def write_file(table: Table, spec: TableSpec) -> bytes:
    """The whole file as bytes."""
    ncols = len(table.columns)
    assert len(spec.columns) == ncols
    rng = np.random.default_rng(spec.seed)
    out = bytearray(b"PAR1")
    row_groups = []
    all_locations = []
    n = table.n_rows
    for rg, r0 in enumerate(range(0, max(n, 1), spec.rg_rows)):
        r1 = min(n, r0 + spec.rg_rows)
        if r1 <= r0:
            break
        chunks = []
        rg_unc = rg_cmp = 0
        rg_start = len(out)
        for ci, (col, cspec) in enumerate(zip(table.columns, spec.columns)):
            part = slice_column(col, r0, r1)
            start = len(out)
            data, meta, locations, codec = write_chunk(part, cspec, spec.page_bytes, start, rng)
            out += data
            chunks.append([start, meta])
            all_locations.append((rg, ci, locations))
            rg_unc += dict((f, v) for f, _, v in meta)[6]
            rg_cmp += dict((f, v) for f, _, v in meta)[7]
        row_groups.append({"chunks": chunks, "num_rows": r1 - r0, "unc": rg_unc, "cmp": rg_cmp,
                           "start": rg_start, "ordinal": rg})
    oi = {}
    if spec.offset_index:
        for rg, ci, locations in all_locations:
            body = T.encode_struct([(1, T.LIST, (T.STRUCT, [
                [(1, T.I64, off), (2, T.I32, size), (3, T.I64, first)] for off, size, first in locations]))])
            oi[(rg, ci)] = (len(out), len(body))
            out += body
    schema = [[(4, T.BINARY, "schema"), (5, T.I32, ncols)]]
    for col in table.columns:
        schema.append([(1, T.I32, TYPE_ID[col.ptype]), (3, T.I32, REQUIRED if col.valid is None else OPTIONAL),
                       (4, T.BINARY, col.name)])
    rgs = []
    for g in row_groups:
        cols = []
        for ci, (start, meta) in enumerate(g["chunks"]):
            o = oi.get((g["ordinal"], ci))
            cols.append([(2, T.I64, start), (3, T.STRUCT, meta),
                         (4, T.I64, None if o is None else o[0]), (5, T.I32, None if o is None else o[1])])
        rgs.append([(1, T.LIST, (T.STRUCT, cols)), (2, T.I64, g["unc"]), (3, T.I64, g["num_rows"]),
                    (5, T.I64, g["start"]), (6, T.I64, g["cmp"]), (7, T.I16, g["ordinal"])])
    footer = T.encode_struct([
        (1, T.I32, 2),
        (2, T.LIST, (T.STRUCT, schema)),
        (3, T.I64, n),
        (4, T.LIST, (T.STRUCT, rgs)),
        (6, T.BINARY, CREATED_BY),
    ])
    out += footer + len(footer).to_bytes(4, "little") + b"PAR1"
    return bytes(out)
