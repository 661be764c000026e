"""Parquet reader for the oracle (test infrastructure only).

Decodes a flat Parquet file into typed columns, one value at a time in the
order the format defines (the scan of the paper's Section 2: row groups ->
column chunks -> pages; decompression then decoding):

* footer: ``PAR1`` ... FileMetaData (Thrift compact) + 4-byte LE length + ``PAR1``;
* a chunk starts at dictionary_page_offset when set, else data_page_offset;
  the next page header follows the previous header end plus its
  compressed_page_size; the walk stops once the data pages' num_values add up
  to the chunk's num_values;
* V1 data page: whole body decompressed with the chunk codec (Snappy or
  Zstandard, the codecs of Section 2); OPTIONAL
  columns first carry a 4-byte LE length + RLE/bit-packed def levels (bit
  width 1); V2 data page: rep/def levels (lengths from the header) are never
  compressed, values are compressed when is_compressed (default true);
* values: PLAIN, RLE_DICTIONARY / PLAIN_DICTIONARY (1-byte bit width + hybrid
  indices into the chunk's dictionary), DELTA_BINARY_PACKED, and the other
  V2 encodings of Section 3's Insight 3: BYTE_STREAM_SPLIT (fixed width),
  DELTA_LENGTH_BYTE_ARRAY and DELTA_BYTE_ARRAY (BYTE_ARRAY);
* row r of a page is null when its definition level is below the maximum
  (1); null slots of fixed-width outputs are 0; BYTE_ARRAY outputs are int64
  offsets (n + 1) plus chars.

Output conventions match the engine's: validity as a bool array per row
(the tests pack it LSB-first, 1 = valid).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import byte_stream_split as _bss
from . import delta as _delta
from . import delta_strings as _dstr
from . import hybrid as _hybrid
from . import plain as _plain
from . import snappy as _snappy
from . import thrift as T
from . import zstd as _zstd
from .parquet_meta import (BYTE_STREAM_SPLIT, DATA_PAGE, DATA_PAGE_V2, DELTA_BINARY_PACKED,
                           DELTA_BYTE_ARRAY, DELTA_LENGTH_BYTE_ARRAY, DICTIONARY_PAGE, OPTIONAL, PLAIN,
                           PLAIN_DICTIONARY, REPEATED, RLE_DICTIONARY, SNAPPY, TYPE_NAME, UNCOMPRESSED, ZSTD)


class ParquetError(ValueError):
    pass


class Unsupported(ParquetError):
    pass


@dataclass
class ColumnInfo:
    name: str
    ptype: str
    max_def: int


@dataclass
class ChunkInfo:
    rg: int
    column: int
    ptype: str
    max_def: int
    codec: int
    num_values: int
    start: int
    total_compressed: int
    data_page_offset: int
    dictionary_page_offset: Optional[int]
    first_row: int          # of the row group in the file
    offset_index: Optional[tuple] = None  # (offset, length)


@dataclass
class PageInfo:
    offset: int             # of the page header in the file
    header_len: int
    page_type: int
    uncompressed: int
    compressed: int
    num_values: int = 0
    encoding: int = 0
    num_nulls: int = -1     # V2 only
    num_rows: int = -1      # V2 only
    def_len: int = 0        # V2 only
    rep_len: int = 0        # V2 only
    is_compressed: bool = True


@dataclass
class FileInfo:
    num_rows: int
    columns: List[ColumnInfo]
    chunks: List[ChunkInfo]
    rg_rows: List[int]
    raw: dict = field(default_factory=dict)


def parse_footer(data) -> FileInfo:
    if len(data) < 12 or bytes(data[:4]) != b"PAR1" or bytes(data[-4:]) != b"PAR1":
        raise ParquetError("missing PAR1 magic")
    flen = int.from_bytes(bytes(data[-8:-4]), "little")
    if flen + 12 > len(data):
        raise ParquetError("footer length larger than the file")
    fstart = len(data) - 8 - flen
    meta, _ = T.decode_struct(data, fstart, len(data) - 8)
    schema = meta.get(2, [])
    if not schema:
        raise ParquetError("empty schema")
    root = schema[0]
    ncols = root.get(5, 0)
    if len(schema) != ncols + 1:
        raise Unsupported("nested schema")
    cols = []
    for el in schema[1:]:
        if el.get(5):
            raise Unsupported("nested schema")
        rep = el.get(3, 0)
        if rep == REPEATED:
            raise Unsupported("repeated column")
        cols.append(ColumnInfo(el[4].decode(), TYPE_NAME[el[1]], 1 if rep == OPTIONAL else 0))
    chunks, rg_rows = [], []
    first_row = 0
    for g, rg in enumerate(meta.get(4, [])):
        nrows = rg[3]
        rg_rows.append(nrows)
        if len(rg[1]) != ncols:
            raise ParquetError("row group has the wrong number of chunks")
        for c, cc in enumerate(rg[1]):
            md = cc.get(3)
            if md is None:
                raise Unsupported("column metadata stored outside the footer")
            dpo = md[9]
            dict_off = md.get(11)
            start = dict_off if dict_off is not None and 0 < dict_off < dpo else dpo
            oi = (cc[4], cc[5]) if 4 in cc and 5 in cc else None
            chunks.append(ChunkInfo(g, c, TYPE_NAME[md[1]], cols[c].max_def, md[4], md[5], start, md[7],
                                    dpo, dict_off, first_row, oi))
        first_row += nrows
    return FileInfo(meta[3], cols, chunks, rg_rows, meta)


def parse_page_header(data, pos: int, end: int) -> PageInfo:
    h, hend = T.decode_struct(data, pos, end)
    try:
        p = PageInfo(pos, hend - pos, h[1], h[2], h[3])
    except KeyError as e:
        raise ParquetError(f"page header misses field {e}")
    if p.uncompressed < 0 or p.compressed < 0:
        raise ParquetError("negative page size")
    if p.page_type == DATA_PAGE:
        d = h[5]
        p.num_values, p.encoding = d[1], d[2]
    elif p.page_type == DICTIONARY_PAGE:
        d = h[7]
        p.num_values, p.encoding = d[1], d[2]
    elif p.page_type == DATA_PAGE_V2:
        d = h[8]
        p.num_values, p.num_nulls, p.num_rows, p.encoding = d[1], d[2], d[3], d[4]
        p.def_len, p.rep_len = d[5], d[6]
        p.is_compressed = d.get(7, True)
    return p


def chunk_pages(data, ch: ChunkInfo) -> List[PageInfo]:
    """Walks the page headers of one chunk."""
    pages = []
    pos = ch.start
    end = ch.start + ch.total_compressed
    if end > len(data):
        raise ParquetError("chunk runs past the end of the file")
    seen = 0
    while seen < ch.num_values:
        if pos >= end:
            raise ParquetError("chunk ends before all values were seen")
        p = parse_page_header(data, pos, end)
        pos += p.header_len + p.compressed
        if pos > end:
            raise ParquetError("page runs past the end of the chunk")
        pages.append(p)
        if p.page_type in (DATA_PAGE, DATA_PAGE_V2):
            seen += p.num_values
    return pages


def _decompress(codec, body, expect):
    if codec == UNCOMPRESSED:
        out = bytes(body)
    elif codec == SNAPPY:
        out = _snappy.decompress(body)
    elif codec == ZSTD:
        out = _zstd.decompress(body)
    else:
        raise Unsupported(f"codec {codec}")
    if len(out) != expect:
        raise ParquetError("decompressed size differs from the header")
    return out


def decode_dictionary(data, p: PageInfo, ch: ChunkInfo):
    body = data[p.offset + p.header_len:p.offset + p.header_len + p.compressed]
    raw = _decompress(ch.codec, body, p.uncompressed)
    if p.encoding not in (PLAIN, PLAIN_DICTIONARY):
        raise Unsupported("dictionary page encoding")
    if ch.ptype == "BYTE_ARRAY":
        items, _ = _plain.decode_byte_array(raw, 0, len(raw), p.num_values)
        return items
    vals, _ = _plain.decode_fixed(raw, 0, len(raw), ch.ptype, p.num_values)
    return vals


def decode_data_page(data, p: PageInfo, ch: ChunkInfo, dictionary):
    """Returns (row values: list (BYTE_ARRAY) or numpy array with null
    slots 0, validity bool array or None)."""
    body = data[p.offset + p.header_len:p.offset + p.header_len + p.compressed]
    nrows = p.num_values
    if p.page_type == DATA_PAGE:
        raw = _decompress(ch.codec, body, p.uncompressed)
        pos = 0
        levels = None
        if ch.max_def:
            if len(raw) < 4:
                raise ParquetError("missing definition level length")
            ln = int.from_bytes(raw[0:4], "little")
            if 4 + ln > len(raw):
                raise ParquetError("definition levels run past the page")
            levels, _ = _hybrid.decode(raw, 4, 4 + ln, 1, nrows)
            pos = 4 + ln
        vals_buf, vpos = raw, pos
    elif p.page_type == DATA_PAGE_V2:
        if p.rep_len:
            raise Unsupported("repetition levels")
        if p.def_len + p.rep_len > len(body):
            raise ParquetError("levels run past the page")
        levels = None
        if ch.max_def:
            levels, _ = _hybrid.decode(body, 0, p.def_len, 1, nrows)
        vbody = body[p.def_len:]
        vexpect = p.uncompressed - p.def_len
        if p.is_compressed and ch.codec != UNCOMPRESSED:
            vals_buf = _decompress(ch.codec, vbody, vexpect)
        else:
            vals_buf = bytes(vbody)
            if len(vals_buf) != vexpect:
                raise ParquetError("V2 value size differs from the header")
        vpos = 0
    else:
        raise ParquetError("not a data page")
    valid = None if levels is None else levels == 1
    if levels is not None and np.any(levels > 1):
        raise ParquetError("definition level above the maximum")
    nn = nrows if valid is None else int(valid.sum())
    if p.page_type == DATA_PAGE_V2 and ch.max_def and p.num_nulls != nrows - nn:
        raise ParquetError("num_nulls disagrees with the definition levels")
    end = len(vals_buf)
    enc = p.encoding
    if enc == PLAIN:
        if ch.ptype == "BYTE_ARRAY":
            dense, _ = _plain.decode_byte_array(vals_buf, vpos, end, nn)
        else:
            dense, _ = _plain.decode_fixed(vals_buf, vpos, end, ch.ptype, nn)
    elif enc in (RLE_DICTIONARY, PLAIN_DICTIONARY):
        if dictionary is None:
            raise ParquetError("dictionary-encoded page without a dictionary page")
        if nn and vpos >= end:
            raise ParquetError("missing index bit width")
        bw = vals_buf[vpos] if vpos < end else 0
        if bw > 32:
            raise ParquetError("index bit width above 32")
        idx, _ = _hybrid.decode(vals_buf, vpos + 1, end, bw, nn)
        if nn and int(idx.max()) >= len(dictionary):
            raise ParquetError("dictionary index out of range")
        if ch.ptype == "BYTE_ARRAY":
            dense = [dictionary[int(i)] for i in idx]
        else:
            dense = np.asarray(dictionary)[idx.astype(np.int64)]
    elif enc == DELTA_BINARY_PACKED:
        if ch.ptype not in ("INT32", "INT64"):
            raise ParquetError("DELTA_BINARY_PACKED on a non-integer column")
        bits = 32 if ch.ptype == "INT32" else 64
        vals, _ = _delta.decode(vals_buf, vpos, end, bits)
        if len(vals) != nn:
            raise ParquetError("DELTA value count differs from the page")
        dense = np.array(vals, dtype=np.int32 if bits == 32 else np.int64)
    elif enc == BYTE_STREAM_SPLIT:
        if ch.ptype == "BYTE_ARRAY":
            raise ParquetError("BYTE_STREAM_SPLIT on a BYTE_ARRAY column")
        dense = _bss.decode(vals_buf, vpos, end, ch.ptype, nn)
    elif enc in (DELTA_LENGTH_BYTE_ARRAY, DELTA_BYTE_ARRAY):
        if ch.ptype != "BYTE_ARRAY":
            raise ParquetError("delta string encoding on a fixed-width column")
        dec = _dstr.decode_length_byte_array if enc == DELTA_LENGTH_BYTE_ARRAY else _dstr.decode_byte_array
        dense, _ = dec(vals_buf, vpos, end, nn)
    else:
        raise Unsupported(f"encoding {enc}")
    # assemble rows
    if ch.ptype == "BYTE_ARRAY":
        if valid is None:
            return list(dense), None
        it = iter(dense)
        return [next(it) if v else b"" for v in valid], valid
    dtype = _plain.DTYPE[ch.ptype]
    out = np.zeros(nrows, dtype=dtype)
    if valid is None:
        out[:] = dense
    else:
        out[valid] = dense
    return out, valid


@dataclass
class ColumnResult:
    name: str
    ptype: str
    values: Optional[np.ndarray] = None   # fixed width, n rows
    valid: Optional[np.ndarray] = None    # bool, or None for REQUIRED
    offsets: Optional[np.ndarray] = None  # BYTE_ARRAY: int64, n + 1
    chars: Optional[np.ndarray] = None    # BYTE_ARRAY: uint8


def decode_chunk(data, ch: ChunkInfo):
    """(row values, validity or None) of one chunk."""
    pages = chunk_pages(data, ch)
    dictionary = None
    parts, valids = [], []
    for p in pages:
        if p.page_type == DICTIONARY_PAGE:
            if dictionary is not None:
                raise ParquetError("two dictionary pages in one chunk")
            dictionary = decode_dictionary(data, p, ch)
        elif p.page_type in (DATA_PAGE, DATA_PAGE_V2):
            v, ok = decode_data_page(data, p, ch, dictionary)
            parts.append(v)
            valids.append(ok)
    if ch.ptype == "BYTE_ARRAY":
        vals = [x for part in parts for x in part]
    else:
        vals = np.concatenate(parts) if parts else np.zeros(0, dtype=_plain.DTYPE[ch.ptype])
    valid = None if ch.max_def == 0 else (np.concatenate(valids) if valids else np.zeros(0, bool))
    return vals, valid


def read_file(data, columns=None) -> List[ColumnResult]:
    """All rows of the requested columns (default: all)."""
    info = parse_footer(data)
    want = range(len(info.columns)) if columns is None else columns
    out = []
    for c in want:
        ci = info.columns[c]
        parts, valids = [], []
        for ch in info.chunks:
            if ch.column != c:
                continue
            v, ok = decode_chunk(data, ch)
            parts.append(v)
            valids.append(ok)
        valid = None if ci.max_def == 0 else np.concatenate(valids) if valids else np.zeros(0, bool)
        if ci.ptype == "BYTE_ARRAY":
            items = [x for part in parts for x in part]
            lens = np.array([len(x) for x in items], dtype=np.int64)
            offsets = np.zeros(len(items) + 1, dtype=np.int64)
            np.cumsum(lens, out=offsets[1:])
            chars = np.frombuffer(b"".join(items), dtype=np.uint8).copy()
            out.append(ColumnResult(ci.name, ci.ptype, None, valid, offsets, chars))
        else:
            vals = np.concatenate(parts) if parts else np.zeros(0, dtype=_plain.DTYPE[ci.ptype])
            out.append(ColumnResult(ci.name, ci.ptype, vals, valid))
    return out


def read_offset_index(data, ch: ChunkInfo):
    """[(offset, size incl. header, first_row_index)] or None."""
    if ch.offset_index is None:
        return None
    off, ln = ch.offset_index
    d, _ = T.decode_struct(data, off, off + ln)
    return [(pl[1], pl[2], pl[3]) for pl in d[1]]
