"""The CPU oracle's reading of single column chunks, for process pools.

A worker gets one chunk's stored bytes (cut out of the file, with the
chunk's offsets moved to match) and returns the rows the oracle reader
decodes from them, as plain numpy arrays: fixed-width values, or int64
offsets from 0 plus chars for BYTE_ARRAY, and the validity per row (or
None).  Nothing here decodes by itself; every value comes from
``oracle.reader``."""
from __future__ import annotations

import dataclasses

import numpy as np

SLACK = 64  # bytes kept after a chunk's last page (the footer follows it in a file)


def cut_chunk(data, ch):
    """(bytes of one chunk plus SLACK, ChunkInfo with offsets into them)."""
    start = ch.start
    end = min(len(data), ch.start + ch.total_compressed + SLACK)
    blob = bytes(data[start:end])
    moved = dataclasses.replace(
        ch, start=0, data_page_offset=ch.data_page_offset - start,
        dictionary_page_offset=None if ch.dictionary_page_offset is None else ch.dictionary_page_offset - start,
        offset_index=None)
    return blob, moved


def expected_chunk(args):
    """Worker: (rg, column, values or offsets, chars or None, valid or None)."""
    from oracle import reader as R
    blob, ch = args
    vals, valid = R.decode_chunk(blob, ch)
    if ch.ptype == "BYTE_ARRAY":
        lens = np.fromiter((len(x) for x in vals), dtype=np.int64, count=len(vals))
        offsets = np.zeros(len(vals) + 1, dtype=np.int64)
        np.cumsum(lens, out=offsets[1:])
        chars = np.frombuffer(b"".join(vals), dtype=np.uint8).copy()
        return ch.rg, ch.column, offsets, chars, valid
    return ch.rg, ch.column, np.ascontiguousarray(vals), None, valid
