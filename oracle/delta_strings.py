"""DELTA_LENGTH_BYTE_ARRAY and DELTA_BYTE_ARRAY (test infrastructure only).

The two string encodings of the V2 set the paper's Section 3 ("Encoding
Flexibility", Insight 3) recommends; both reuse DELTA_BINARY_PACKED for
their integer streams.  Definitions, as the public format states them:

DELTA_LENGTH_BYTE_ARRAY: the lengths of the N values as one
DELTA_BINARY_PACKED stream of INT32, then the N values' bytes back to back.
A negative length, or bytes that run past the page, make the page corrupt.

DELTA_BYTE_ARRAY (incremental or front coding): the prefix lengths as one
DELTA_BINARY_PACKED INT32 stream, then the suffixes as
DELTA_LENGTH_BYTE_ARRAY.  Value i is the first prefix[i] bytes of value i-1
followed by suffix i; value -1 is the empty string, so every page starts
afresh and prefix[0] must be 0.  Both streams hold the same count; a prefix
longer than the previous value makes the page corrupt.  For an OPTIONAL
column only the non-null values are stored, and the chain skips the nulls.
"""
from __future__ import annotations

from . import delta as _delta


class DeltaStringError(ValueError):
    pass


def _lengths(buf, pos, end, count):
    vals, pos = _delta.decode(buf, pos, end, 32)
    if len(vals) != count:
        raise DeltaStringError("length stream holds a different count than the page")
    if any(v < 0 for v in vals):
        raise DeltaStringError("negative length")
    return vals, pos


def decode_length_byte_array(buf, pos: int, end: int, count: int):
    """(list of bytes, position after the last value's bytes)."""
    lens, pos = _lengths(buf, pos, end, count)
    out = []
    for n in lens:
        if pos + n > end:
            raise DeltaStringError("value bytes run past the end of the page")
        out.append(bytes(buf[pos:pos + n]))
        pos += n
    return out, pos


def decode_byte_array(buf, pos: int, end: int, count: int):
    """(list of bytes, position after the last suffix's bytes)."""
    prefix, pos = _lengths(buf, pos, end, count)
    suffix, pos = decode_length_byte_array(buf, pos, end, count)
    out, prev = [], b""
    for p, s in zip(prefix, suffix):
        if p > len(prev):
            raise DeltaStringError("prefix longer than the previous value")
        prev = prev[:p] + s
        out.append(prev)
    return out, pos


def encode_length_byte_array(items) -> bytes:
    items = [bytes(s) for s in items]
    return _delta.encode([len(s) for s in items], 32) + b"".join(items)


def common_prefix(a: bytes, b: bytes) -> int:
    n = 0
    while n < len(a) and n < len(b) and a[n] == b[n]:
        n += 1
    return n


def encode_byte_array(items) -> bytes:
    items = [bytes(s) for s in items]
    prefix, suffix, prev = [], [], b""
    for s in items:
        p = common_prefix(prev, s)
        prefix.append(p)
        suffix.append(s[p:])
        prev = s
    return _delta.encode(prefix, 32) + encode_length_byte_array(suffix)
