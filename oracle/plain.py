"""PLAIN encoding (test infrastructure only).

Fixed-width physical types are stored little-endian back to back (INT32: 4
bytes, INT64 and DOUBLE: 8 bytes, DOUBLE bitwise IEEE 754); BYTE_ARRAY
values are a 4-byte little-endian length followed by the bytes.  Dictionary
pages are PLAIN-encoded too.
"""
from __future__ import annotations

import numpy as np

WIDTH = {"INT32": 4, "INT64": 8, "DOUBLE": 8}
DTYPE = {"INT32": "<i4", "INT64": "<i8", "DOUBLE": "<f8"}


class PlainError(ValueError):
    pass


def encode_fixed(values, ptype: str) -> bytes:
    return np.asarray(values).astype(DTYPE[ptype]).tobytes()


def decode_fixed(buf, pos: int, end: int, ptype: str, count: int):
    nbytes = count * WIDTH[ptype]
    if pos + nbytes > end:
        raise PlainError("PLAIN values run past the end of the page")
    return np.frombuffer(bytes(buf[pos:pos + nbytes]), dtype=DTYPE[ptype]).copy(), pos + nbytes


def encode_byte_array(items) -> bytes:
    out = bytearray()
    for s in items:
        out += len(s).to_bytes(4, "little") + bytes(s)
    return bytes(out)


def decode_byte_array(buf, pos: int, end: int, count: int):
    """Returns (list of bytes, end position)."""
    items = []
    for _ in range(count):
        if pos + 4 > end:
            raise PlainError("BYTE_ARRAY length runs past the end of the page")
        n = int.from_bytes(bytes(buf[pos:pos + 4]), "little")
        pos += 4
        if pos + n > end:
            raise PlainError("BYTE_ARRAY value runs past the end of the page")
        items.append(bytes(buf[pos:pos + n]))
        pos += n
    return items, pos
