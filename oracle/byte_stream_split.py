"""BYTE_STREAM_SPLIT (test infrastructure only).

One of the V2 encodings the paper's Section 3 ("Encoding Flexibility",
Insight 3) counts among the modern, GPU-friendly ones: no bit twiddling,
only a fixed byte permutation.  Definition, as the public format states it:

a page of N values of a K-byte type is K streams of N bytes each; stream b
holds byte b (little-endian order) of every value, value order kept.  So
the value region is a K x N byte matrix whose transpose is the PLAIN
encoding of the same values.  N is the region size divided by K; a region
whose size is not a multiple of K is corrupt.  For an OPTIONAL column only
the non-null values are stored (N >= the page's non-null count).
"""
from __future__ import annotations

import numpy as np

from .plain import DTYPE, WIDTH


class ByteStreamSplitError(ValueError):
    pass


def decode(buf, pos: int, end: int, ptype: str, count: int) -> np.ndarray:
    """The first ``count`` values of the streams in buf[pos:end]."""
    width = WIDTH[ptype]
    size = end - pos
    if size < 0 or size % width:
        raise ByteStreamSplitError("value region is not a whole number of values")
    n = size // width
    if count > n:
        raise ByteStreamSplitError("fewer values in the streams than the page needs")
    out = bytearray(count * width)
    for k in range(count):
        for b in range(width):
            out[k * width + b] = buf[pos + b * n + k]
    return np.frombuffer(bytes(out), dtype=DTYPE[ptype]).copy()


def encode(values, ptype: str) -> bytes:
    """Streams of ``values`` (byte b of every value, for b = 0 .. K-1)."""
    raw = np.asarray(values).astype(DTYPE[ptype]).tobytes()
    width = WIDTH[ptype]
    n = len(raw) // width
    out = bytearray(len(raw))
    for k in range(n):
        for b in range(width):
            out[b * n + k] = raw[k * width + b]
    return bytes(out)
