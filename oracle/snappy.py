"""Snappy raw block format (test infrastructure only).

Parquet compresses each page body separately with the chunk's codec (the
paper's Section 2: compression applied per column chunk; Section 3 "No
Unnecessary Compression").  The raw block format, as its public description
defines it: a ULEB128 uncompressed length, then elements selected by the low
two bits of a tag byte:

* 00 literal: length-1 = tag >> 2 when < 60; tags 60..63 mean the next 1..4
  little-endian bytes hold length-1; the literal bytes follow;
* 01 copy: length = 4 + ((tag >> 2) & 7), offset = ((tag >> 5) << 8) | next byte;
* 10 copy: length = (tag >> 2) + 1, offset = next 2 bytes little-endian;
* 11 copy: length = (tag >> 2) + 1, offset = next 4 bytes little-endian.

A copy repeats bytes from ``offset`` back in the output, one byte at a time
(so offset < length repeats a pattern).  The output must end exactly at the
declared length.
"""
from __future__ import annotations

from .thrift import read_uleb128, uleb128


class SnappyError(ValueError):
    pass


def decompress(buf) -> bytes:
    n, pos = read_uleb128(buf, 0)
    out = bytearray()
    end = len(buf)
    while pos < end:
        tag = buf[pos]
        pos += 1
        kind = tag & 3
        if kind == 0:
            l = tag >> 2
            if l < 60:
                length = l + 1
            else:
                nb = l - 59
                if pos + nb > end:
                    raise SnappyError("literal length runs past the input")
                length = int.from_bytes(bytes(buf[pos:pos + nb]), "little") + 1
                pos += nb
            if pos + length > end:
                raise SnappyError("literal runs past the input")
            if len(out) + length > n:
                raise SnappyError("output exceeds the declared length")
            out += buf[pos:pos + length]
            pos += length
            continue
        if kind == 1:
            if pos + 1 > end:
                raise SnappyError("copy runs past the input")
            length = 4 + ((tag >> 2) & 7)
            offset = ((tag >> 5) << 8) | buf[pos]
            pos += 1
        elif kind == 2:
            if pos + 2 > end:
                raise SnappyError("copy runs past the input")
            length = (tag >> 2) + 1
            offset = int.from_bytes(bytes(buf[pos:pos + 2]), "little")
            pos += 2
        else:
            if pos + 4 > end:
                raise SnappyError("copy runs past the input")
            length = (tag >> 2) + 1
            offset = int.from_bytes(bytes(buf[pos:pos + 4]), "little")
            pos += 4
        if offset == 0 or offset > len(out):
            raise SnappyError("copy offset outside the output written so far")
        if len(out) + length > n:
            raise SnappyError("output exceeds the declared length")
        for _ in range(length):
            out.append(out[-offset])
    if len(out) != n:
        raise SnappyError("output shorter than the declared length")
    return bytes(out)


# ---------------------------------------------------------------- compressor

def _literal(data) -> bytes:
    out = bytearray()
    n = len(data)
    if n == 0:
        return b""
    if n <= 60:
        out.append((n - 1) << 2)
    else:
        nb = ((n - 1).bit_length() + 7) // 8
        out.append((59 + nb) << 2)
        out += (n - 1).to_bytes(nb, "little")
    out += data
    return bytes(out)


def _copy(offset: int, length: int, allow_copy1: bool = True) -> bytes:
    out = bytearray()
    while length > 0:
        if allow_copy1 and 4 <= length <= 11 and offset < 2048:
            out.append(((offset >> 8) << 5) | ((length - 4) << 2) | 1)
            out.append(offset & 0xFF)
            return bytes(out)
        c = min(length, 64)
        if offset < 65536:
            out.append(((c - 1) << 2) | 2)
            out += offset.to_bytes(2, "little")
        else:
            out.append(((c - 1) << 2) | 3)
            out += offset.to_bytes(4, "little")
        length -= c
    return bytes(out)


def compress(data, min_match: int = 4, allow_copy1: bool = True) -> bytes:
    """Greedy LZ77 over 4-byte prefixes (most recent earlier occurrence)."""
    data = bytes(data)
    out = bytearray(uleb128(len(data)))
    table = {}
    i = 0
    lit = 0
    n = len(data)
    while i + min_match <= n:
        key = data[i:i + min_match]
        cand = table.get(key)
        table[key] = i
        if cand is not None:
            l = min_match
            while i + l < n and data[cand + l] == data[i + l]:
                l += 1
            out += _literal(data[lit:i])
            out += _copy(i - cand, l, allow_copy1)
            for k in range(i + 1, min(i + l, n - min_match + 1)):
                table[data[k:k + min_match]] = k
            i += l
            lit = i
        else:
            i += 1
    out += _literal(data[lit:])
    return bytes(out)


def compress_literal_only(data) -> bytes:
    """A valid (non-compressing) block: literals of at most 65536 bytes."""
    data = bytes(data)
    out = bytearray(uleb128(len(data)))
    for a in range(0, len(data), 65536):
        out += _literal(data[a:a + 65536])
    return bytes(out)
