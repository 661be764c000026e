"""DELTA_BINARY_PACKED (test infrastructure only).

The V2 integer encoding the paper's Section 3 ("Encoding Flexibility",
Insight 3) singles out as fast to decode.  Definition, as the public format
states it:

header: ULEB128 block size (a multiple of 128), ULEB128 miniblocks per
block (values per miniblock a multiple of 32), ULEB128 total value count,
zigzag ULEB128 first value.  Then blocks, each: zigzag ULEB128 min delta,
one bit-width byte per miniblock, then each needed miniblock's
(delta - min delta) values packed LSB-first at that width.  Value i is
value i-1 + min delta + packed delta, wrapping in the physical type
(two's complement, 32 or 64 bits).  Miniblocks past the last value carry a
width byte but no body.
"""
from __future__ import annotations

import numpy as np

from .hybrid import pack_lsb, unpack_lsb
from .thrift import read_uleb128, uleb128, unzigzag, zigzag


class DeltaError(ValueError):
    pass


def _wrap(v: int, bits: int) -> int:
    """Two's-complement wrap of a Python int to ``bits`` bits, signed."""
    v &= (1 << bits) - 1
    return v - (1 << bits) if v >> (bits - 1) else v


def decode(buf, pos: int, end: int, bits: int):
    """Decodes one DELTA_BINARY_PACKED stream of a ``bits``-bit integer type.
    Returns (python list of ints, position after the stream)."""
    block_size, pos = read_uleb128(buf, pos, end)
    miniblocks, pos = read_uleb128(buf, pos, end)
    total, pos = read_uleb128(buf, pos, end)
    first_u, pos = read_uleb128(buf, pos, end)
    if block_size == 0 or block_size % 128 or miniblocks == 0 or block_size % miniblocks:
        raise DeltaError("bad block size / miniblock count")
    per_mb = block_size // miniblocks
    if per_mb % 32:
        raise DeltaError("values per miniblock not a multiple of 32")
    out = []
    if total == 0:
        return out, pos
    prev = _wrap(unzigzag(first_u), bits)
    out.append(prev)
    while len(out) < total:
        min_u, pos = read_uleb128(buf, pos, end)
        min_delta = unzigzag(min_u)
        if pos + miniblocks > end:
            raise DeltaError("bit widths run past the end of the stream")
        widths = list(buf[pos:pos + miniblocks])
        pos += miniblocks
        for w in widths:
            if len(out) >= total:
                break
            if w > bits:
                raise DeltaError(f"miniblock bit width {w} wider than the type")
            nbytes = per_mb * w // 8
            if pos + nbytes > end:
                raise DeltaError("miniblock runs past the end of the stream")
            packed = unpack_lsb(buf[pos:pos + nbytes], 0, per_mb, w)
            pos += nbytes
            for p in packed[:total - len(out)]:
                prev = _wrap(prev + min_delta + int(p), bits)
                out.append(prev)
    return out, pos


def wrap(v: int, bits: int) -> int:
    return _wrap(v, bits)


def encode_header(count: int, first: int, bits: int, block_size: int = 128, miniblocks: int = 4) -> bytes:
    return (uleb128(block_size) + uleb128(miniblocks) + uleb128(count)
            + uleb128(zigzag(_wrap(int(first), bits) if count else 0, bits)))


def encode_block(deltas, bits: int, block_size: int = 128, miniblocks: int = 4) -> bytes:
    """One block for up to ``block_size`` wrapped deltas."""
    per_mb = block_size // miniblocks
    mask = (1 << bits) - 1
    mn = min(deltas)
    packed = [(d - mn) & mask for d in deltas]
    out = bytearray(uleb128(zigzag(mn, bits)))
    widths, bodies = [], []
    for m in range(miniblocks):
        part = packed[m * per_mb:(m + 1) * per_mb]
        if not part:
            widths.append(0)
            continue
        w = max(part).bit_length()
        widths.append(w)
        padded = np.zeros(per_mb, dtype=np.uint64)
        padded[:len(part)] = np.array(part, dtype=np.uint64)
        bodies.append(pack_lsb(padded, w))
    out += bytes(widths)
    for body in bodies:
        out += body
    return bytes(out)


def encode(values, bits: int, block_size: int = 128, miniblocks: int = 4) -> bytes:
    """One DELTA_BINARY_PACKED stream for ``values`` (signed ints)."""
    vals = [_wrap(int(v), bits) for v in values]
    n = len(vals)
    out = bytearray(encode_header(n, vals[0] if n else 0, bits, block_size, miniblocks))
    deltas = [_wrap(vals[i] - vals[i - 1], bits) for i in range(1, n)]
    for b in range(0, len(deltas), block_size):
        out += encode_block(deltas[b:b + block_size], bits, block_size, miniblocks)
    return bytes(out)
