"""RLE / bit-packed hybrid encoding (test infrastructure only).

The run-length/bit-packing hybrid carries Parquet's definition levels and
dictionary indices (the V1 dictionary encoding the paper's Section 3 calls
the default, and the level streams of both page versions).  Definition, as
the public format states it:

* the stream is a sequence of runs, each introduced by a ULEB128 header h;
* h & 1 == 1: a bit-packed run of (h >> 1) groups of 8 values; the values are
  packed LSB-first at ``bit_width`` bits each, so the run body is
  (h >> 1) * bit_width bytes;
* h & 1 == 0: a repeated run, the value repeated (h >> 1) times, stored in
  ceil(bit_width / 8) little-endian bytes;
* padding values in the last bit-packed group past the logical count are
  ignored by the reader.

The reader below follows that definition run by run; bit unpacking is
vectorised with numpy (bit j of the stream is bit j % 8 of byte j // 8).
"""
from __future__ import annotations

import numpy as np

from .thrift import read_uleb128, uleb128


class HybridError(ValueError):
    pass


def unpack_lsb(data, bit_offset: int, count: int, width: int) -> np.ndarray:
    """``count`` unsigned ``width``-bit values packed LSB-first starting at
    bit ``bit_offset`` of ``data``; returned as uint64."""
    if width == 0 or count == 0:
        return np.zeros(count, dtype=np.uint64)
    first = bit_offset // 8
    last = (bit_offset + count * width + 7) // 8
    if last > len(data):
        raise HybridError("bit-packed values run past the end of the buffer")
    bits = np.unpackbits(np.frombuffer(bytes(data[first:last]), dtype=np.uint8), bitorder="little")
    start = bit_offset - first * 8
    bits = bits[start:start + count * width].reshape(count, width).astype(np.uint64)
    out = np.zeros(count, dtype=np.uint64)
    for j in range(width):
        out |= bits[:, j] << np.uint64(j)
    return out


def pack_lsb(values, width: int) -> bytes:
    """Inverse of ``unpack_lsb`` (bit_offset 0); pads the last byte with 0."""
    values = np.asarray(values, dtype=np.uint64)
    if width == 0 or values.size == 0:
        return b""
    bits = ((values[:, None] >> np.arange(width, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.uint8)
    return np.packbits(bits.reshape(-1), bitorder="little").tobytes()


def bit_width_for(max_value: int) -> int:
    """Number of bits needed to store values in [0, max_value]."""
    return int(max_value).bit_length()


def decode(buf, pos: int, end: int, bit_width: int, count: int):
    """Decodes ``count`` values of a hybrid stream occupying buf[pos:end].
    Returns (uint64 array, position after the last run read)."""
    if not 0 <= bit_width <= 64:
        raise HybridError(f"bit width {bit_width} out of range")
    out = np.zeros(count, dtype=np.uint64)
    n = 0
    value_bytes = (bit_width + 7) // 8
    while n < count:
        h, pos = read_uleb128(buf, pos, end)
        if h & 1:
            groups = h >> 1
            nbytes = groups * bit_width
            if pos + nbytes > end:
                raise HybridError("bit-packed run runs past the end of the stream")
            take = min(groups * 8, count - n)
            out[n:n + take] = unpack_lsb(buf[pos:pos + nbytes], 0, take, bit_width)
            pos += nbytes
            n += take
        else:
            run = h >> 1
            if pos + value_bytes > end:
                raise HybridError("repeated run value runs past the end of the stream")
            v = int.from_bytes(bytes(buf[pos:pos + value_bytes]), "little")
            if bit_width < 64 and v >> bit_width:
                raise HybridError("repeated value wider than the bit width")
            pos += value_bytes
            take = min(run, count - n)
            out[n:n + take] = v
            n += take
            if run == 0 and pos >= end:
                raise HybridError("empty runs up to the end of the stream")
    return out, pos


# ---------------------------------------------------------------- writer

def _rle_run(value: int, count: int, bit_width: int) -> bytes:
    return uleb128(count << 1) + int(value).to_bytes((bit_width + 7) // 8, "little")


def _packed_run(values, bit_width: int) -> bytes:
    groups = (len(values) + 7) // 8
    padded = np.zeros(groups * 8, dtype=np.uint64)
    padded[:len(values)] = values
    return uleb128((groups << 1) | 1) + pack_lsb(padded, bit_width)


def _equal_run_length(values, i: int) -> int:
    j = i
    while j < len(values) and values[j] == values[i]:
        j += 1
    return j - i


def encode(values, bit_width: int, policy: str = "default", rng=None) -> bytes:
    """Encodes a sequence of unsigned values.  The decoder result is unique;
    the policy only picks one of the many valid byte streams:

    * ``default``: a repeated run for every stretch of >= 8 equal values,
      other values in bit-packed runs of at most 63 groups;
    * ``rle``: every maximal stretch of equal values as a repeated run;
    * ``packed``: bit-packed runs only (at most 63 groups each);
    * ``mixed``: a seeded random mixture of the above (needs ``rng``).
    """
    values = [int(v) for v in np.asarray(values, dtype=np.uint64)]
    n = len(values)
    out = bytearray()
    if policy == "rle":
        i = 0
        while i < n:
            r = _equal_run_length(values, i)
            out += _rle_run(values[i], r, bit_width)
            i += r
        return bytes(out)
    if policy == "packed":
        for i in range(0, n, 63 * 8):
            out += _packed_run(values[i:i + 63 * 8], bit_width)
        return bytes(out)
    if policy == "default":
        pending = []
        i = 0

        def flush():
            for a in range(0, len(pending), 63 * 8):
                out.extend(_packed_run(pending[a:a + 63 * 8], bit_width))
            pending.clear()

        while i < n:
            r = _equal_run_length(values, i)
            if r >= 8 and len(pending) % 8 == 0:
                flush()
                out += _rle_run(values[i], r, bit_width)
                i += r
            else:
                pending.append(values[i])
                i += 1
        flush()
        return bytes(out)
    if policy == "mixed":
        assert rng is not None
        i = 0
        while i < n:
            if rng.random() < 0.5:
                r = _equal_run_length(values, i)
                take = int(rng.integers(1, r + 1))
                out += _rle_run(values[i], take, bit_width)
                i += take
            else:
                groups = int(rng.integers(1, 64))
                take = min(groups * 8, n - i)
                if take < groups * 8 and i + take < n:
                    raise AssertionError
                out += _packed_run(values[i:i + take], bit_width)
                i += take
        return bytes(out)
    raise ValueError(f"unknown hybrid policy {policy!r}")
