"""Thrift compact protocol, written out plainly (test infrastructure only).

Parquet stores its FileMetaData, PageHeader and OffsetIndex structures with
the Thrift compact protocol (the metadata of the file hierarchy in the
paper's Section 2).  Rules implemented here:

* integers i16/i32/i64 are zigzag-encoded then written as ULEB128 varints;
* a field header is one byte ``(id_delta << 4) | type`` when the delta from
  the previous field id of the same struct is 1..15, otherwise the type byte
  followed by the zigzag varint field id;
* booleans as fields carry their value in the type nibble (1 true, 2 false);
  inside lists they are one byte (1 true, 2 false);
* binary/string = varint length + bytes; double = 8 bytes little-endian;
* list/set header = ``(size << 4) | elem_type`` when size < 15, else
  ``0xF0 | elem_type`` followed by the varint size;
* a struct ends with a STOP byte (0); a nested struct starts a fresh
  last-field-id of 0.

Structs are handled as plain dicts ``{field_id: value}``; for writing, each
field is given as ``(field_id, type, value)``.
"""
from __future__ import annotations

import struct as _struct

STOP, BOOL_TRUE, BOOL_FALSE, BYTE, I16, I32, I64, DOUBLE, BINARY, LIST, SET, MAP, STRUCT = range(13)


class ThriftError(ValueError):
    pass


# ---------------------------------------------------------------- varints

def uleb128(n: int) -> bytes:
    assert n >= 0
    out = bytearray()
    while True:
        b = n & 0x7F
        n >>= 7
        if n:
            out.append(b | 0x80)
        else:
            out.append(b)
            return bytes(out)


def zigzag(n: int, bits: int = 64) -> int:
    """Map signed -> unsigned: 0,-1,1,-2,... -> 0,1,2,3,..."""
    return (n << 1) ^ (n >> (bits - 1)) if n < 0 else n << 1


def unzigzag(u: int) -> int:
    return (u >> 1) ^ -(u & 1)


def read_uleb128(buf, pos: int, limit: int = None):
    """Returns (value, new_pos).  At most 10 bytes (64-bit values)."""
    limit = len(buf) if limit is None else limit
    result = 0
    shift = 0
    for i in range(10):
        if pos >= limit:
            raise ThriftError("varint runs past the end of the buffer")
        b = buf[pos]
        pos += 1
        result |= (b & 0x7F) << shift
        if not b & 0x80:
            return result, pos
        shift += 7
    raise ThriftError("varint longer than 10 bytes")


# ---------------------------------------------------------------- writer

def _write_value(out: bytearray, ttype: int, value) -> None:
    if ttype == BYTE:
        out.append(value & 0xFF)
    elif ttype in (I16, I32, I64):
        out += uleb128(zigzag(int(value)))
    elif ttype == DOUBLE:
        out += _struct.pack("<d", value)
    elif ttype == BINARY:
        data = value.encode() if isinstance(value, str) else bytes(value)
        out += uleb128(len(data)) + data
    elif ttype in (LIST, SET):
        elem_type, items = value
        n = len(items)
        if n < 15:
            out.append((n << 4) | elem_type)
        else:
            out.append(0xF0 | elem_type)
            out += uleb128(n)
        for it in items:
            if elem_type in (BOOL_TRUE, BOOL_FALSE):
                out.append(BOOL_TRUE if it else BOOL_FALSE)
            else:
                _write_value(out, elem_type, it)
    elif ttype == STRUCT:
        out += encode_struct(value)
    else:
        raise ThriftError(f"cannot write type {ttype}")


def encode_struct(fields) -> bytes:
    """fields: iterable of (field_id, type, value); None values are skipped.
    Field ids must ascend (the writer emits them in the given order)."""
    out = bytearray()
    last = 0
    for fid, ttype, value in fields:
        if value is None:
            continue
        wire_type = ttype
        if ttype in (BOOL_TRUE, BOOL_FALSE):
            wire_type = BOOL_TRUE if value else BOOL_FALSE
        delta = fid - last
        if 0 < delta <= 15:
            out.append((delta << 4) | wire_type)
        else:
            out.append(wire_type)
            out += uleb128(zigzag(fid))
        if ttype not in (BOOL_TRUE, BOOL_FALSE):
            _write_value(out, ttype, value)
        last = fid
    out.append(STOP)
    return bytes(out)


# ---------------------------------------------------------------- reader

class Reader:
    """Decodes compact-protocol structs into {field_id: value} dicts."""

    def __init__(self, buf, pos: int = 0, end: int = None, max_depth: int = 32):
        self.buf = buf
        self.pos = pos
        self.end = len(buf) if end is None else end
        self.max_depth = max_depth

    def _byte(self) -> int:
        if self.pos >= self.end:
            raise ThriftError("struct runs past the end of the buffer")
        b = self.buf[self.pos]
        self.pos += 1
        return b

    def _varint(self) -> int:
        v, self.pos = read_uleb128(self.buf, self.pos, self.end)
        return v

    def _value(self, ttype: int, depth: int):
        if ttype in (BOOL_TRUE, BOOL_FALSE):  # only reached inside containers
            return self._byte() == BOOL_TRUE
        if ttype == BYTE:
            return self._byte()
        if ttype in (I16, I32, I64):
            return unzigzag(self._varint())
        if ttype == DOUBLE:
            if self.pos + 8 > self.end:
                raise ThriftError("double runs past the end")
            v = _struct.unpack_from("<d", self.buf, self.pos)[0]
            self.pos += 8
            return v
        if ttype == BINARY:
            n = self._varint()
            if self.pos + n > self.end:
                raise ThriftError("binary runs past the end")
            v = bytes(self.buf[self.pos:self.pos + n])
            self.pos += n
            return v
        if ttype in (LIST, SET):
            h = self._byte()
            n = h >> 4
            et = h & 0x0F
            if n == 15:
                n = self._varint()
            return [self._value(et, depth + 1) for _ in range(n)]
        if ttype == MAP:
            n = self._varint()
            if n == 0:
                return {}
            kv = self._byte()
            return {self._value(kv >> 4, depth + 1): self._value(kv & 0xF, depth + 1) for _ in range(n)}
        if ttype == STRUCT:
            return self.struct(depth + 1)
        raise ThriftError(f"unknown compact type {ttype}")

    def struct(self, depth: int = 0) -> dict:
        if depth > self.max_depth:
            raise ThriftError("structs nested too deeply")
        out = {}
        last = 0
        while True:
            h = self._byte()
            if h == STOP:
                return out
            ttype = h & 0x0F
            delta = h >> 4
            fid = last + delta if delta else unzigzag(self._varint())
            if ttype == BOOL_TRUE:
                out[fid] = True
            elif ttype == BOOL_FALSE:
                out[fid] = False
            else:
                out[fid] = self._value(ttype, depth)
            last = fid


def decode_struct(buf, pos: int = 0, end: int = None):
    """Returns (dict, end_position)."""
    r = Reader(buf, pos, end)
    d = r.struct()
    return d, r.pos
