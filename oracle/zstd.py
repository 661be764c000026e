"""Zstandard frame decompression (test infrastructure only).

The paper's Section 2 names Zstandard among the codecs Parquet applies per
column chunk.  This module follows the Zstandard format definition (frames,
blocks, literals and sequences sections, FSE and Huffman entropy coding)
step by step in the format's own order, one symbol at a time:

* frame: magic 0xFD2FB528, frame header (content-size, single-segment,
  checksum and dictionary-id flags; window descriptor; content size), then
  blocks until the last-block bit, then an optional 4-byte checksum (skipped,
  as the format allows); skippable frames (magic 0x184D2A5?) are skipped;
* block: 3-byte header (last bit, type, size); raw, RLE or compressed;
* compressed block: literals section (raw, RLE, Huffman-coded with a new or
  the previous table, one or four streams) + sequences section (literal
  length, offset and match length codes, each coded with the predefined,
  an RLE, a transmitted or the previous FSE table; extra bits; three repeat
  offsets), then the sequences are executed against the frame's output.

Dictionaries are not supported (Parquet does not use them).  Every
structural inconsistency raises ZstdError.
"""
from __future__ import annotations

MAGIC = 0xFD2FB528


class ZstdError(ValueError):
    pass


# ------------------------------------------------------------------ tables of the format

# Literal length codes 0..35: (baseline, extra bits).
LL_CODES = [(i, 0) for i in range(16)] + [
    (16, 1), (18, 1), (20, 1), (22, 1), (24, 2), (28, 2), (32, 3), (40, 3), (48, 4), (64, 6), (128, 7),
    (256, 8), (512, 9), (1024, 10), (2048, 11), (4096, 12), (8192, 13), (16384, 14), (32768, 15), (65536, 16)]
# Match length codes 0..52: (baseline, extra bits).
ML_CODES = [(i + 3, 0) for i in range(32)] + [
    (35, 1), (37, 1), (39, 1), (41, 1), (43, 2), (47, 2), (51, 3), (59, 3), (67, 4), (83, 4), (99, 5),
    (131, 7), (259, 8), (515, 9), (1027, 10), (2051, 11), (4099, 12), (8195, 13), (16387, 14), (32771, 15),
    (65539, 16)]
# Predefined distributions (normalized counts, -1 = "less than one") and
# their accuracy logs.
LL_DEFAULT = ([4, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 3, 2, 1, 1, 1, 1, 1,
               -1, -1, -1, -1], 6)
ML_DEFAULT = ([1, 4, 3, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
               1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1, -1, -1], 6)
OF_DEFAULT = ([1, 1, 1, 1, 1, 1, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1], 5)
LL_MAX_AL, ML_MAX_AL, OF_MAX_AL, HUF_WEIGHT_MAX_AL = 9, 9, 8, 6
MAX_BLOCK = 128 * 1024


# ------------------------------------------------------------------ bit readers

class ForwardBits:
    """Little-endian bit reader from the start of buf[pos:end] (FSE table
    descriptions): bit i of the stream is bit (i % 8) of byte i // 8."""

    def __init__(self, buf, pos, end):
        self.buf, self.start, self.end = buf, pos, end
        self.bit = 0

    def peek(self, n):
        lo = self.start + (self.bit >> 3)
        hi = min(self.end, self.start + ((self.bit + n + 7) >> 3))
        v = int.from_bytes(bytes(self.buf[lo:hi]), "little") >> (self.bit & 7)
        return v & ((1 << n) - 1)

    def skip(self, n):
        self.bit += n
        if self.start + ((self.bit + 7) >> 3) > self.end:
            raise ZstdError("table description runs past its bytes")

    def read(self, n):
        v = self.peek(n)
        self.skip(n)
        return v

    def bytes_used(self):
        return (self.bit + 7) >> 3


class BackwardBits:
    """Reader of a stream written backwards: the last byte holds a 1 marker
    bit above the data; reading starts just below it and walks towards the
    first byte, the earlier bits of each field being the more significant.
    Past the first byte the stream reads as zeros (`pos` then goes below 0)."""

    def __init__(self, buf, start, end):
        if end <= start:
            raise ZstdError("empty bitstream")
        last = buf[end - 1]
        if last == 0:
            raise ZstdError("bitstream without its end marker")
        self.buf, self.start = buf, start
        self.pos = (end - start - 1) * 8 + last.bit_length() - 1

    def peek(self, n):
        if n == 0:
            return 0
        lo_bit = self.pos - n
        if self.pos <= 0:
            return 0
        if lo_bit < 0:
            return self._bits(0, self.pos) << (-lo_bit)
        return self._bits(lo_bit, n)

    def _bits(self, lo_bit, n):
        b0 = self.start + (lo_bit >> 3)
        b1 = self.start + ((lo_bit + n - 1) >> 3)
        v = int.from_bytes(bytes(self.buf[b0:b1 + 1]), "little") >> (lo_bit & 7)
        return v & ((1 << n) - 1)

    def read(self, n):
        v = self.peek(n)
        self.pos -= n
        return v

    def overflowed(self):
        return self.pos < 0


# ------------------------------------------------------------------ FSE

def read_fse_description(buf, pos, end, max_al, n_symbols_max):
    """Normalized counts of an FSE table description at buf[pos:end].
    Returns (counts, accuracy log, bytes used)."""
    br = ForwardBits(buf, pos, end)
    al = br.read(4) + 5
    if al > max_al:
        raise ZstdError("FSE accuracy log too large")
    remaining = 1 << al
    counts = []
    while remaining > 0:
        if len(counts) >= n_symbols_max:
            raise ZstdError("too many FSE symbols")
        # values 0 .. remaining + 1 (probability + 1); the smallest ones take a bit less
        n_values = remaining + 2
        nbits = n_values.bit_length()          # 2^nbits > n_values - 1
        if (1 << (nbits - 1)) >= n_values:
            nbits -= 1
        spare = (1 << nbits) - n_values
        low = br.peek(nbits - 1)
        if low < spare:
            value = low
            br.skip(nbits - 1)
        else:
            value = br.peek(nbits)
            if value >= (1 << (nbits - 1)):
                value -= spare
            br.skip(nbits)
        prob = value - 1
        counts.append(prob)
        remaining -= 1 if prob == -1 else prob
        if prob == 0:
            # 2-bit repeat flags: how many more zero probabilities follow
            while True:
                rep = br.read(2)
                counts.extend([0] * rep)
                if len(counts) > n_symbols_max:
                    raise ZstdError("too many FSE symbols")
                if rep != 3:
                    break
    if remaining < 0:
        raise ZstdError("FSE probabilities exceed the table")
    return counts, al, br.bytes_used()


class FseTable:
    """Decoding table of one FSE distribution: per state, its symbol, the
    bits to read and the base of the next state."""

    def __init__(self, counts, al):
        size = 1 << al
        self.al = al
        sym = [0] * size
        high = size - 1
        nxt = [0] * len(counts)
        for s, c in enumerate(counts):
            if c == -1:
                sym[high] = s
                high -= 1
                nxt[s] = 1
            else:
                nxt[s] = c
        pos, step, mask = 0, (size >> 1) + (size >> 3) + 3, size - 1
        for s, c in enumerate(counts):
            for _ in range(max(c, 0)):
                sym[pos] = s
                pos = (pos + step) & mask
                while pos > high:
                    pos = (pos + step) & mask
        if pos != 0:
            raise ZstdError("FSE counts do not fill the table")
        self.sym, self.nbits, self.base = sym, [0] * size, [0] * size
        for st in range(size):
            s = sym[st]
            x = nxt[s]
            nxt[s] += 1
            nb = al - (x.bit_length() - 1)
            self.nbits[st] = nb
            self.base[st] = (x << nb) - size

    @staticmethod
    def rle(symbol):
        t = FseTable.__new__(FseTable)
        t.al, t.sym, t.nbits, t.base = 0, [symbol], [0], [0]
        return t


# ------------------------------------------------------------------ Huffman

class HufTable:
    """Prefix-code table from the symbols' weights: number of bits =
    max_bits + 1 - weight; codes handed out from the longest (lowest
    weight) up, symbols in increasing order within a weight."""

    def __init__(self, weights):
        total = sum(1 << (w - 1) for w in weights if w > 0)
        if total == 0:
            raise ZstdError("Huffman weights are all zero")
        max_bits = total.bit_length()
        rest = (1 << max_bits) - total
        if rest & (rest - 1):
            raise ZstdError("Huffman weights do not sum to a power of two")
        weights = list(weights) + [rest.bit_length()]   # the implied last weight
        if max_bits > 11 or len(weights) > 256:
            raise ZstdError("Huffman table too large")
        self.max_bits = max_bits
        self.nbits = [max_bits + 1 - w if w > 0 else 0 for w in weights]
        self.table = []
        for w in range(1, max_bits + 1):
            for s, ws in enumerate(weights):
                if ws == w:
                    self.table.extend([s] * (1 << (w - 1)))
        if len(self.table) != 1 << max_bits:
            raise ZstdError("Huffman codes do not fill the table")

    def decode_stream(self, buf, start, end, count):
        br = BackwardBits(buf, start, end)
        out = bytearray()
        for _ in range(count):
            s = self.table[br.peek(self.max_bits)]
            br.read(self.nbits[s])
            out.append(s)
        if br.pos != 0:
            raise ZstdError("Huffman stream not consumed exactly")
        return out


def read_huffman_description(buf, pos, end):
    """Returns (HufTable, bytes used)."""
    if pos >= end:
        raise ZstdError("missing Huffman tree description")
    head = buf[pos]
    if head >= 128:
        n = head - 127
        nbytes = (n + 1) // 2
        if pos + 1 + nbytes > end:
            raise ZstdError("Huffman weights run past the block")
        weights = []
        for i in range(n):
            b = buf[pos + 1 + i // 2]
            weights.append(b >> 4 if i % 2 == 0 else b & 15)
        return HufTable(weights), 1 + nbytes
    size = head
    if pos + 1 + size > end or size == 0:
        raise ZstdError("Huffman weights run past the block")
    counts, al, used = read_fse_description(buf, pos + 1, pos + 1 + size, HUF_WEIGHT_MAX_AL, 256)
    t = FseTable(counts, al)
    br = BackwardBits(buf, pos + 1 + used, pos + 1 + size)
    s1, s2 = br.read(al), br.read(al)
    weights = []
    while True:
        if len(weights) > 254:
            raise ZstdError("too many Huffman weights")
        weights.append(t.sym[s1])
        s1 = t.base[s1] + br.read(t.nbits[s1])
        if br.overflowed():
            weights.append(t.sym[s2])
            break
        weights.append(t.sym[s2])
        s2 = t.base[s2] + br.read(t.nbits[s2])
        if br.overflowed():
            weights.append(t.sym[s1])
            break
    if any(w > 11 for w in weights):
        raise ZstdError("Huffman weight above 11")
    return HufTable(weights), 1 + size


# ------------------------------------------------------------------ blocks

class FrameState:
    def __init__(self):
        self.huf = None
        self.tables = {"LL": None, "OF": None, "ML": None}
        self.rep = [1, 4, 8]


def decode_literals(buf, pos, end, st: FrameState):
    """Returns (literals, position after the literals section)."""
    if pos >= end:
        raise ZstdError("missing literals section")
    b0 = buf[pos]
    ltype, sf = b0 & 3, (b0 >> 2) & 3
    if ltype in (0, 1):
        if sf in (0, 2):
            regen, hlen = b0 >> 3, 1
        elif sf == 1:
            regen, hlen = (b0 >> 4) + (buf[pos + 1] << 4), 2
        else:
            regen, hlen = (b0 >> 4) + (buf[pos + 1] << 4) + (buf[pos + 2] << 12), 3
        pos += hlen
        if ltype == 0:
            if pos + regen > end:
                raise ZstdError("raw literals run past the block")
            return bytes(buf[pos:pos + regen]), pos + regen
        if pos >= end:
            raise ZstdError("missing RLE literal byte")
        return bytes([buf[pos]]) * regen, pos + 1
    bits, hlen, streams = {0: (10, 3, 1), 1: (10, 3, 4), 2: (14, 4, 4), 3: (18, 5, 4)}[sf]
    if pos + hlen > end:
        raise ZstdError("literals header runs past the block")
    h = int.from_bytes(bytes(buf[pos:pos + hlen]), "little")
    regen = (h >> 4) & ((1 << bits) - 1)
    csize = (h >> (4 + bits)) & ((1 << bits) - 1)
    pos += hlen
    if pos + csize > end:
        raise ZstdError("compressed literals run past the block")
    cend = pos + csize
    if ltype == 2:
        st.huf, used = read_huffman_description(buf, pos, cend)
        pos += used
    elif st.huf is None:
        raise ZstdError("treeless literals without a previous Huffman table")
    if streams == 1:
        return bytes(st.huf.decode_stream(buf, pos, cend, regen)), cend
    if pos + 6 > cend:
        raise ZstdError("missing jump table")
    s1, s2, s3 = (int.from_bytes(bytes(buf[pos + 2 * i:pos + 2 * i + 2]), "little") for i in range(3))
    p = pos + 6
    bounds = [p, p + s1, p + s1 + s2, p + s1 + s2 + s3, cend]
    if bounds[3] > cend:
        raise ZstdError("jump table points past the literals")
    per = (regen + 3) // 4
    counts = [per, per, per, regen - 3 * per]
    if counts[3] < 0:
        raise ZstdError("literal count too small for four streams")
    out = bytearray()
    for i in range(4):
        out += st.huf.decode_stream(buf, bounds[i], bounds[i + 1], counts[i])
    return bytes(out), cend


def _table(buf, pos, end, mode, name, st: FrameState):
    default, max_al, nsym = {"LL": (LL_DEFAULT, LL_MAX_AL, 36), "OF": (OF_DEFAULT, OF_MAX_AL, 32),
                             "ML": (ML_DEFAULT, ML_MAX_AL, 53)}[name]
    if mode == 0:
        t, used = FseTable(*default), 0
    elif mode == 1:
        if pos >= end:
            raise ZstdError("missing RLE symbol")
        if buf[pos] >= nsym:
            raise ZstdError("RLE symbol out of range")
        t, used = FseTable.rle(buf[pos]), 1
    elif mode == 2:
        counts, al, used = read_fse_description(buf, pos, end, max_al, nsym)
        t = FseTable(counts, al)
    else:
        if st.tables[name] is None:
            raise ZstdError("repeat mode without a previous table")
        t, used = st.tables[name], 0
    st.tables[name] = t
    return t, pos + used


def decode_sequences(buf, pos, end, st: FrameState):
    """[(literal length, offset, match length)]."""
    if pos >= end:
        raise ZstdError("missing sequences section")
    b0 = buf[pos]
    if b0 == 0:
        if pos + 1 != end:
            raise ZstdError("bytes after an empty sequences section")
        return []
    if b0 < 128:
        nseq, pos = b0, pos + 1
    elif b0 < 255:
        nseq, pos = ((b0 - 128) << 8) + buf[pos + 1], pos + 2
    else:
        nseq, pos = buf[pos + 1] + (buf[pos + 2] << 8) + 0x7F00, pos + 3
    if pos >= end:
        raise ZstdError("missing symbol compression modes")
    modes = buf[pos]
    pos += 1
    if modes & 3:
        raise ZstdError("reserved bits of the compression modes set")
    ll_t, pos = _table(buf, pos, end, modes >> 6, "LL", st)
    of_t, pos = _table(buf, pos, end, (modes >> 4) & 3, "OF", st)
    ml_t, pos = _table(buf, pos, end, (modes >> 2) & 3, "ML", st)
    br = BackwardBits(buf, pos, end)
    ll_s, of_s, ml_s = br.read(ll_t.al), br.read(of_t.al), br.read(ml_t.al)
    seqs = []
    for i in range(nseq):
        of_code, ml_code, ll_code = of_t.sym[of_s], ml_t.sym[ml_s], ll_t.sym[ll_s]
        if of_code > 31 or ll_code >= len(LL_CODES) or ml_code >= len(ML_CODES):
            raise ZstdError("sequence code out of range")
        of_value = (1 << of_code) + br.read(of_code)
        ml = ML_CODES[ml_code][0] + br.read(ML_CODES[ml_code][1])
        ll = LL_CODES[ll_code][0] + br.read(LL_CODES[ll_code][1])
        seqs.append((ll, of_value, ml))
        if i + 1 < nseq:
            ll_s = ll_t.base[ll_s] + br.read(ll_t.nbits[ll_s])
            ml_s = ml_t.base[ml_s] + br.read(ml_t.nbits[ml_s])
            of_s = of_t.base[of_s] + br.read(of_t.nbits[of_s])
    if br.pos != 0:
        raise ZstdError("sequence bitstream not consumed exactly")
    return seqs


def execute_sequences(out: bytearray, literals, seqs, st: FrameState):
    """Appends the block's bytes to the frame output `out`."""
    lp = 0
    rep = st.rep
    for ll, ov, ml in seqs:
        if lp + ll > len(literals):
            raise ZstdError("sequence takes more literals than the block has")
        out += literals[lp:lp + ll]
        lp += ll
        if ov > 3:
            off = ov - 3
            rep[:] = [off, rep[0], rep[1]]
        else:
            idx = ov - 1 if ll > 0 else ov      # with no literals the repeat index shifts by one
            if idx == 0:
                off = rep[0]
            elif idx == 1:
                off = rep[1]
                rep[:] = [off, rep[0], rep[2]]
            elif idx == 2:
                off = rep[2]
                rep[:] = [off, rep[0], rep[1]]
            else:
                off = rep[0] - 1
                rep[:] = [off, rep[0], rep[1]]
        if off <= 0 or off > len(out):
            raise ZstdError("match offset reaches before the frame")
        src = len(out) - off
        for k in range(ml):              # byte by byte: the match may overlap its own output
            out.append(out[src + k])
    out += literals[lp:]


def decompress_frame(buf, pos):
    """One frame (or a skippable frame) at pos.  Returns (bytes, end)."""
    magic = int.from_bytes(bytes(buf[pos:pos + 4]), "little")
    if 0x184D2A50 <= magic <= 0x184D2A5F:
        size = int.from_bytes(bytes(buf[pos + 4:pos + 8]), "little")
        if pos + 8 + size > len(buf):
            raise ZstdError("skippable frame runs past the input")
        return b"", pos + 8 + size
    if magic != MAGIC:
        raise ZstdError("not a Zstandard frame")
    pos += 4
    fhd = buf[pos]
    pos += 1
    fcs_flag, single, checksum, dict_flag = fhd >> 6, (fhd >> 5) & 1, (fhd >> 2) & 1, fhd & 3
    if fhd & 8:
        raise ZstdError("reserved frame header bit set")
    if not single:
        pos += 1                          # window descriptor (the output is kept whole)
    dict_len = (0, 1, 2, 4)[dict_flag]
    if dict_len and int.from_bytes(bytes(buf[pos:pos + dict_len]), "little") != 0:
        raise ZstdError("dictionaries are not supported")
    pos += dict_len
    fcs_len = (1 if single else 0, 2, 4, 8)[fcs_flag]
    content_size = None
    if fcs_len:
        content_size = int.from_bytes(bytes(buf[pos:pos + fcs_len]), "little") + (256 if fcs_len == 2 else 0)
        pos += fcs_len
    st = FrameState()
    out = bytearray()
    while True:
        if pos + 3 > len(buf):
            raise ZstdError("block header runs past the input")
        h = int.from_bytes(bytes(buf[pos:pos + 3]), "little")
        pos += 3
        last, btype, bsize = h & 1, (h >> 1) & 3, h >> 3
        if btype == 0:
            if pos + bsize > len(buf):
                raise ZstdError("raw block runs past the input")
            out += buf[pos:pos + bsize]
            pos += bsize
        elif btype == 1:
            if pos >= len(buf):
                raise ZstdError("RLE block without its byte")
            out += bytes([buf[pos]]) * bsize
            pos += 1
        elif btype == 2:
            if bsize > MAX_BLOCK or pos + bsize > len(buf):
                raise ZstdError("compressed block too large or past the input")
            end = pos + bsize
            literals, p = decode_literals(buf, pos, end, st)
            seqs = decode_sequences(buf, p, end, st)
            execute_sequences(out, literals, seqs, st)
            pos = end
        else:
            raise ZstdError("reserved block type")
        if last:
            break
    if checksum:
        pos += 4
    if content_size is not None and content_size != len(out):
        raise ZstdError("frame content size differs from the decoded bytes")
    return bytes(out), pos


def decompress(data) -> bytes:
    """All frames of `data`, concatenated."""
    buf = bytes(data)
    out = bytearray()
    pos = 0
    while pos < len(buf):
        part, pos = decompress_frame(buf, pos)
        out += part
    return bytes(out)


# ------------------------------------------------------------------ a store-only encoder

def compress_stored(data, block=MAX_BLOCK) -> bytes:
    """A valid frame holding `data` in raw blocks (runs of one byte as RLE
    blocks): no entropy coding, for writers that need Zstandard pages."""
    data = bytes(data)
    n = len(data)
    out = bytearray(MAGIC.to_bytes(4, "little"))
    out.append(0xE0 if n > 0xFFFFFFFF else 0xA0)   # 8- or 4-byte content size, single segment
    out += n.to_bytes(8 if n > 0xFFFFFFFF else 4, "little")
    pos = 0
    while True:
        chunk = data[pos:pos + block]
        last = 1 if pos + len(chunk) >= n else 0
        if chunk and chunk.count(chunk[0]) == len(chunk):
            out += ((len(chunk) << 3) | (1 << 1) | last).to_bytes(3, "little") + chunk[:1]
        else:
            out += ((len(chunk) << 3) | last).to_bytes(3, "little") + chunk
        pos += len(chunk)
        if last:
            break
    return bytes(out)
