"""Pins of the CPU oracle against hand-worked byte vectors, closed forms
and brute force (no GPU).  The oracle itself is test infrastructure; these
tests check it against things other than itself."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import byte_stream_split, delta, delta_strings, hybrid, snappy, thrift, zstd
from oracle import reader as R

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_vectors.json")))


def hx(s):
    return bytes.fromhex(s.replace(" ", ""))


# ------------------------------------------------------------------ thrift

def test_page_header_hand_vector_decode():
    g = GOLD["page_header_v1"]
    p = R.parse_page_header(hx(g["hex"]), 0, len(hx(g["hex"])))
    v = g["value"]
    assert (p.page_type, p.uncompressed, p.compressed) == (v["type"], v["uncompressed_page_size"], v["compressed_page_size"])
    d = v["data_page_header"]
    assert (p.num_values, p.encoding) == (d["num_values"], d["encoding"])
    assert p.header_len == 19


def test_page_header_hand_vector_encode():
    g = GOLD["page_header_v1"]
    enc = thrift.encode_struct([(1, thrift.I32, 0), (2, thrift.I32, 100), (3, thrift.I32, 100),
                                (5, thrift.STRUCT, [(1, thrift.I32, 8), (2, thrift.I32, 0),
                                                    (3, thrift.I32, 3), (4, thrift.I32, 3)])])
    assert enc == hx(g["hex"])


@pytest.mark.parametrize("n,zz", [(0, 0), (-1, 1), (1, 2), (-2, 3), (2, 4), (2**31 - 1, 2**32 - 2),
                                  (-2**31, 2**32 - 1), (-2**63, 2**64 - 1)])
def test_zigzag_closed_form(n, zz):
    assert thrift.zigzag(n) == zz
    assert thrift.unzigzag(zz) == n


@pytest.mark.parametrize("n,enc", [(0, "00"), (1, "01"), (127, "7F"), (128, "80 01"), (300, "AC 02"),
                                   (2**64 - 1, "FF FF FF FF FF FF FF FF FF 01")])
def test_uleb128_closed_form(n, enc):
    assert thrift.uleb128(n) == hx(enc)
    assert thrift.read_uleb128(hx(enc), 0) == (n, len(hx(enc)))


def test_thrift_long_field_delta_and_list_header():
    # field id jump of 16 forces the long form: type byte then zigzag id
    enc = thrift.encode_struct([(1, thrift.I32, 5), (17, thrift.I64, -1)])
    assert enc == hx("15 0A 06 22 01 00")
    d, end = thrift.decode_struct(enc)
    assert d == {1: 5, 17: -1} and end == len(enc)
    # list of 20 i32: header 0xF5 + ULEB size
    enc = thrift.encode_struct([(1, thrift.LIST, (thrift.I32, list(range(20))))])
    assert enc[:3] == hx("19 F5 14")
    assert thrift.decode_struct(enc)[0] == {1: list(range(20))}


def test_thrift_bool_fields_and_truncation():
    enc = thrift.encode_struct([(1, thrift.BOOL_TRUE, True), (2, thrift.BOOL_TRUE, False)])
    assert enc == hx("11 12 00")
    assert thrift.decode_struct(enc)[0] == {1: True, 2: False}
    with pytest.raises(thrift.ThriftError):
        thrift.decode_struct(enc[:-1])


# ------------------------------------------------------------------ hybrid

def _bigint_unpack(data, bit_offset, count, width):
    """An independent statement of LSB-first packing: the stream is one
    little-endian integer; value i is bits [i*w, (i+1)*w) of it."""
    big = int.from_bytes(bytes(data), "little")
    return [(big >> (bit_offset + i * width)) & ((1 << width) - 1) for i in range(count)]


def test_hybrid_hand_vectors():
    g = GOLD["hybrid_bitpacked_bw3"]
    vals, end = hybrid.decode(hx(g["hex"]), 0, 4, 3, 8)
    assert vals.tolist() == g["values"] and end == 4
    assert hybrid.encode(g["values"], 3, "packed") == hx(g["hex"])
    g = GOLD["hybrid_rle_bw3"]
    vals, _ = hybrid.decode(hx(g["hex"]), 0, 3, 3, 100)
    assert vals.tolist() == [5] * 100
    assert hybrid.encode([5] * 100, 3, "default") == hx(g["hex"])
    g = GOLD["def_levels_v1"]
    b = hx(g["hex"])
    n = int.from_bytes(b[:4], "little")
    vals, _ = hybrid.decode(b, 4, 4 + n, 1, 8)
    assert vals.tolist() == g["values"]


@pytest.mark.parametrize("width", [0, 1, 2, 3, 4])
def test_hybrid_brute_force_small(width):
    """Every sequence of length <= 6 over an alphabet of up to 3 symbols (or
    the whole range for width <= 1): every writer policy decodes back."""
    alphabet = list(range(min(3, 1 << width))) if width else [0]
    rng = np.random.default_rng(width)
    for n in range(0, 7):
        for seq in itertools.product(alphabet, repeat=n):
            for pol in ("default", "rle", "packed", "mixed"):
                enc = hybrid.encode(seq, width, pol, rng)
                dec, end = hybrid.decode(enc, 0, len(enc), width, n)
                assert dec.tolist() == list(seq), (seq, pol)
                assert end == len(enc) or n == 0


@pytest.mark.parametrize("width", [1, 5, 7, 10, 13, 20, 31, 32, 33, 63, 64])
def test_bitpack_against_bigint_definition(width):
    rng = np.random.default_rng(width)
    vals = rng.integers(0, 2**63, size=77, dtype=np.uint64) & np.uint64((1 << width) - 1 if width < 64 else 2**64 - 1)
    if width == 64:
        vals = vals | np.uint64(1 << 63)
    packed = hybrid.pack_lsb(vals, width)
    assert len(packed) == (77 * width + 7) // 8
    for off in (0, width * 3):
        got = hybrid.unpack_lsb(packed, off, 77 - off // width if width else 77, width)
        assert got.tolist() == _bigint_unpack(packed, off, len(got), width)
    assert hybrid.unpack_lsb(packed, 0, 77, width).tolist() == [int(v) for v in vals]


def test_hybrid_padding_ignored_and_errors():
    # 3 values bit-packed in one padded group; trailing pad is ignored
    enc = hybrid.encode([1, 0, 1], 1, "packed")
    assert hybrid.decode(enc, 0, len(enc), 1, 3)[0].tolist() == [1, 0, 1]
    with pytest.raises(hybrid.HybridError):
        hybrid.decode(hx("05 FF"), 0, 2, 1, 16)   # 2 groups announced, 1 byte present
    with pytest.raises(ValueError):
        hybrid.decode(hx("04"), 0, 1, 3, 2)       # repeated value missing
    with pytest.raises(hybrid.HybridError):
        hybrid.decode(hx("04 09"), 0, 2, 3, 2)    # repeated value wider than 3 bits


# ------------------------------------------------------------------ delta

def test_delta_hand_vectors():
    for key in ("delta_int32_descending", "delta_single_value"):
        g = GOLD[key]
        b = hx(g["hex"])
        vals, end = delta.decode(b, 0, len(b), g["bits"])
        assert vals == g["values"] and end == len(b)
        assert delta.encode(g["values"], g["bits"]) == b


@pytest.mark.parametrize("bits", [32, 64])
def test_delta_wraparound_extremes(bits):
    lo, hi = -(1 << (bits - 1)), (1 << (bits - 1)) - 1
    seqs = [[lo, hi, lo, hi], [hi, lo, 0, -1, hi], [0, hi, hi, lo, lo, 0], [lo] * 300, list(range(hi - 200, hi + 1))]
    for s in seqs:
        enc = delta.encode(s, bits)
        assert delta.decode(enc, 0, len(enc), bits)[0] == s


def test_delta_sorted_keys_and_random():
    rng = np.random.default_rng(7)
    for n in (0, 1, 2, 31, 32, 33, 127, 128, 129, 130, 1000, 4097):
        for bits in (32, 64):
            s = np.cumsum(rng.integers(0, 8, size=n)).tolist()
            r = rng.integers(-(1 << (bits - 1)), (1 << (bits - 1)), size=n, dtype=np.int64).tolist()
            for seq in (s, r):
                enc = delta.encode(seq, bits)
                assert delta.decode(enc, 0, len(enc), bits)[0] == seq


def test_delta_block_structure_closed_form():
    # 1 + 128*2 values with constant step 3: min delta 3, all packed deltas 0,
    # so each block is zigzag(3)=1 byte + 4 zero width bytes, no bodies.
    seq = [10 + 3 * i for i in range(257)]
    enc = delta.encode(seq, 64)
    assert enc == hx("80 01 04 81 02 14") + (hx("06 00 00 00 00") * 2)


def test_delta_errors():
    with pytest.raises(delta.DeltaError):
        delta.decode(hx("81 01 04 02 00"), 0, 5, 32)      # block size 129
    with pytest.raises(delta.DeltaError):
        delta.decode(hx("80 01 04 02 00 00 21 00 00 00"), 0, 10, 32)  # width 33 on INT32
    with pytest.raises(ValueError):
        delta.decode(hx("80 01 04 03 00 00 01 00 00 00"), 0, 10, 32)  # body missing


# ------------------------------------------------------------------ snappy

def test_snappy_hand_vectors():
    for key in ("snappy_copy2", "snappy_copy1"):
        g = GOLD[key]
        assert snappy.decompress(hx(g["hex"])) == g["text"].encode()


def test_snappy_brute_force_short_strings():
    for n in range(0, 9):
        for t in itertools.product(b"ab", repeat=n):
            s = bytes(t)
            for enc in (snappy.compress(s), snappy.compress(s, allow_copy1=False),
                        snappy.compress_literal_only(s)):
                assert snappy.decompress(enc) == s


def test_snappy_long_literals_and_far_copies():
    rng = np.random.default_rng(3)
    blob = rng.integers(0, 256, size=70000, dtype=np.uint8).tobytes()
    data = blob + b"x" * 100 + blob[:5000]       # copy with offset > 65535
    enc = snappy.compress(data)
    assert snappy.decompress(enc) == data
    assert any(enc[i] & 3 == 3 for i in range(len(enc)))  # some 4-byte-offset copy
    lit = snappy.compress_literal_only(blob)
    assert snappy.decompress(lit) == blob


def test_snappy_errors():
    with pytest.raises(snappy.SnappyError):
        snappy.decompress(hx("04 01 05 00"))          # copy before any output
    with pytest.raises(snappy.SnappyError):
        snappy.decompress(hx("05 0C 61 62 63 64"))    # shorter than declared
    with pytest.raises(snappy.SnappyError):
        snappy.decompress(hx("02 0C 61 62 63 64"))    # longer than declared


# ------------------------------------------------------------------ byte stream split

def test_byte_stream_split_hand_vectors():
    for key in ("bss_double", "bss_int32"):
        g = GOLD[key]
        b = hx(g["hex"])
        got = byte_stream_split.decode(b, 0, len(b), g["ptype"], len(g["values"]))
        assert got.tolist() == g["values"]
        assert byte_stream_split.encode(g["values"], g["ptype"]) == b


@pytest.mark.parametrize("ptype,dtype", [("INT32", "<i4"), ("INT64", "<i8"), ("DOUBLE", "<f8")])
def test_byte_stream_split_is_a_byte_transpose(ptype, dtype):
    # special case reducing to a library routine: the streams are the K x N
    # transpose of the N x K little-endian byte matrix of the values
    rng = np.random.default_rng(17)
    for n in (0, 1, 7, 33, 1000):
        raw = rng.integers(0, 256, size=n * np.dtype(dtype).itemsize, dtype=np.uint8)
        vals = raw.view(dtype)
        k = np.dtype(dtype).itemsize
        streams = raw.reshape(n, k).T.copy().tobytes()
        assert byte_stream_split.encode(vals, ptype) == streams
        got = byte_stream_split.decode(streams, 0, len(streams), ptype, n)
        assert got.view(np.uint8).tobytes() == raw.tobytes()


def test_byte_stream_split_nulls_and_errors():
    b = hx(GOLD["bss_int32"]["hex"])
    # an OPTIONAL page reads the first values of full-length streams
    assert byte_stream_split.decode(b, 0, len(b), "INT32", 2).tolist() == GOLD["bss_int32"]["values"][:2]
    with pytest.raises(byte_stream_split.ByteStreamSplitError):
        byte_stream_split.decode(b, 0, len(b) - 1, "INT32", 2)   # not a whole number of values
    with pytest.raises(byte_stream_split.ByteStreamSplitError):
        byte_stream_split.decode(b, 0, len(b), "INT32", 4)       # more values than the streams hold


# ------------------------------------------------------------------ delta strings

def test_delta_length_byte_array_hand_vector():
    g = GOLD["delta_length_byte_array"]
    b = hx(g["hex"])
    vals, end = delta_strings.decode_length_byte_array(b, 0, len(b), len(g["strings"]))
    assert vals == [x.encode() for x in g["strings"]] and end == len(b)
    assert delta_strings.encode_length_byte_array([x.encode() for x in g["strings"]]) == b


def test_delta_byte_array_hand_vector():
    g = GOLD["delta_byte_array"]
    b = hx(g["hex"])
    vals, end = delta_strings.decode_byte_array(b, 0, len(b), len(g["strings"]))
    assert vals == [x.encode() for x in g["strings"]] and end == len(b)
    assert delta_strings.encode_byte_array([x.encode() for x in g["strings"]]) == b


def test_delta_strings_brute_force_small():
    # every sequence of up to 4 strings over {'', a, b, aa, ab, ba, aab}
    words = [b"", b"a", b"b", b"aa", b"ab", b"ba", b"aab"]
    for n in range(0, 5):
        for seq in itertools.product(words, repeat=n):
            seq = list(seq)
            e1 = delta_strings.encode_length_byte_array(seq)
            assert delta_strings.decode_length_byte_array(e1, 0, len(e1), n) == (seq, len(e1))
            e2 = delta_strings.encode_byte_array(seq)
            assert delta_strings.decode_byte_array(e2, 0, len(e2), n) == (seq, len(e2))


def test_delta_byte_array_without_shared_prefixes_is_length_encoding():
    # strings with distinct first bytes share no prefix: the stream is a
    # zero prefix stream followed by the DELTA_LENGTH_BYTE_ARRAY of the values
    seq = [b"x1", b"y22", b"z", b"w4444"]
    zeros = delta.encode([0, 0, 0, 0], 32)
    assert delta_strings.encode_byte_array(seq) == zeros + delta_strings.encode_length_byte_array(seq)
    assert zeros == hx("80 01 04 04 00") + hx("00 00 00 00 00")


def test_delta_strings_long_shared_prefixes():
    rng = np.random.default_rng(23)
    stem = bytes(rng.integers(97, 123, size=300, dtype=np.uint8))
    seq = sorted(stem[:int(rng.integers(0, 301))] + bytes(rng.integers(97, 123, size=int(rng.integers(0, 5)),
                                                                       dtype=np.uint8)) for _ in range(700))
    e = delta_strings.encode_byte_array(seq)
    assert delta_strings.decode_byte_array(e, 0, len(e), len(seq))[0] == seq
    assert len(e) < sum(len(x) for x in seq) // 4   # front coding pays on sorted keys


def test_delta_strings_errors():
    ok = delta_strings.encode_byte_array([b"ab", b"ac"])
    with pytest.raises(delta_strings.DeltaStringError):     # count differs from the page
        delta_strings.decode_byte_array(ok, 0, len(ok), 3)
    bad_prefix = delta.encode([0, 3], 32) + delta_strings.encode_length_byte_array([b"ab", b"c"])
    with pytest.raises(delta_strings.DeltaStringError):     # prefix 3 > len('ab')
        delta_strings.decode_byte_array(bad_prefix, 0, len(bad_prefix), 2)
    first_prefix = delta.encode([1, 0], 32) + delta_strings.encode_length_byte_array([b"ab", b"c"])
    with pytest.raises(delta_strings.DeltaStringError):     # first value has no predecessor
        delta_strings.decode_byte_array(first_prefix, 0, len(first_prefix), 2)
    neg = delta.encode([2, -1], 32) + b"ab"
    with pytest.raises(delta_strings.DeltaStringError):     # negative length
        delta_strings.decode_length_byte_array(neg, 0, len(neg), 2)
    short = delta_strings.encode_length_byte_array([b"abc", b"defg"])
    with pytest.raises(delta_strings.DeltaStringError):     # bytes past the end
        delta_strings.decode_length_byte_array(short, 0, len(short) - 1, 2)


# ------------------------------------------------------------------ zstandard

def test_zstd_hand_vectors():
    for key in ("zstd_raw_block", "zstd_rle_literals_no_sequences", "zstd_one_sequence_rle_tables"):
        g = GOLD[key]
        assert zstd.decompress(hx(g["hex"])) == g["text"].encode(), key
    g = GOLD["zstd_rle_block"]
    ch, n = g["text_repeat"]
    assert zstd.decompress(hx(g["hex"])) == ch.encode() * n


def _zstd_inputs(rng):
    """Byte strings of many shapes: random, small alphabets, word soup,
    long runs, integer columns, skewed bytes in blocks of 128 KB (Huffman
    literal sections with 18-bit sizes), several blocks per frame."""
    out = [b"", b"a", bytes(range(256)) * 40]
    for trial in range(120):
        kind = trial % 6
        n = int(rng.integers(0, 300_000 if trial % 13 == 0 else 5000))
        if kind == 0:
            x = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        elif kind == 1:
            x = rng.integers(0, int(rng.integers(1, 6)), n, dtype=np.uint8).tobytes()
        elif kind == 2:
            words = [rng.integers(97, 123, int(rng.integers(1, 12)), dtype=np.uint8).tobytes()
                     for _ in range(int(rng.integers(1, 50)))]
            x = b"".join(words[int(i)] for i in rng.integers(0, len(words), max(1, n // 6)))
        elif kind == 3:
            x = np.repeat(rng.integers(0, 256, max(1, n // 50), dtype=np.uint8), 50).tobytes()
        elif kind == 4:
            x = np.cumsum(rng.integers(-3, 4, max(1, n // 4))).astype(np.int32).tobytes()
        else:
            x = np.minimum(rng.geometric(0.08, 200_000), 255).astype(np.uint8).tobytes()
        out.append(x)
    return out


def test_zstd_against_libzstd():
    """Frames written by libzstd (through pyarrow) at levels -5 .. 22 decode
    to their input: every literal and sequence coding mode of the format
    occurs among them (raw, RLE, Huffman 1 and 4 streams, new and repeated
    tables; predefined, RLE, transmitted and repeated FSE tables; all three
    repeat offsets)."""
    pa = pytest.importorskip("pyarrow")
    rng = np.random.default_rng(1)
    levels = [-5, -1, 1, 2, 3, 5, 9, 15, 19, 22]
    for i, x in enumerate(_zstd_inputs(rng)):
        lvl = levels[i % len(levels)]
        comp = pa.Codec("zstd", compression_level=lvl).compress(x, asbytes=True)
        assert zstd.decompress(comp) == x, (i, lvl, len(x))


def test_zstd_stored_frames_round_trip_and_libzstd_reads_them():
    rng = np.random.default_rng(2)
    cases = [b"", b"z", b"q" * 300_000, rng.integers(0, 256, 300_000, dtype=np.uint8).tobytes()]
    cases += [bytes(t) for n in range(0, 4) for t in itertools.product(b"ab", repeat=n)]
    for x in cases:
        enc = zstd.compress_stored(x)
        assert zstd.decompress(enc) == x
    pa = pytest.importorskip("pyarrow")
    for x in cases[:4]:
        enc = zstd.compress_stored(x)
        assert pa.Codec("zstd").decompress(enc, decompressed_size=len(x), asbytes=True) == x


def test_zstd_frames_concatenate_and_skip():
    a, b = zstd.compress_stored(b"first"), zstd.compress_stored(b"second")
    skip = (0x184D2A53).to_bytes(4, "little") + (3).to_bytes(4, "little") + b"xyz"
    assert zstd.decompress(a + skip + b) == b"firstsecond"


def test_zstd_errors():
    # good: magic | 20 | 0C | 55 00 00 | 18 'abc' | 01 54 03 02 06 | 06
    good = hx(GOLD["zstd_one_sequence_rle_tables"]["hex"])
    bad = [
        b"\x00" + good[1:],                                   # not the magic number
        good[:4] + bytes([good[4] | 8]) + good[5:],           # reserved descriptor bit
        good[:-1],                                            # block runs past the input
        good[:5] + bytes([13]) + good[6:],                    # content size 13, 12 bytes decoded
        good[:6] + bytes([good[6] | 6]) + good[7:],           # reserved block type 3
        good[:18] + b"\x0e",                                  # 3 data bits, 2 read: not consumed exactly
        good[:16] + hx("03 06 08"),                           # offset code 3 + 0: offset 5 > 3 bytes out
        hx("28 B5 2F FD 21 01 03 19 00 00 61 62 63"),         # dictionary id 1
    ]
    for b in bad:
        with pytest.raises(zstd.ZstdError):
            zstd.decompress(b)
