"""The engine's Zstandard decoding core (csrc/zstd_dec.cuh: the host/device
functions its kernel runs) compiled for the CPU with g++ and compared, frame
by frame, with the CPU oracle: hand-worked frames, libzstd frames of many
shapes and levels, every page of the committed Zstandard fixtures, and
malformed frames (an error code, never a crash).  No GPU needed."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import reader as R
from oracle import zstd as Z
from oracle.parquet_meta import DATA_PAGE_V2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def core(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("zstd") / "zstd_core.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                    os.path.join(ROOT, "paper_2602_17335_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "zstd_host_harness.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    lib.zstd_host_decode.argtypes = [ctypes.c_char_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64]
    lib.zstd_host_decode.restype = ctypes.c_int

    def decode(frame, n):
        buf = np.zeros(n + 32, dtype=np.uint8)
        rc = lib.zstd_host_decode(bytes(frame), len(frame), buf.ctypes.data, n)
        return rc, buf[:n].tobytes()
    return decode


def test_hand_worked_frames(core):
    import json
    gold = json.load(open(os.path.join(HERE, "golden", "hand_vectors.json")))
    for key in ("zstd_raw_block", "zstd_rle_block", "zstd_rle_literals_no_sequences", "zstd_one_sequence_rle_tables"):
        frame = bytes.fromhex(gold[key]["hex"].replace(" ", ""))
        want = Z.decompress(frame)
        assert core(frame, len(want)) == (0, want), key


def test_libzstd_frames(core):
    pa = pytest.importorskip("pyarrow")
    from test_oracle_pins import _zstd_inputs
    rng = np.random.default_rng(1)
    levels = [-5, -1, 1, 2, 3, 5, 9, 15, 19, 22]
    for i, x in enumerate(_zstd_inputs(rng)):
        frame = pa.Codec("zstd", compression_level=levels[i % len(levels)]).compress(x, asbytes=True)
        assert core(frame, len(x)) == (0, x), i


@pytest.mark.parametrize("name", ["zstd_eight_column_v1.parquet", "zstd_eight_column_v2.parquet"])
def test_fixture_pages(core, name):
    data = open(os.path.join(HERE, "golden", name), "rb").read()
    n = 0
    for ch in R.parse_footer(data).chunks:
        for p in R.chunk_pages(data, ch):
            body = data[p.offset + p.header_len:p.offset + p.header_len + p.compressed]
            skip = p.def_len + p.rep_len if p.page_type == DATA_PAGE_V2 else 0
            if p.page_type == DATA_PAGE_V2 and not p.is_compressed:
                continue
            frame = body[skip:]
            want = Z.decompress(frame)
            assert len(want) == p.uncompressed - skip
            assert core(frame, len(want)) == (0, want)
            n += 1
    assert n > 20


def test_native_writer_frames(core):
    """Frames of the engine's own writer (sequences under the predefined
    tables, raw and RLE blocks, several blocks per page)."""
    import synth
    from paper_2602_17335_gb300.tables import write_table
    from test_native_writer import _native, zstd_pages
    _native()
    tab = synth.config2_table(200_000, 200_000, string_pool_size=300, zipf_k=500)
    data = bytes(write_table(tab, synth.config2_spec(200_000, 1 << 20, "ZSTD", 2)))
    n = 0
    for _, frame, size in zstd_pages(data):
        want = Z.decompress(frame)
        assert len(want) == size and core(frame, size) == (0, want)
        n += 1
    assert n > 10


def test_malformed_frames_return_errors(core):
    import json
    gold = json.load(open(os.path.join(HERE, "golden", "hand_vectors.json")))
    good = bytes.fromhex(gold["zstd_one_sequence_rle_tables"]["hex"].replace(" ", ""))
    bad = [b"\x00" + good[1:], good[:4] + bytes([good[4] | 8]) + good[5:], good[:-1],
           good[:5] + bytes([13]) + good[6:], good[:6] + bytes([good[6] | 6]) + good[7:], good[:18] + b"\x0e",
           good[:16] + bytes.fromhex("030608"), bytes.fromhex("28B52FFD2101031900006162 63".replace(" ", ""))]
    for b in bad:
        rc, _ = core(b, 12)
        assert rc != 0
    # a page smaller than the frame's output is an error, not an overflow
    assert core(good, 11)[0] != 0
    rng = np.random.default_rng(5)
    pa = pytest.importorskip("pyarrow")
    x = rng.integers(0, 4, 20000, dtype=np.uint8).tobytes()
    frame = bytearray(pa.Codec("zstd", compression_level=3).compress(x, asbytes=True))
    for _ in range(200):   # random byte flips: any result but a crash
        f = bytearray(frame)
        k = int(rng.integers(4, len(f)))
        f[k] ^= 1 << int(rng.integers(0, 8))
        core(bytes(f), len(x))


_FUZZ = r'''
import ctypes, pickle, sys
lib = ctypes.CDLL(sys.argv[1])
lib.zstd_host_decode_exact.argtypes = [ctypes.c_char_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64]
cases = pickle.load(open(sys.argv[2], "rb"))
rejected = 0
for frame, cap in cases:
    buf = (ctypes.c_uint8 * max(cap, 1))()
    rejected += lib.zstd_host_decode_exact(frame, len(frame), buf, cap) != 0
print(len(cases), rejected)
'''


def test_fuzzed_frames_stay_in_bounds_under_asan(tmp_path):
    """Corrupted and truncated libzstd frames, decoded with the input and the
    output in heap blocks of exactly their sizes under AddressSanitizer and
    UBSan: every access stays inside them (what the kernel relies on)."""
    import pickle
    import sys
    pa = pytest.importorskip("pyarrow")
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    asan = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    ubsan = subprocess.run(["g++", "-print-file-name=libubsan.so"], capture_output=True, text=True).stdout.strip()
    if not (os.path.isabs(asan) and os.path.exists(asan) and os.path.isabs(ubsan) and os.path.exists(ubsan)):
        pytest.skip("no sanitizer runtime")
    so = str(tmp_path / "zstd_core_asan.so")
    subprocess.run(["g++", "-O1", "-g", "-std=c++17", "-shared", "-fPIC", "-fsanitize=address,undefined",
                    "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "paper_2602_17335_gb300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "zstd_host_harness.cpp"), "-o", so],
                   check=True)
    from test_oracle_pins import _zstd_inputs
    rng = np.random.default_rng(9)
    cases = []
    for i, x in enumerate(_zstd_inputs(np.random.default_rng(1))[:40]):
        frame = pa.Codec("zstd", compression_level=[1, 3, 19][i % 3]).compress(x, asbytes=True)
        for t in range(25):
            f = bytearray(frame)
            for _ in range(int(rng.integers(1, 4))):
                f[int(rng.integers(0, len(f)))] = int(rng.integers(0, 256))
            if t % 7 == 0:
                f = f[:int(rng.integers(0, len(f)))]
            cases.append((bytes(f), len(x) if t % 2 else int(rng.integers(0, len(x) + 10))))
    pk = str(tmp_path / "cases.pkl")
    pickle.dump(cases, open(pk, "wb"))
    env = dict(os.environ, LD_PRELOAD=asan + ":" + ubsan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", _FUZZ, so, pk], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "Sanitizer" not in r.stderr and "runtime error" not in r.stderr, r.stderr[-3000:]
    n, rejected = map(int, r.stdout.split())
    assert n == len(cases) and rejected > n // 2
