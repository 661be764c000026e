"""The row-group pipeline's host page walk (csrc/host_pages.cpp: the index's
header walk over a chunk in host memory) compiled for the CPU with g++,
against the CPU oracle's chunk walk: every page of V1/V2, dictionary,
Snappy, Zstandard and V2-encoding files, with its offset within the chunk,
first row, type, encoding, counts and sizes; truncated chunks are rejected
without reading outside their bytes (AddressSanitizer).  No GPU needed."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle import reader as R
from oracle import writer as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(ROOT, "paper_2602_17335_gb300", "csrc")
INC = ["-I", CSRC, "-I", os.path.join(ROOT, "include")]


def _compile(out, extra=()):
    subprocess.run(["g++", "-std=c++17", "-shared", "-fPIC", *extra, *INC, os.path.join(HERE, "host_pages_harness.cpp"),
                    os.path.join(CSRC, "host_pages.cpp"), "-o", out], check=True)


def _bind(path):
    lib = ctypes.CDLL(path)
    lib.host_walk.restype = ctypes.c_int64
    lib.host_walk.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]

    def walk(b, num_values):
        out = np.zeros((4096, 10), dtype=np.int64)
        n = lib.host_walk(bytes(b), len(b), num_values, out.ctypes.data, 4096)
        return n, out[:max(n, 0)]
    return walk


@pytest.fixture(scope="module")
def walk(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("host_pages") / "host_pages.so")
    _compile(out, ["-O2"])
    return _bind(out)


def _files():
    tab = synth.config2_table(6000, 2500, string_pool_size=200, zipf_k=300)
    v2 = synth.v2_encodings_table(4000, 2000)
    out = [W.write_file(tab, synth.config2_spec(2500, 2048, codec, version))
           for codec, version in (("UNCOMPRESSED", 1), ("SNAPPY", 2), ("ZSTD", 1))]
    out.append(W.write_file(v2, synth.v2_encodings_spec(2000, 1500)))
    out.append(open(os.path.join(HERE, "golden", "zstd_eight_column_v2.parquet"), "rb").read())
    return out


def test_host_walk_matches_the_oracle(walk):
    chunks = 0
    for data in _files():
        for ch in R.parse_footer(data).chunks:
            b = data[ch.start:ch.start + ch.total_compressed]
            n, got = walk(b, ch.num_values)
            exp = R.chunk_pages(data, ch)
            assert n == len(exp)
            row = 0
            for g, p in zip(got, exp):
                first = 0 if p.page_type == 2 else row
                if p.page_type != 2:
                    row += p.num_values
                assert list(g) == [p.offset - ch.start, first, p.page_type, p.encoding, p.num_values,
                                   p.num_nulls if p.page_type == 3 else -1, p.def_len, p.header_len,
                                   p.uncompressed, p.compressed]
            chunks += 1
    assert chunks > 40


def test_truncated_chunks_are_rejected(walk):
    data = _files()[1]
    for ch in R.parse_footer(data).chunks[:6]:
        b = data[ch.start:ch.start + ch.total_compressed]
        for cut in sorted({1, 7, len(b) // 3, len(b) // 2, len(b) - 1}):
            assert walk(b[:cut], ch.num_values)[0] == -1
        assert walk(b, ch.num_values + 1)[0] == -1  # more values than the pages hold


_ASAN_RUN = r'''
import ctypes, pickle, sys
import numpy as np
lib = ctypes.CDLL(sys.argv[1])
lib.host_walk.restype = ctypes.c_int64
lib.host_walk.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]
out = np.zeros((4096, 10), dtype=np.int64)
cases = pickle.load(open(sys.argv[2], "rb"))
bad = 0
for b, nv in cases:
    buf = ctypes.create_string_buffer(b, len(b))  # exactly the chunk's bytes
    bad += lib.host_walk(buf, len(b), nv, out.ctypes.data, 4096) < 0
print(len(cases), bad)
'''


def test_mutated_chunks_stay_in_bounds_under_asan(tmp_path):
    import pickle
    import sys
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    asan = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not (os.path.isabs(asan) and os.path.exists(asan)):
        pytest.skip("no sanitizer runtime")
    so = str(tmp_path / "host_pages_asan.so")
    _compile(so, ["-O1", "-g", "-fsanitize=address", "-fno-omit-frame-pointer"])
    rng = np.random.default_rng(9)
    data = _files()[0]
    cases = []
    for ch in R.parse_footer(data).chunks[:8]:
        b = data[ch.start:ch.start + ch.total_compressed]
        for t in range(25):
            m = bytearray(b)
            for _ in range(int(rng.integers(1, 5))):
                m[int(rng.integers(0, min(len(m), 400)))] = int(rng.integers(0, 256))
            if t % 2 == 0:
                m = m[:int(rng.integers(0, len(m) + 1))]
            cases.append((bytes(m), ch.num_values))
    pk = str(tmp_path / "cases.pkl")
    pickle.dump(cases, open(pk, "wb"))
    script = str(tmp_path / "run.py")
    open(script, "w").write(_ASAN_RUN)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0")
    r = subprocess.run([sys.executable, script, so, pk], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    n, bad = map(int, r.stdout.split())
    assert n == len(cases) and bad > 0
