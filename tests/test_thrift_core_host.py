"""The index kernel's PageHeader parser (csrc/thrift_dev.cuh, run on the GPU
by the page-header index) compiled for the CPU with g++, against the CPU
oracle's Thrift reader: every page header of V1/V2, dictionary, Snappy and
Zstandard files parses to the same fields and length, and mutated headers
never make it read outside their bytes (AddressSanitizer, exact-size
buffers).  No GPU needed."""
import ctypes
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import synth
from oracle import reader as R
from oracle import writer as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
INC = ["-I", os.path.join(ROOT, "paper_2602_17335_gb300", "csrc"), "-I", os.path.join(ROOT, "include")]


def _compile(out, extra=()):
    subprocess.run(["g++", "-std=c++17", "-shared", "-fPIC", *extra, *INC,
                    os.path.join(HERE, "thrift_host_harness.cpp"), "-o", out], check=True)


@pytest.fixture(scope="module")
def parse(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("thrift") / "thrift_core.so")
    _compile(out, ["-O2"])
    lib = ctypes.CDLL(out)
    lib.page_header_host.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_void_p]

    def run(b):
        o = np.zeros(9, dtype=np.int32)
        n = lib.page_header_host(bytes(b), len(b), o.ctypes.data)
        return n, o.tolist()
    return run


def _files():
    tab = synth.config2_table(6000, 2500, string_pool_size=200, zipf_k=300)
    v2 = synth.v2_encodings_table(4000, 2000)
    out = [W.write_file(tab, synth.config2_spec(2500, 2048, codec, version))
           for codec, version in (("UNCOMPRESSED", 1), ("SNAPPY", 2), ("ZSTD", 1))]
    out.append(W.write_file(v2, synth.v2_encodings_spec(2000, 1500)))
    for name in ("zstd_eight_column_v1.parquet", "zstd_eight_column_v2.parquet"):
        out.append(open(os.path.join(HERE, "golden", name), "rb").read())
    return out


def _headers(data):
    for ch in R.parse_footer(data).chunks:
        end = ch.start + ch.total_compressed
        for p in R.chunk_pages(data, ch):
            yield data[p.offset:end], p


def test_every_header_matches_the_oracle(parse):
    n = 0
    for data in _files():
        for b, p in _headers(data):
            hl, f = parse(b)
            assert hl == p.header_len
            assert f[:5] == [p.page_type, p.uncompressed, p.compressed, p.num_values, p.encoding]
            if p.page_type == 3:
                assert f[5:9] == [p.num_nulls, p.def_len, p.rep_len, 1 if p.is_compressed else 0]
            n += 1
    assert n > 500


def test_truncated_headers_are_rejected(parse):
    data = _files()[1]
    for b, p in list(_headers(data))[:50]:
        for cut in range(p.header_len):
            assert parse(b[:cut])[0] == -1


_FUZZ = r'''
import ctypes, pickle, sys
import numpy as np
lib = ctypes.CDLL(sys.argv[1])
lib.page_header_host_exact.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_void_p]
o = np.zeros(9, dtype=np.int32)
cases = pickle.load(open(sys.argv[2], "rb"))
bad = sum(lib.page_header_host_exact(c, len(c), o.ctypes.data) < 0 for c in cases)
print(len(cases), bad)
'''


def test_mutated_headers_stay_in_bounds_under_asan(tmp_path):
    import pickle
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    asan = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    ubsan = subprocess.run(["g++", "-print-file-name=libubsan.so"], capture_output=True, text=True).stdout.strip()
    if not (os.path.isabs(asan) and os.path.exists(asan) and os.path.isabs(ubsan) and os.path.exists(ubsan)):
        pytest.skip("no sanitizer runtime")
    so = str(tmp_path / "thrift_asan.so")
    _compile(so, ["-O1", "-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer"])
    rng = np.random.default_rng(4)
    heads = [b[:p.header_len] for data in _files()[:2] for b, p in _headers(data)][:400]
    cases = []
    for h in heads:
        for t in range(10):
            m = bytearray(h)
            for _ in range(int(rng.integers(1, 4))):
                m[int(rng.integers(0, len(m)))] = int(rng.integers(0, 256))
            if t % 3 == 0:
                m = m[:int(rng.integers(0, len(m) + 1))]
            cases.append(bytes(m))
    pk = str(tmp_path / "cases.pkl")
    pickle.dump(cases, open(pk, "wb"))
    env = dict(os.environ, LD_PRELOAD=asan + ":" + ubsan, ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", _FUZZ, so, pk], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "Sanitizer" not in r.stderr and "runtime error" not in r.stderr, r.stderr[-3000:]
    n, bad = map(int, r.stdout.split())
    assert n == len(cases) and bad > 0
