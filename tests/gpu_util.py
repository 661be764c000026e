"""Helpers shared by the GPU tests: build-once engine, device upload and
element-by-element comparison against the CPU oracle's reading."""
import numpy as np


def engine():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_17335_gb300.scan import Engine
    return Engine(0)


def to_dev(data):
    import torch
    return torch.frombuffer(bytearray(data), dtype=torch.uint8).to("cuda")


def bitmap_words(valid):
    bits = np.packbits(np.asarray(valid, dtype=bool), bitorder="little")
    out = np.zeros(((len(valid) + 31) // 32) * 4, dtype=np.uint8)
    out[:len(bits)] = bits
    return out


def slice_result(r, lo, hi):
    """Rows [lo, hi) of an oracle ColumnResult."""
    from oracle.reader import ColumnResult
    valid = None if r.valid is None else r.valid[lo:hi]
    if r.ptype == "BYTE_ARRAY":
        off = r.offsets[lo:hi + 1] - r.offsets[lo]
        chars = r.chars[r.offsets[lo]:r.offsets[hi]]
        return ColumnResult(r.name, r.ptype, None, valid, off, chars)
    return ColumnResult(r.name, r.ptype, r.values[lo:hi], valid)


def assert_columns_equal(outs, expect, chars_sizes=None):
    """Bit-exact: values (null slots zero), validity bitmap, offsets, chars."""
    for i, (o, e) in enumerate(zip(outs, expect)):
        if e.ptype == "BYTE_ARRAY":
            got_off = o.values.cpu().numpy()
            assert np.array_equal(got_off, e.offsets), f"{e.name}: offsets differ"
            n = int(got_off[-1]) if len(got_off) else 0
            got_chars = o.chars.cpu().numpy()[:n]
            assert np.array_equal(got_chars, e.chars), f"{e.name}: chars differ"
        else:
            got = o.values.cpu().numpy()
            exp = e.values
            assert got.dtype.itemsize == exp.dtype.itemsize
            if not np.array_equal(got.view(np.uint8), exp.view(np.uint8)):
                bad = np.nonzero(got.view(exp.dtype) != exp)[0] if exp.dtype.kind != "f" else \
                    np.nonzero(got.view(np.int64) != exp.view(np.int64))[0]
                raise AssertionError(f"{e.name}: {len(bad)} values differ, first rows {bad[:10]}: "
                                     f"got {got[bad[:5]]} expected {exp[bad[:5]]}")
        if e.valid is None:
            assert o.validity is None
        else:
            words = bitmap_words(e.valid)
            got = o.validity.cpu().numpy().view(np.uint8)[:len(words)]
            assert np.array_equal(got, words), f"{e.name}: validity differs"


def _cudart():
    import ctypes
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            lib = ctypes.CDLL(name)
            lib.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
            lib.cudaMemcpy.restype = ctypes.c_int
            return lib
        except OSError:
            continue
    raise RuntimeError("CUDA runtime library not found")


def server_result_outs(res):
    """Copies a serving result's server-owned device columns into torch
    tensors (ColumnOut objects), so they compare like scan outputs."""
    import torch
    from paper_2602_17335_gb300 import native as N
    from paper_2602_17335_gb300.scan import alloc_outputs
    rt = _cudart()
    sizes = [res.sizes[i] for i in range(res.n_columns)]
    outs = alloc_outputs(sizes)
    for i, o in enumerate(outs):
        c = res.columns[i]
        s = sizes[i]
        vb = (s.n_rows + 1) * 8 if s.type == N.PQ_TYPE_BYTE_ARRAY else s.values_bytes
        assert rt.cudaMemcpy(o.values.data_ptr(), c.values, vb, 4) == 0
        if o.validity is not None and s.validity_bytes:
            assert rt.cudaMemcpy(o.validity.data_ptr(), c.validity, s.validity_bytes, 4) == 0
        if o.chars is not None and s.chars_bytes:
            assert rt.cudaMemcpy(o.chars.data_ptr(), c.chars, s.chars_bytes, 4) == 0
    torch.cuda.synchronize()
    return outs
