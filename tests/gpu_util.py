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
