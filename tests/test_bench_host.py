"""Host-side pieces of bench.py that need no GPU: the traffic-capture key,
the pyarrow context point and the one-rank reductions."""
import builtins

import pytest

import bench
import synth


class _Args:
    rows, rg_rows, page_bytes, codec, page_version, mode, no_offset_index = 1 << 26, 1 << 23, 1 << 20, \
        "UNCOMPRESSED", 1, "batched", False

    def __init__(self, table):
        self.table = table


def test_traffic_key_separates_tables():
    assert bench.traffic_key(_Args("eight")) != bench.traffic_key(_Args("v2"))
    assert bench.stored_traffic(_Args("v2"))[0] is None


def test_single_rank_reductions_are_identities():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.sum_over_ranks(7.0, 1) == 7.0
    assert bench.whole_job_gbs(2e9, 0.5) == pytest.approx(4.0)


def test_pyarrow_context_point(monkeypatch):
    from oracle import writer as W
    data = W.write_file(synth.config2_table(4000, 4000, string_pool_size=50, zipf_k=100),
                        synth.config2_spec(4000, 8192))
    pytest.importorskip("pyarrow")
    got = bench.pyarrow_context(data, 1e6)
    assert got["value"] > 0 and got["unit"] == "GB/s" and "not the oracle" in got["kind"]
    real_import = builtins.__import__

    def no_pyarrow(name, *a, **k):
        if name.startswith("pyarrow"):
            raise ImportError(name)
        return real_import(name, *a, **k)
    monkeypatch.setattr(builtins, "__import__", no_pyarrow)
    assert "unavailable" in bench.pyarrow_context(data, 1e6)
