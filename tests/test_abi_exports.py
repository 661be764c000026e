"""The C ABI library loads (no GPU needed) and exports every function that
include/pq.h declares; the binding knows every one of them."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(pq_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_scan_path():
    names = _declared()
    for n in ("pq_index_chunks", "pq_plan_scan", "pq_scan_columns", "pq_serve_submit", "pq_serve_poll",
              "pq_delta_decode_static"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_17335_gb300 import native as N
    lib = N.lib()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared in include/pq.h but not exported: {missing}"
    unbound = [n for n in _declared() if n not in N.exported_symbols()]
    assert not unbound, f"no binding signature for: {unbound}"
