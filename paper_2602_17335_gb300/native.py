"""ctypes binding of the C ABI in ``include/pq.h`` — argument marshalling only.

Every function keeps its C name; structs mirror the header field by field.
Loading fails loudly (``RuntimeError``) when the built library is missing:
there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpqscan.so")

PQ_OK, PQ_ERR_INVALID_ARG, PQ_ERR_CORRUPT, PQ_ERR_UNSUPPORTED = 0, 1, 2, 3
PQ_ERR_OOM, PQ_ERR_BUDGET, PQ_ERR_TIMEOUT, PQ_ERR_CUDA, PQ_ERR_CAPACITY = 4, 5, 6, 7, 8
PQ_TYPE_INT32, PQ_TYPE_INT64, PQ_TYPE_FLOAT, PQ_TYPE_DOUBLE, PQ_TYPE_BYTE_ARRAY = 1, 2, 4, 5, 6
PQ_SCAN_BATCHED, PQ_SCAN_PLAIN, PQ_SCAN_GRAPH, PQ_SCAN_RESIDENT_DICT, PQ_SCAN_TIMING = 0, 1, 2, 4, 8
STAGES = ("prepare", "snappy", "dict", "walk", "expand", "strings")

STATUS_NAMES = {0: "PQ_OK", 1: "PQ_ERR_INVALID_ARG", 2: "PQ_ERR_CORRUPT", 3: "PQ_ERR_UNSUPPORTED",
                4: "PQ_ERR_OOM", 5: "PQ_ERR_BUDGET", 6: "PQ_ERR_TIMEOUT", 7: "PQ_ERR_CUDA",
                8: "PQ_ERR_CAPACITY"}


class pq_file(C.Structure):
    _fields_ = [("data", C.c_void_p), ("size", C.c_uint64)]


class pq_index_info(C.Structure):
    _fields_ = [("n_files", C.c_int32), ("n_columns", C.c_int32), ("n_row_groups", C.c_int32),
                ("n_chunks", C.c_int32), ("n_pages", C.c_int64), ("n_data_pages", C.c_int64),
                ("num_rows", C.c_int64), ("stored_bytes", C.c_uint64), ("uncompressed_bytes", C.c_uint64),
                ("used_offset_index", C.c_int32), ("reserved", C.c_int32)]


class pq_column_info(C.Structure):
    _fields_ = [("name", C.c_char * 64), ("type", C.c_int32), ("optional", C.c_int32),
                ("type_length", C.c_int32), ("reserved", C.c_int32)]


class pq_page_info(C.Structure):
    _fields_ = [("header_offset", C.c_int64), ("file", C.c_int32), ("chunk", C.c_int32),
                ("page_type", C.c_int32), ("encoding", C.c_int32), ("header_len", C.c_int32),
                ("uncompressed_size", C.c_int32), ("compressed_size", C.c_int32), ("num_values", C.c_int32),
                ("num_nulls", C.c_int32), ("def_len", C.c_int32), ("first_row", C.c_int64)]


class pq_request(C.Structure):
    _fields_ = [("columns", C.POINTER(C.c_int32)), ("n_columns", C.c_int32), ("flags", C.c_uint32),
                ("row_begin", C.c_int64), ("row_count", C.c_int64)]


class pq_out_size(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("type", C.c_int32), ("optional", C.c_int32),
                ("values_bytes", C.c_uint64), ("validity_bytes", C.c_uint64), ("chars_bytes", C.c_uint64)]


class pq_plan_info(C.Structure):
    _fields_ = [("n_columns", C.c_int32), ("n_pages", C.c_int32), ("n_dict_pages", C.c_int32),
                ("n_items", C.c_int32), ("read_bytes", C.c_uint64), ("decoded_bytes", C.c_uint64),
                ("scratch_bytes", C.c_uint64), ("launches_per_scan", C.c_int32), ("reserved", C.c_int32)]


class pq_column(C.Structure):
    _fields_ = [("values", C.c_void_p), ("validity", C.c_void_p), ("chars", C.c_void_p),
                ("chars_capacity", C.c_uint64)]


class pq_serve_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("slots", C.c_int32), ("timeout_ms", C.c_int32)]


class pq_serve_request(C.Structure):
    _fields_ = [("columns", C.POINTER(C.c_int32)), ("n_columns", C.c_int32), ("reserved", C.c_int32),
                ("row_begin", C.c_int64), ("row_count", C.c_int64)]


class pq_serve_result(C.Structure):
    _fields_ = [("status", C.c_int), ("n_columns", C.c_int32), ("columns", C.POINTER(pq_column)),
                ("sizes", C.POINTER(pq_out_size)), ("queue_ms", C.c_double), ("latency_ms", C.c_double),
                ("decoded_bytes", C.c_uint64), ("admit_ms", C.c_double), ("done_ms", C.c_double)]


class pq_write_column(C.Structure):
    _fields_ = [("name", C.c_char_p), ("type", C.c_int32), ("encoding", C.c_int32), ("codec", C.c_int32),
                ("page_version", C.c_int32), ("compress_threshold", C.c_double), ("values", C.c_void_p),
                ("chars", C.c_void_p), ("valid", C.c_void_p)]


class pq_tuning(C.Structure):
    _fields_ = [("item_rows", C.c_int32), ("item_rows_opt", C.c_int32), ("expand_ctas_per_sm", C.c_int32),
                ("branches", C.c_int32), ("walk_window", C.c_int32), ("snappy_block_kib", C.c_int32),
                ("staged_expand", C.c_int32), ("reserved", C.c_int32)]


_P = C.c_void_p
_SIGS = {
    "pq_version": (C.c_char_p, []),
    "pq_status_string": (C.c_char_p, [C.c_int]),
    "pq_ctx_create": (C.c_int, [C.c_int, C.POINTER(_P)]),
    "pq_ctx_destroy": (None, [_P]),
    "pq_last_error": (C.c_char_p, [_P]),
    "pq_index_chunks": (C.c_int, [_P, C.POINTER(pq_file), C.c_int, _P, C.POINTER(_P)]),
    "pq_index_get_info": (C.c_int, [_P, C.POINTER(pq_index_info)]),
    "pq_index_get_column": (C.c_int, [_P, C.c_int, C.POINTER(pq_column_info)]),
    "pq_index_copy_pages": (C.c_int, [_P, C.POINTER(pq_page_info), C.c_int64, C.POINTER(C.c_int64)]),
    "pq_free_index": (None, [_P]),
    "pq_plan_scan": (C.c_int, [_P, _P, C.POINTER(pq_request), C.POINTER(_P), C.POINTER(pq_out_size)]),
    "pq_plan_get_info": (C.c_int, [_P, C.POINTER(pq_plan_info)]),
    "pq_plan_stage_ms": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "pq_free_plan": (None, [_P]),
    "pq_scan_columns": (C.c_int, [_P, _P, C.POINTER(pq_column), _P]),
    "pq_scan_wait": (C.c_int, [_P, _P, _P, C.POINTER(C.c_uint64)]),
    "pq_scan_host": (C.c_int, [_P, C.POINTER(pq_file), C.c_int, C.POINTER(pq_request), C.POINTER(pq_column),
                               C.POINTER(pq_out_size)]),
    "pq_serve_create": (C.c_int, [_P, _P, C.POINTER(pq_serve_config), C.POINTER(_P)]),
    "pq_serve_submit": (C.c_int, [_P, C.POINTER(pq_serve_request), C.POINTER(C.c_uint64)]),
    "pq_serve_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(pq_serve_result), C.POINTER(C.c_int)]),
    "pq_serve_release": (C.c_int, [_P, C.c_uint64]),
    "pq_serve_destroy": (None, [_P]),
    "pq_write_table": (C.c_int, [C.POINTER(pq_write_column), C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_int,
                                 C.c_int, C.POINTER(C.POINTER(C.c_uint8)), C.POINTER(C.c_uint64)]),
    "pq_write_free": (None, [C.POINTER(C.c_uint8)]),
    "pq_delta_decode_static": (C.c_int, [_P, _P, C.c_uint64, C.c_int, C.c_int64, _P, _P]),
    "pq_ctx_set_tuning": (C.c_int, [_P, C.POINTER(pq_tuning)]),
    "pq_ctx_get_tuning": (C.c_int, [_P, C.POINTER(pq_tuning)]),
    "pq_batch_create": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(C.POINTER(pq_column)), C.c_uint32,
                                  C.POINTER(_P)]),
    "pq_batch_launch": (C.c_int, [_P, _P]),
    "pq_batch_wait": (C.c_int, [_P]),
    "pq_batch_free": (None, [_P]),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded engine library (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"engine library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            try:
                fn = getattr(L, name)
            except AttributeError:
                continue  # reported by missing_symbols()
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def missing_symbols():
    """Names declared in include/pq.h that the loaded library does not export."""
    L = lib()
    return [n for n in _SIGS if not hasattr(L, n)]


class PqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, ctx=None):
    if status != PQ_OK:
        msg = lib().pq_last_error(ctx).decode() if ctx else ""
        raise PqError(status, msg)
    return status


# Thin wrappers with the C names (marshalling only).
def pq_version():
    return lib().pq_version().decode()


def pq_ctx_create(device=0):
    h = C.c_void_p()
    check(lib().pq_ctx_create(device, C.byref(h)))
    return h


def pq_ctx_destroy(ctx):
    lib().pq_ctx_destroy(ctx)


def pq_last_error(ctx):
    return lib().pq_last_error(ctx).decode()


def pq_index_chunks(ctx, files, stream=None):
    """files: list of (device pointer, size)."""
    arr = (pq_file * len(files))(*[pq_file(p, n) for p, n in files])
    h = C.c_void_p()
    check(lib().pq_index_chunks(ctx, arr, len(files), stream, C.byref(h)), ctx)
    return h


def pq_index_get_info(idx):
    info = pq_index_info()
    check(lib().pq_index_get_info(idx, C.byref(info)))
    return info


def pq_index_get_column(idx, column):
    info = pq_column_info()
    check(lib().pq_index_get_column(idx, column, C.byref(info)))
    return info


def pq_index_copy_pages(idx):
    n = C.c_int64()
    check(lib().pq_index_copy_pages(idx, None, 0, C.byref(n)))
    arr = (pq_page_info * max(n.value, 1))()
    check(lib().pq_index_copy_pages(idx, arr, n.value, C.byref(n)))
    return arr[:n.value]


def pq_free_index(idx):
    lib().pq_free_index(idx)


def pq_plan_scan(ctx, idx, columns=None, row_begin=0, row_count=-1, flags=PQ_SCAN_BATCHED):
    """Returns (plan handle, list of pq_out_size)."""
    req = pq_request()
    ncols = pq_index_get_info(idx).n_columns if columns is None else len(columns)
    keep = None
    if columns is not None:
        keep = (C.c_int32 * max(len(columns), 1))(*columns)
        req.columns = C.cast(keep, C.POINTER(C.c_int32))
        req.n_columns = len(columns)
    req.flags = flags
    req.row_begin = row_begin
    req.row_count = row_count
    sizes = (pq_out_size * max(ncols, 1))()
    h = C.c_void_p()
    check(lib().pq_plan_scan(ctx, idx, C.byref(req), C.byref(h), sizes), ctx)
    return h, list(sizes[:ncols])


def pq_plan_get_info(plan):
    info = pq_plan_info()
    check(lib().pq_plan_get_info(plan, C.byref(info)))
    return info


def pq_plan_stage_ms(plan):
    ms = (C.c_float * len(STAGES))()
    check(lib().pq_plan_stage_ms(plan, ms))
    return dict(zip(STAGES, ms[:]))


def pq_scan_host(ctx, host_files, columns=None, row_begin=0, row_count=-1, flags=PQ_SCAN_BATCHED, outs=None):
    """host_files: list of (host pointer, size).  With outs=None returns the
    output sizes; otherwise fills the host buffers described by `outs`
    (list of pq_column with host pointers)."""
    arr = (pq_file * len(host_files))(*[pq_file(p, n) for p, n in host_files])
    req = pq_request()
    keep = None
    if columns is not None:
        keep = (C.c_int32 * max(len(columns), 1))(*columns)
        req.columns = C.cast(keep, C.POINTER(C.c_int32))
        req.n_columns = len(columns)
    req.flags = flags
    req.row_begin = row_begin
    req.row_count = row_count
    sizes = (pq_out_size * 64)()
    o = None if outs is None else (pq_column * max(len(outs), 1))(*outs)
    check(lib().pq_scan_host(ctx, arr, len(host_files), C.byref(req), o, sizes), ctx)
    return sizes


def pq_free_plan(plan):
    lib().pq_free_plan(plan)


def pq_scan_columns(ctx, plan, outs, stream=None):
    """outs: list of pq_column (device pointers)."""
    arr = (pq_column * max(len(outs), 1))(*outs)
    return check(lib().pq_scan_columns(ctx, plan, arr, stream), ctx)


def pq_scan_wait(ctx, plan, ncols, stream=None):
    """Returns (status, chars bytes per column); does not raise."""
    chars = (C.c_uint64 * max(ncols, 1))()
    st = lib().pq_scan_wait(ctx, plan, stream, chars)
    return st, list(chars[:ncols])


def pq_write_table(columns, n_rows, rg_rows, page_bytes, offset_index=True, n_threads=0):
    """columns: list of pq_write_column (pointers kept alive by the caller).
    Returns the file as a numpy uint8 array."""
    import numpy as np
    arr = (pq_write_column * len(columns))(*columns)
    out = C.POINTER(C.c_uint8)()
    size = C.c_uint64()
    check(lib().pq_write_table(arr, len(columns), n_rows, rg_rows, page_bytes, 1 if offset_index else 0,
                               n_threads, C.byref(out), C.byref(size)))
    try:
        return np.ctypeslib.as_array(out, shape=(size.value,)).copy() if size.value else np.zeros(0, np.uint8)
    finally:
        lib().pq_write_free(out)


def pq_delta_decode_static(ctx, d_stream, stream_len, ptype, n_values, d_values, stream=None):
    """Allocation-free decode of one DELTA_BINARY_PACKED stream (device
    pointers); returns the status without raising."""
    return lib().pq_delta_decode_static(ctx, d_stream, stream_len, ptype, n_values, d_values, stream)


def pq_serve_create(ctx, idx, budget_bytes, slots=4, timeout_ms=0):
    cfg = pq_serve_config(budget_bytes, slots, timeout_ms)
    srv = C.c_void_p()
    check(lib().pq_serve_create(ctx, idx, C.byref(cfg), C.byref(srv)), ctx)
    return srv.value


def pq_serve_submit(srv, columns, row_begin, row_count):
    """Returns (status, ticket); does not raise (PQ_ERR_BUDGET is an answer)."""
    arr = (C.c_int32 * len(columns))(*columns)
    req = pq_serve_request(arr, len(columns), 0, row_begin, row_count)
    t = C.c_uint64()
    st = lib().pq_serve_submit(srv, C.byref(req), C.byref(t))
    return st, t.value


def pq_serve_poll(srv, ticket):
    """Returns None while running, else the filled pq_serve_result."""
    res = pq_serve_result()
    done = C.c_int()
    st = lib().pq_serve_poll(srv, ticket, C.byref(res), C.byref(done))
    if st != PQ_OK:
        raise PqError(st, "pq_serve_poll")
    return res if done.value else None


def pq_serve_release(srv, ticket):
    return lib().pq_serve_release(srv, ticket)


def pq_serve_destroy(srv):
    lib().pq_serve_destroy(srv)


def pq_ctx_set_tuning(ctx, item_rows=2048, item_rows_opt=512, expand_ctas_per_sm=0, branches=8, walk_window=0,
                      snappy_block_kib=256, staged_expand=1):
    t = pq_tuning(item_rows, item_rows_opt, expand_ctas_per_sm, branches, walk_window, snappy_block_kib,
                  staged_expand, 0)
    check(lib().pq_ctx_set_tuning(ctx, C.byref(t)), ctx)


def pq_ctx_get_tuning(ctx):
    t = pq_tuning()
    check(lib().pq_ctx_get_tuning(ctx, C.byref(t)), ctx)
    return {"item_rows": t.item_rows, "item_rows_opt": t.item_rows_opt,
            "expand_ctas_per_sm": t.expand_ctas_per_sm, "branches": t.branches, "walk_window": t.walk_window,
            "snappy_block_kib": t.snappy_block_kib, "staged_expand": t.staged_expand}


def pq_batch_create(ctx, plans, outs_per_plan, flags=0):
    """plans: plan handles; outs_per_plan: list of lists of pq_column."""
    n = len(plans)
    parr = (C.c_void_p * n)(*plans)
    keep = [(pq_column * max(len(o), 1))(*o) for o in outs_per_plan]
    oarr = (C.POINTER(pq_column) * n)(*[C.cast(k, C.POINTER(pq_column)) for k in keep])
    b = C.c_void_p()
    check(lib().pq_batch_create(ctx, n, parr, oarr, flags, C.byref(b)), ctx)
    return b.value


def pq_batch_launch(ctx, batch, stream=None):
    check(lib().pq_batch_launch(batch, stream), ctx)


def pq_batch_wait(batch):
    return lib().pq_batch_wait(batch)


def pq_batch_free(batch):
    lib().pq_batch_free(batch)
