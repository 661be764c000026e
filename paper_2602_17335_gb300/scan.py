"""Torch-side convenience around the C ABI: device buffers for files and
outputs, and one call that indexes, plans and scans.  PyTorch only supplies
device memory and streams; every step of the scan runs in the engine's
CUDA kernels through ``native``."""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import torch

from . import native as N

_DTYPE = {N.PQ_TYPE_INT32: torch.int32, N.PQ_TYPE_INT64: torch.int64, N.PQ_TYPE_DOUBLE: torch.float64,
          N.PQ_TYPE_FLOAT: torch.float32}


@dataclass
class ColumnOut:
    size: N.pq_out_size
    values: torch.Tensor                 # values, or int64 offsets for BYTE_ARRAY
    validity: Optional[torch.Tensor]     # int32 words (bitmap), OPTIONAL only
    chars: Optional[torch.Tensor]        # uint8, BYTE_ARRAY only

    def desc(self) -> N.pq_column:
        c = N.pq_column()
        c.values = self.values.data_ptr() if self.values.numel() else None
        c.validity = self.validity.data_ptr() if self.validity is not None and self.validity.numel() else None
        c.chars = self.chars.data_ptr() if self.chars is not None and self.chars.numel() else None
        c.chars_capacity = 0 if self.chars is None else self.chars.numel()
        return c


def alloc_outputs(sizes: List[N.pq_out_size], device="cuda") -> List[ColumnOut]:
    outs = []
    for s in sizes:
        if s.type == N.PQ_TYPE_BYTE_ARRAY:
            vals = torch.empty(s.n_rows + 1, dtype=torch.int64, device=device)
            chars = torch.empty(max(int(s.chars_bytes), 1), dtype=torch.uint8, device=device)
        else:
            vals = torch.empty(s.n_rows, dtype=_DTYPE[s.type], device=device)
            chars = None
        valid = torch.empty(max(int(s.validity_bytes) // 4, 1), dtype=torch.int32, device=device) if s.optional else None
        outs.append(ColumnOut(s, vals, valid, chars))
    return outs


def stream_handle(stream: Optional[torch.cuda.Stream] = None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


class Engine:
    """One engine context on one device."""

    def __init__(self, device: int = 0):
        self.device = device
        self.ctx = N.pq_ctx_create(device)

    def close(self):
        if self.ctx:
            N.pq_ctx_destroy(self.ctx)
            self.ctx = None

    def index(self, files: List[torch.Tensor], stream=None):
        return N.pq_index_chunks(self.ctx, [(t.data_ptr(), t.numel()) for t in files], stream_handle(stream))

    def plan(self, idx, columns=None, row_begin=0, row_count=-1, flags=N.PQ_SCAN_BATCHED):
        return N.pq_plan_scan(self.ctx, idx, columns, row_begin, row_count, flags)

    def scan(self, plan, outs: List[ColumnOut], stream=None):
        N.pq_scan_columns(self.ctx, plan, [o.desc() for o in outs], stream_handle(stream))

    def wait(self, plan, ncols, stream=None):
        return N.pq_scan_wait(self.ctx, plan, ncols, stream_handle(stream))

    def read(self, files: List[torch.Tensor], columns=None, row_begin=0, row_count=-1,
             flags=N.PQ_SCAN_BATCHED):
        """Index + plan + scan + wait; returns the ColumnOut list (raises on error)."""
        idx = self.index(files)
        try:
            plan, sizes = self.plan(idx, columns, row_begin, row_count, flags)
            try:
                outs = alloc_outputs(sizes)
                self.scan(plan, outs)
                st, chars = self.wait(plan, len(outs))
                if st != N.PQ_OK:
                    raise N.PqError(st, N.pq_last_error(self.ctx))
                for o, c in zip(outs, chars):
                    if o.chars is not None:
                        o.chars = o.chars[:c]
                return outs
            finally:
                N.pq_free_plan(plan)
        finally:
            N.pq_free_index(idx)
