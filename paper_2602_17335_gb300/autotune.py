"""Autotuner for the batched scan's knobs (``pq_tuning`` in include/pq.h).

The knobs set scheduling granularity, block sizes and staging depth:
- rows per work item (pages without definition levels, and pages with
  them): how much of a page one warp takes;
- resident CTAs per SM of the expansion kernels;
- how many streams one scan's columns are forked onto;
- the staging depth of the page walks (bytes per shared-memory chain
  window);
- the compressed page size from which a block of 8 warps, rather than one
  warp, decompresses a Snappy page;
- whether dictionary columns take the staged (shared-memory) expansion.

The paper's Section 3 (Insight 1) ties a GPU reader's parallelism to its
page count. Here parallelism comes from work items, so the best item size
depends on the mix of pages, encodings and sizes. It is found by timing.

The tuner does coordinate descent: each knob in turn over its candidate
values, keeping the fastest setting; a setting is timed once. It times with
a caller-supplied function that rebuilds the plans under the tuning it is
given and returns milliseconds per run. The chosen tuning is left set on the
context.
"""
from __future__ import annotations

from typing import Callable, Dict, List, Tuple

from . import native as N

DEFAULT: Dict[str, int] = {"item_rows": 2048, "item_rows_opt": 512, "expand_ctas_per_sm": 0, "branches": 8,
                           "walk_window": 0, "snappy_block_kib": 256, "staged_expand": 1}

CANDIDATES: Dict[str, List[int]] = {
    "item_rows": [1024, 2048, 4096, 8192],
    "item_rows_opt": [256, 512],
    "expand_ctas_per_sm": [0, 2],
    "branches": [4, 8],
    "walk_window": [0, 8192, 32768],
    "snappy_block_kib": [64, 256, 1024],
    "staged_expand": [0, 1],
}


def autotune(ctx, time_ms: Callable[[Dict[str, int]], float], rounds: int = 1,
             candidates: Dict[str, List[int]] = None) -> Tuple[Dict[str, int], float, List[Tuple[Dict[str, int], float]]]:
    """Returns (best tuning, its ms, every trial).  `time_ms(tuning)` must
    apply nothing itself: the tuner sets the tuning on `ctx` before each call."""
    cands = candidates or CANDIDATES
    trials: List[Tuple[Dict[str, int], float]] = []
    timed: Dict[Tuple, float] = {}

    def run(t: Dict[str, int]) -> float:
        key = tuple(sorted(t.items()))
        if key in timed:  # a setting is timed once, even when the descent comes back to it
            return timed[key]
        N.pq_ctx_set_tuning(ctx, **t)
        ms = time_ms(t)
        trials.append((dict(t), ms))
        timed[key] = ms
        return ms

    best = dict(DEFAULT)
    best_ms = run(best)
    for _ in range(rounds):
        for knob, values in cands.items():
            for v in values:
                if v == best[knob]:
                    continue
                t = dict(best, **{knob: v})
                ms = run(t)
                if ms < best_ms:
                    best, best_ms = t, ms
    N.pq_ctx_set_tuning(ctx, **best)
    return best, best_ms, trials
