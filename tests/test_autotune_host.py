"""The autotuner's search (coordinate descent over the scan's knobs) on a
synthetic cost surface, with the context call recorded instead of made: no
GPU needed."""
from paper_2602_17335_gb300 import autotune as A


def _run(cost, monkeypatch, rounds=1):
    applied = []
    monkeypatch.setattr(A.N, "pq_ctx_set_tuning", lambda ctx, **t: applied.append(dict(t)))
    seen = []

    def time_ms(t):
        assert applied[-1] == t           # the tuner applies a tuning before timing it
        seen.append(dict(t))
        return cost(t)
    best, best_ms, trials = A.autotune(object(), time_ms, rounds=rounds)
    return best, best_ms, trials, applied, seen


def test_finds_the_separable_optimum(monkeypatch):
    target = {"item_rows": 4096, "item_rows_opt": 256, "expand_ctas_per_sm": 2, "branches": 4,
              "walk_window": 32768, "snappy_block_kib": 64, "staged_expand": 0}

    def cost(t):
        return 1.0 + sum(abs(t[k] - target[k]) / (1 + target[k]) for k in target)
    best, best_ms, trials, applied, seen = _run(cost, monkeypatch)
    assert best == target
    assert best_ms == cost(target) == min(ms for _, ms in trials)
    assert applied[-1] == target          # the chosen tuning stays set
    assert len(trials) == 1 + sum(len(v) - 1 for v in A.CANDIDATES.values())


def test_keeps_the_default_when_nothing_is_faster(monkeypatch):
    def cost(t):
        return 1.0 if t == A.DEFAULT else 2.0
    best, best_ms, _, applied, _ = _run(cost, monkeypatch)
    assert best == A.DEFAULT and best_ms == 1.0 and applied[-1] == A.DEFAULT


def test_second_round_reaches_a_coupled_optimum(monkeypatch):
    # item_rows pays off only once branches is 4: one pass over the knobs in
    # order misses it, a second pass finds it
    def cost(t):
        c = 10.0
        if t["branches"] == 4:
            c -= 1.0
            if t["item_rows"] == 8192:
                c -= 5.0
        return c
    best1, ms1, _, _, _ = _run(cost, monkeypatch, rounds=1)
    best2, ms2, _, _, _ = _run(cost, monkeypatch, rounds=2)
    assert best1["branches"] == 4 and best1["item_rows"] == 2048 and ms1 == 9.0
    assert best2["branches"] == 4 and best2["item_rows"] == 8192 and ms2 == 4.0
