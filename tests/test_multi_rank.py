"""The multi-GPU path's host logic, run as two gloo ranks on the CPU.

On N GPUs every rank scans its own seeded table of the same shape (weak
scaling) and the data path has no collective; the step time is the slowest
rank's and the job's bytes are the sum over ranks.  These tests run exactly
that logic (bench.py's max_over_ranks, sum_over_ranks, whole_job_gbs and
the per-rank table) with world size 2 over gloo."""
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_and_shard():
    mp = pytest.importorskip("torch.multiprocessing")
    import multi_rank_worker
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=multi_rank_worker.run, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    (r0, slow0, total0, gbs0, rows0), (r1, slow1, total1, gbs1, rows1) = out
    assert (r0, r1) == (0, 1)
    # the slowest rank's time, on every rank
    assert slow0 == slow1 == 15.0
    # the bytes of both ranks, on every rank; the job rate from them
    assert total0 == total1 == rows0[0][1] + rows0[1][1]
    assert gbs0 == gbs1 == pytest.approx(total0 / 15e-3 / 1e9)
    # each rank scans its own data (seeded by rank), with the same schema
    assert rows0 == rows1
    assert rows0[0][0] != rows0[1][0]
    assert rows0[0][2] == rows0[1][2]
    # weak scaling: per-rank work of the same size (strings differ in length only)
    assert abs(rows0[0][1] - rows0[1][1]) < 0.05 * rows0[0][1]
