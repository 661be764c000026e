"""Worker of the two-rank gloo tests (a module of its own, so that spawned
processes can import it by name)."""
import hashlib
import os


def run(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        from oracle import reader as R
        from oracle import writer as W
        # the rank's own table, as the bench stages it (file = rank)
        tab = synth.config2_table(3000, 1500, file=rank, string_pool_size=50, zipf_k=100)
        data = W.write_file(tab, synth.config2_spec(1500, 2048))
        res = R.read_file(data)
        decoded = sum((r.values.nbytes if r.values is not None else r.offsets.nbytes + r.chars.nbytes)
                      + (0 if r.valid is None else (len(r.valid) + 31) // 32 * 4) for r in res)
        step_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        slow = bench.max_over_ranks(step_ms, world)
        total = bench.sum_over_ranks(decoded, world)
        rows = [None] * world
        dist.all_gather_object(rows, (hashlib.sha256(data).hexdigest(), decoded, [r.name for r in res]))
        q.put((rank, slow, total, bench.whole_job_gbs(total, slow * 1e-3), rows))
    finally:
        dist.destroy_process_group()
