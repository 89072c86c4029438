"""The replica split used by bench.py --gpus N (independent systems, no data-
path collective) and its host-side bookkeeping, as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch

    import synth
    from paper_2411_04686_gb300 import serve
    specs = synth.shard_specs(synth.batch_specs(37, seed=0), rank, world)
    reqs = serve.shard(list(range(101)), rank, world)
    rows = torch.tensor([float(sum(s.n for s in specs)), float(len(specs)), float(len(reqs))])
    dist.all_reduce(rows, op=dist.ReduceOp.SUM)
    t = torch.tensor([1.0 + rank])                  # per-rank time; the job time is the max
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, rows.tolist(), t.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_without_overlap():
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    total_rows = float(sum(s.n for s in synth.batch_specs(37, seed=0)))
    for rank, (rows, nsys, nreq), tmax in res:
        assert rows == total_rows and nsys == 37 and nreq == 101
        assert tmax == 2.0
