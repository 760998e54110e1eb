"""Multi-rank path of the benchmark on CPU (gloo, world size 2): the independent instances of
the batched workload are partitioned across ranks with no data-path collective, every
instance lands on exactly one rank, and the per-rank loads stay balanced; the timing reduction
takes the maximum over ranks."""
import os
import socket

import pytest
import torch
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
    import scenarios as S
    from paper_2203_04508_gb300.slab import shard_instances
    sizes = [sc.nodes for sc in S.c4_batch()]
    mine = shard_instances(sizes, world)[rank]
    load = torch.tensor([float(sum(sizes[k] for k in mine))])
    loads = [torch.zeros(1) for _ in range(world)]
    dist.all_gather(loads, load)
    ids = torch.zeros(len(sizes))
    ids[mine] = 1.0
    dist.all_reduce(ids)
    t = torch.tensor([10.0 * (rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, [float(x.item()) for x in loads], ids.tolist(), float(t.item())))
    dist.destroy_process_group()


def test_instances_shard_across_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, loads, ids, tmax in res:
        assert all(v == 1.0 for v in ids)          # every instance on exactly one rank
        assert max(loads) / min(loads) < 1.02      # balanced
        assert tmax == 20.0                        # max over ranks
