"""Sharding of the batched workload across ranks: partition properties on the
CPU and a world-size-2 gloo run of the rank-local logic (no GPU)."""

import os
import socket

import pytest

from paper_2105_01533_gb300 import shard
from paper_2105_01533_gb300 import workloads as W


def test_lpt_partition_properties():
    works = [5, 9, 1, 1, 7, 3, 3, 2, 8, 4]
    parts = shard.lpt_partition(works, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(works)))
    loads = [sum(works[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(works)
    assert shard.lpt_partition(works, 3) == parts          # deterministic
    assert shard.lpt_partition(works, 1) == [list(range(len(works)))]
    with pytest.raises(ValueError):
        shard.lpt_partition(works, 0)


def test_circuit_work_orders_by_size():
    cs = W.batched_workload_fast(8, first_seed=40)
    w = [shard.circuit_work(c) for c in cs]
    assert all(x > 0 for x in w)
    big = max(range(8), key=lambda i: w[i])
    assert cs[big].cap * len(cs[big].gates) >= min(c.cap * len(c.gates) for c in cs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cs = W.batched_workload_fast(40, first_seed=70, depth=(200, 400))
    mine = shard.my_share(cs, rank, world)
    upd = float(sum(len(c.gates) for c in mine))
    secs = 1.0 + rank
    tot_u, max_s = shard.reduce_totals(upd, secs)
    q.put((rank, [c.seed for c in mine], upd, tot_u, max_s))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_are_disjoint_and_cover():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    seeds0, seeds1 = set(out[0][1]), set(out[1][1])
    assert not (seeds0 & seeds1) and len(seeds0 | seeds1) == 40
    total = out[0][2] + out[1][2]
    for r in out:
        assert r[3] == total and r[4] == 2.0
