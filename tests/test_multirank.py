"""The N > 1 host logic of the benchmark on CPU, with world_size-2 gloo ranks:
replicas reduce their step times by max over ranks, and the batched scan
shards whole instances across ranks (largest first onto the least-loaded
rank) with no instance lost or duplicated."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    from relsim_inputs import tearing_scan
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, dist)
        insts = tearing_scan(48, seed=0)
        sizes = [2 * hc.nx * hc.ny * hc.ppc for hc in insts]
        owner = bench.lpt_shard(sizes, world)
        mine = [i for i in range(len(insts)) if owner[i] == rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        q.put((rank, t, got, sizes))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_times_and_shard_the_scan():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, got, sizes in res:
        assert t == 2.5                      # max over ranks of 1.5 + rank
        a, b = got
        assert sorted(a + b) == list(range(48)) and not set(a) & set(b)
        la, lb = sum(sizes[i] for i in a), sum(sizes[i] for i in b)
        assert abs(la - lb) <= max(sizes)    # LPT: within one instance
    assert res[0][2] == res[1][2]            # both ranks see the same partition


def test_lpt_shard_single_rank_takes_everything():
    import bench
    assert bench.lpt_shard([5, 3, 9], 1) == [0, 0, 0]
    owner = bench.lpt_shard([10, 1, 1, 1, 7], 2)
    assert owner[0] != owner[4]
