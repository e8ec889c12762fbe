"""The multi-rank (weak-scaling) host logic of bench.py on two gloo ranks, CPU only.

Chains shard by global index with no exchange; each rank seeds its own chains;
the reported time is the slowest rank's.  Runs as two spawned processes talking
over 127.0.0.1.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, C, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_2603_28907_gb300 import workloads as W
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    ids = bench.rank_chains(rank, C)
    gathered = [None] * world
    dist.all_gather_object(gathered, ids)
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(4, rank))
    t = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    # a rank's starting geometries depend only on the global chain index
    w = W.tiny()
    g0 = W.geometry(w, [w.seed_init, ids[0]])
    gathered_g = [None] * world
    dist.all_gather_object(gathered_g, float(g0.sum()))
    if rank == 0:
        out.put((gathered, seeds, t, gathered_g))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_sharding_and_timing():
    world, C = 2, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, C, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, seeds, t, gsum = q.get(timeout=100)
    for p in procs:
        p.join(30)
        assert p.exitcode == 0
    flat = [i for ids in gathered for i in ids]
    assert sorted(flat) == list(range(world * C))          # disjoint and complete
    assert len(set(seeds)) == world                          # distinct keys per rank
    assert t == 11.0                                         # slowest rank's time
    from paper_2603_28907_gb300 import workloads as W
    w = W.tiny()
    assert gsum[1] == pytest.approx(float(W.geometry(w, [w.seed_init, C]).sum()))
