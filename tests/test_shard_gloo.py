"""Multi-rank frame sharding on CPU (gloo, world size 2 and 3).

Each rank computes its own shard of the mixed 256-frame batch with no
communication; an all-gather then checks that the shards are disjoint,
cover every frame, and are balanced to within one largest frame. Every rank
also filters two small frames of its shard with the oracle and the gathered
flagged counts are compared with a single-process run.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1201_3972_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        specs = synth.workload_batch()
        work = [s.pixels for s in specs]
        mine = shard.shard(work, world, rank)
        counts = []
        for i in mine[:2]:
            s = specs[i]
            f = synth.make_frame(48, 64, s.dtype, s.seed, s.sigma, s.p)
            counts.append(oracle.fnr(f, s.k)[1])
        payload = [None] * world
        dist.all_gather_object(payload, (mine, sum(work[i] for i in mine), counts))
        if rank == 0:
            q.put(payload)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_shards_are_disjoint_complete_balanced(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    payload = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    specs = synth.workload_batch()
    work = [s.pixels for s in specs]
    allidx = sorted(i for mine, _, _ in payload for i in mine)
    assert allidx == list(range(len(specs)))
    loads = [ld for _, ld, _ in payload]
    assert max(loads) - min(loads) <= max(work)
    assert sum(loads) == sum(work)
    import oracle
    for r, (mine, _, counts) in enumerate(payload):
        for i, c in zip(mine[:2], counts):
            s = specs[i]
            f = synth.make_frame(48, 64, s.dtype, s.seed, s.sigma, s.p)
            assert oracle.fnr(f, s.k)[1] == c


def test_assignment_is_deterministic_and_local():
    work = [5, 9, 1, 9, 3, 7]
    a = shard.assignment(work, 2)
    assert a == shard.assignment(work, 2)
    assert sorted(shard.shard(work, 2, 0) + shard.shard(work, 2, 1)) == list(range(6))
    with pytest.raises(ValueError):
        shard.shard(work, 2, 2)
