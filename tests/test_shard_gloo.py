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


# ---------------------------------------------------------------------------
# Row bands of one frame (a frame split across ranks)
# ---------------------------------------------------------------------------

def test_row_bands_partition_rows():
    for H in (1, 2, 7, 64, 513):
        for k in (3, 5, 9, 21):
            for parts in (1, 2, 3, 5, 8, 600):
                bands = shard.row_bands(H, k, parts)
                assert len(bands) == parts
                r = (k - 1) // 2
                y = 0
                heights = []
                for b in bands:
                    assert b.y0 == y and b.y1 >= b.y0
                    heights.append(b.y1 - b.y0)
                    if b.y1 > b.y0:
                        assert b.h0 == max(0, b.y0 - r) and b.h1 == min(H, b.y1 + r)
                    y = b.y1
                assert y == H and max(heights) - min(heights) <= 1


def test_row_bands_reject_bad_args():
    for args in ((0, 3, 2), (10, 4, 2), (10, 1, 2), (10, 3, 0)):
        with pytest.raises(ValueError):
            shard.row_bands(*args)


def _stitch_bands(frame, k, parts, border="replicate"):
    """Filter every halo-extended band as a frame of its own with the oracle and
    keep its own rows."""
    import oracle
    out = np.empty_like(frame)
    flagged = 0
    for b in shard.row_bands(frame.shape[0], k, parts):
        if b.y1 == b.y0:
            continue
        sub, _ = oracle.fnr_border(np.ascontiguousarray(frame[b.h0:b.h1]), k, border)
        out[b.y0:b.y1] = sub[b.y0 - b.h0:b.y1 - b.h0]
    return out


@pytest.mark.parametrize("border", ["replicate", "mirror", "zero"])
def test_bands_with_halo_equal_whole_frame(border):
    """Bands + halo == whole frame, for every border reading, including bands
    thinner than the halo and more bands than rows."""
    import oracle
    rng = np.random.default_rng(11)
    for H, W in ((1, 9), (5, 6), (23, 17), (64, 40)):
        for k in (3, 5, 9):
            f = rng.integers(0, 256, (H, W)).astype(np.uint8)
            want, _ = oracle.fnr_border(f, k, border)
            for parts in (1, 2, 3, 7, H + 3):
                np.testing.assert_array_equal(_stitch_bands(f, k, parts, border), want)


def test_band_without_halo_differs():
    """The halo is needed: filtering the bare bands changes rows next to the
    cuts (checks that the test above can fail)."""
    import oracle
    f = synth.make_frame(64, 80, synth.U8, 5, 2.0, 0.2)
    want, _ = oracle.fnr(f, 5)
    got = np.empty_like(f)
    for b in shard.row_bands(64, 5, 4):
        got[b.y0:b.y1] = oracle.fnr(np.ascontiguousarray(f[b.y0:b.y1]), 5)[0]
    assert not np.array_equal(got, want)


def _band_rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        H, W, k = 97, 61, 7
        f = synth.make_frame(H, W, synth.U14, 77, 8.0, 0.2)
        b = shard.row_bands(H, k, world)[rank]
        # each rank holds only its halo-extended rows, as on its own device
        local = np.ascontiguousarray(f[b.h0:b.h1])
        sub, _ = oracle.fnr(local, k)
        mine = sub[b.y0 - b.h0:b.y1 - b.h0]
        payload = [None] * world
        dist.all_gather_object(payload, (b.y0, b.y1, mine))
        if rank == 0:
            out = np.empty_like(f)
            for y0, y1, rows in payload:
                out[y0:y1] = rows
            q.put(bool(np.array_equal(out, oracle.fnr(f, k)[0])))
    finally:
        dist.destroy_process_group()


def test_band_split_across_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    ok = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ok
