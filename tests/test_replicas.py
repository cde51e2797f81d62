"""Host logic of the multi-GPU replicas, on CPU: the per-rank partition of a
ragged batch and the max-over-ranks timing reduction, with two gloo ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1809_06839_gb300 import synth
from paper_1809_06839_gb300.replicas import max_over_ranks, shard_by_pixels


def check_partition(sizes, world):
    slices = [shard_by_pixels(sizes, world, r) for r in range(world)]
    assert slices[0][0] == 0 and slices[-1][1] == len(sizes)
    for (a, b), (c, d) in zip(slices, slices[1:]):
        assert b == c and a <= b
    px = [sum(h * w for h, w in sizes[a:b]) for a, b in slices]
    biggest = max((h * w for h, w in sizes), default=0)
    mean = sum(px) / world
    assert all(abs(p - mean) <= biggest for p in px), (px, mean, biggest)
    return slices


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_is_contiguous_and_balanced(world):
    sizes = synth.uniform_sizes(2000, 333, 500, seed=5)
    check_partition(sizes, world)
    ragged = synth.uniform_sizes(97, 16, 1024, seed=6)
    check_partition(ragged, world)


def test_partition_edge_cases():
    assert shard_by_pixels([], 2, 0) == (0, 0) and shard_by_pixels([], 2, 1) == (0, 0)
    check_partition([(10, 10)], 4)                      # fewer images than ranks
    check_partition([(1000, 1000)] + [(1, 1)] * 50, 3)  # one dominant image
    with pytest.raises(ValueError):
        shard_by_pixels([(1, 1)], 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = synth.uniform_sizes(300, 64, 900, seed=9)
        mine = shard_by_pixels(sizes, world, rank)
        got = [None] * world
        dist.all_gather_object(got, mine)
        t = max_over_ranks(0.5 + rank, dist, torch.device("cpu"))
        dist.barrier()
        q.put((rank, got, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_shards_and_timing():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = synth.uniform_sizes(300, 64, 900, seed=9)
    expect = check_partition(sizes, world)
    for rank, got, t in res:
        assert [tuple(g) for g in got] == expect
        assert t == 1.5                                   # the slower rank's time on every rank
