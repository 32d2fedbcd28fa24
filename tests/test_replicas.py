"""The N > 1 host path on CPU: world_size-2 gloo ranks shard a batch of
independent graphs, solve their shards (with the oracle, standing in for the
device), and meet only at the barrier and the max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_2407_07058_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shards_are_a_balanced_partition():
    sizes = [int(x) for x in synth.cfg4_sizes(4096)]
    for world in (1, 2, 3, 4, 8):
        parts = replicas.shard_graphs(sizes, world)
        flat = sorted(g for p in parts for g in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[g] ** 2 for g in p) for p in parts]
        # LPT bound: no rank exceeds the mean by more than the largest graph
        assert max(loads) - sum(loads) / world <= max(sizes) ** 2
        assert parts == replicas.shard_graphs(sizes, world)   # deterministic
    assert replicas.shard_graphs([], 2) == [[], []]
    assert replicas.shard_graphs([5], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        replicas.shard_graphs(sizes, 0)
    with pytest.raises(ValueError):
        replicas.rank_graphs(sizes, 2, 2)


def test_helpers_without_a_process_group():
    replicas.barrier()
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.sum_over_ranks(2.0) == 2.0


def _rank_main(rank, world, port, sizes, q):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.rank_graphs(sizes, rank, world)
        out = {g: oracle.appd(synth.uniform01(sizes[g], seed=900 + g)).view(np.uint32).tobytes()
               for g in mine}
        replicas.barrier()
        ms = replicas.max_over_ranks(10.0 + rank)
        units = replicas.sum_over_ranks(float(sum(sizes[g] ** 2 for g in mine)))
        gathered = [None] * world
        dist.all_gather_object(gathered, out)
        if rank == 0:
            merged = {}
            for part in gathered:
                assert not set(part) & set(merged)
                merged.update(part)
            q.put((ms, units, merged))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_time():
    sizes = [3, 17, 1, 40, 9, 33, 2, 64, 5]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    ms, units, merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert ms == 11.0
    assert units == float(sum(n * n for n in sizes))
    import oracle
    assert sorted(merged) == list(range(len(sizes)))
    for g, n in enumerate(sizes):
        ref = oracle.appd(synth.uniform01(n, seed=900 + g)).view(np.uint32).tobytes()
        assert merged[g] == ref
