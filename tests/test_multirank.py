"""The bench's multi-rank path on CPU: two gloo ranks, as under torchrun with
one process per GPU.  The single-system solve runs as replicas; the batched
and served forms split whole systems (requests grouped by matrix key) over
the ranks with no collective on the data path, only host-side reductions of
times and gathers of per-request results."""
import os
import socket

import numpy as np
import pytest

import bench
import gen


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        # replicas: the slowest rank's time sets the job's rate
        t = [0.25, 0.5][rank]
        tmax = bench.max_over_ranks(t, world)
        res["value"] = world * 10 / tmax
        # batched form: this rank's systems, gathered in rank order
        mine = bench.batched_shard(rank, world)
        res["batched_all"] = bench.gather_lists(mine, world)
        # served form: this rank's requests, with their keys
        reqs = gen.serving_requests(200, 0, lo=20, hi=160)
        rk = bench.shard_requests(reqs, lambda q: q.side ** 3, world)
        res["served"] = bench.gather_lists([(q.index, q.key, rank) for q in reqs if rk[q.index] == rank], world)
        res["flags"] = bench.gather_lists([rank == 0], world)
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        res = got[r]
        # both ranks see the slowest rank's time
        assert res["value"] == pytest.approx(2 * 10 / 0.5)
        # every batched system is solved on exactly one rank
        assert sorted(res["batched_all"]) == list(range(bench.BATCH_SYSTEMS))
        assert res["flags"] == [True, False]
    assert got[0]["batched_all"] == got[1]["batched_all"]
    # every request is served once, and all requests of a key on one rank
    served = got[0]["served"]
    assert sorted(i for i, _, _ in served) == list(range(200))
    rank_of_key = {}
    for _, key, r in served:
        assert rank_of_key.setdefault(key, r) == r


def test_shard_balance():
    sides, _ = gen.batched_sides(bench.BATCH_SYSTEMS, 0)
    w = [5.0 * int(m) ** 2 for m in sides]
    for world in (1, 2, 3, 8):
        rank_of = bench.shard_by_weight(w, world)
        loads = np.bincount(rank_of, weights=w, minlength=world)
        # greedy heaviest-first: no rank exceeds the mean by more than the heaviest item
        assert loads.max() <= loads.sum() / world + max(w) + 1e-9
        assert sorted(set(rank_of)) == list(range(world))
    # deterministic and independent of the caller
    assert bench.shard_by_weight(w, 4) == bench.shard_by_weight(list(w), 4)
    # heaviest first, ties to the lower rank: 3 -> rank 0, 3 -> rank 1, 2 -> rank 0 (loads 3, 3)
    assert bench.shard_by_weight([3.0, 3.0, 2.0], 2) == [0, 1, 0]
