"""The multi-GPU path (replicas and shards, timing collectives only) with two gloo ranks on the
CPU: shards are disjoint and cover the set, the time is the maximum over ranks, the work the sum."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2411_06563_gb300 import inputs, replicas as R  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, _ = R.world()
        cavs = inputs.batch_mix()
        mine = R.shard(cavs, r, ws)
        pts = sum((c["N"] - 2) ** 3 for c in mine)
        R.barrier()
        t = 1.0 + 0.5 * r                   # a per-rank "time"
        out[rank] = (len(mine), R.sum_over_ranks(len(mine)), R.max_over_ranks(t),
                     R.sum_over_ranks(pts), pts, [c["N"] for c in mine][:3])
        R.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    cavs = inputs.batch_mix()
    total_pts = sum((c["N"] - 2) ** 3 for c in cavs)
    for rank in range(world):
        n_mine, n_all, t_max, pts_all, _, first = out[rank]
        assert n_all == len(cavs) and t_max == 1.5 and pts_all == total_pts
        assert first == [c["N"] for c in cavs[rank::world]][:3]
    assert out[0][0] + out[1][0] == len(cavs)
    assert out[0][4] + out[1][4] == total_pts


def test_shard_without_process_group():
    items = list(range(7))
    parts = [R.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert R.max_over_ranks(2.5) == 2.5 and R.sum_over_ranks(4) == 4.0
    with pytest.raises(ValueError):
        R.shard(items, 3, 3)
