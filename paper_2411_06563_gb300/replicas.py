"""Replicas across GPUs of one node: one process per GPU, no data-path collective.

Every cavity is independent and one cavity fits one GPU, so several GPUs run replicas (the
single-cavity benchmark) or disjoint shards of a set of cavities (the batched benchmark). The
only cross-rank communication is for timing and totals: a barrier before and after the timed
region, the maximum of the per-rank times and the sum of the per-rank work. The helpers take the
device of the reduction tensor from the process group's backend (CPU tensors for gloo, the
current CUDA device for nccl), so the same code runs in the CPU tests.
"""

import os


def world():
    """(world_size, rank, local_rank) from the launcher's environment (1, 0, 0 when alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank, world_size):
    """The items of one rank: every world_size-th item from index rank (disjoint, covering)."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("rank %d outside a world of %d" % (rank, world_size))
    return list(items)[rank::world_size]


def _device():
    import torch
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def _reduce(x, op):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x):
    """The largest x over all ranks (x itself without a process group)."""
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX)


def sum_over_ranks(x):
    """The sum of x over all ranks (x itself without a process group)."""
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM)


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
