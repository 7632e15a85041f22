"""Sharding of one reconstruction over several GPUs (one process each).

The final contraction's rows are the high output bits (Kronecker order), so
a rank that writes rows [r0, r1) writes the contiguous output range
[r0 * cols, r1 * cols): no exchange is needed on the data path.  The only
collective is the max-over-ranks of the step time (and, if wanted, the sum of
the per-rank totals)."""
from __future__ import annotations


def row_range(rows: int, world: int, rank: int):
    """Contiguous, balanced split of `rows` rows: the first rows % world ranks
    get one extra row."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(rows, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, group=None):
    """Max of a per-rank float over the process group (CPU tensor for gloo,
    device tensor for nccl)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
