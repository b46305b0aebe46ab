"""Host-side logic of the multi-GPU replica mode: one process per GPU, independent systems.

Frequencies (or right-hand sides) are independent units of work, so N GPUs run N replicas of the
solver, each on a contiguous block of the sweep, with no collective on the data path.  What the
ranks share is host-side bookkeeping only, done here with ``torch.distributed`` on whatever process
group the caller set up (NCCL on GPU machines, gloo for the CPU tests):

* ``block(n, world, rank)``: the contiguous block of n units that a rank owns;
* ``max_over_ranks(value)``: the slowest rank's time, which defines the job's time;
* ``gather_to_rank0(obj)``: per-rank reports collected on rank 0 (in rank order).
"""
from __future__ import annotations


def block(n: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of the n units owned by ``rank``: contiguous blocks, sizes differing by at most one,
    the larger blocks first; every unit is owned by exactly one rank."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad partition request n={n} world={world} rank={rank}")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def max_over_ranks(value: float) -> float:
    """The largest ``value`` over all ranks (the job's time is its slowest rank's); the value itself
    when no process group is set up."""
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(value)
    import torch
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_to_rank0(obj):
    """A list of every rank's ``obj`` (index = rank) on rank 0, None on the other ranks; [obj] when
    no process group is set up."""
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out
