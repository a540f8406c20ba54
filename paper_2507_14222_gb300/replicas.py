"""Running IG on several GPUs of one node: independent replicas.

IG's problems -- a fit and the scoring of its flows -- are independent, so
N ranks (one process per GPU) each take their own problems and no data
crosses between them.  What the ranks share is bookkeeping only: which
problems each one takes, and the job's totals (the slowest rank's time, the
work summed over ranks), exchanged once per measurement through
torch.distributed (NCCL on GPUs, gloo on CPU hosts).
"""
from __future__ import annotations

SEED_STRIDE = 7919  # seed offset between ranks' synthetic problems (a prime)


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank's own problem: rank 0 keeps the base seed."""
    return base + SEED_STRIDE * rank


def assign(n_items: int, rank: int, world: int) -> range:
    """The contiguous block of item indices rank takes out of n_items: block
    sizes differ by at most one, lower ranks take the larger blocks."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("need 0 <= rank < world and n_items >= 0")
    per, extra = divmod(n_items, world)
    lo = rank * per + min(rank, extra)
    return range(lo, lo + per + (1 if rank < extra else 0))


def _dist():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        return dist
    return None


def job_totals(elapsed_ms: float, units: float, device=None) -> tuple[float, float]:
    """(largest elapsed_ms over ranks, sum of units over ranks).

    Collective: every rank must call it.  `device` is where the exchange
    tensor lives ("cuda" under NCCL, None / "cpu" under gloo).  Without an
    initialised process group of more than one rank it returns its inputs.
    """
    dist = _dist()
    if dist is None:
        return float(elapsed_ms), float(units)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(device_ids=None):
    """Barrier over all ranks (no-op on one rank)."""
    dist = _dist()
    if dist is not None:
        if device_ids is not None:
            dist.barrier(device_ids=device_ids)
        else:
            dist.barrier()
