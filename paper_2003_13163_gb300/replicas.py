"""Replica bookkeeping for runs on several GPUs of one node.

A single circuit does not shard: the gates of a brickwork step are applied in
sequence with canonical-form truncation (Sec. 4.1) and the end-of-step sweep
is a chain-serial recurrence. Several GPUs therefore run independent circuit
realisations (the paper averages N_s = 24 of them, Sec. 4.1): rank r simulates
the circuit of seed base + r, and the job's throughput is the work of all ranks
over the slowest rank's time. No simulation data crosses ranks; the process
group only provides the barrier and the max/sum reductions of timings.
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the circuit realisation simulated by `rank`."""
    return base_seed + rank


def seeds_for(base_seed: int, n_realisations: int, world_size: int, rank: int) -> list[int]:
    """Round-robin split of an ensemble of circuit seeds over the ranks."""
    return [base_seed + i for i in range(n_realisations) if i % world_size == rank]


def _reduce(x: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM}[op])
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    return _reduce(x, "max", device)


def sum_over_ranks(x: float, device=None) -> float:
    return _reduce(x, "sum", device)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_rate(units_this_rank: float, seconds_this_rank: float, device=None) -> tuple[float, float, float]:
    """Whole-job throughput: (sum of units over ranks) / (max time over ranks).
    Returns (rate, total_units, max_seconds)."""
    tot = sum_over_ranks(units_this_rank, device)
    tmax = max_over_ranks(seconds_this_rank, device)
    return (tot / tmax if tmax > 0 else 0.0), tot, tmax
