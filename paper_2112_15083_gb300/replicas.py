"""Replica ranks for the sampling bench (one process per GPU, weak scaling).

Batches are independent (Sec. II.A draws each batch's closed bits on its own), so N
ranks run independent batch groups with no data-path collective: rank r draws the batch
counters starting at r * 2^40, the step time of the job is the slowest rank's, and the
accepted samples add up.  The only collective is this end-of-run reduction.
"""
RANK_STRIDE = 1 << 40


def batch_t0(rank: int, step: int, batches_per_step: int) -> int:
    """First batch counter of `step` on `rank` (counters of different ranks never meet
    below 2^40 batches per rank)."""
    return rank * RANK_STRIDE + step * batches_per_step


def reduce_run(ms: float, accepted: float, device=None):
    """(max over ranks of ms, sum over ranks of accepted) with torch.distributed (any
    backend; a single process returns its own values)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(accepted)
    t = torch.tensor([float(ms), float(accepted)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])
