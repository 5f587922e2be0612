"""Host-side logic of the multi-GPU ensemble run (one process per GPU).

Samples are independent (Sec. 2.4: every MLMC sample is its own solve), so
the ranks split the ensemble into disjoint blocks of sample ids and never
exchange data while solving.  After a timed region the job's throughput is
the work of all ranks divided by the slowest rank's time: one all-reduce of
the elapsed time (MAX) and one of the work (SUM).  The functions take the
process group's tensors on whatever device the backend uses (NCCL: CUDA,
gloo: CPU), so the same code runs in the benchmark and in CPU tests.

The estimator is the one exchange step of a multi-process OF-MLMC run: each
rank solves a level-stratified share of every level's pairs, and the
per-level summaries are exchanged once per estimator iteration.
"""
from typing import List, Tuple


def rank_sample_ids(rank: int, per_rank: int) -> List[int]:
    """Sample ids of one rank: the block [rank * per_rank, (rank + 1) * per_rank).
    Blocks of different ranks are disjoint and together cover 0 .. world * per_rank - 1."""
    if rank < 0 or per_rank < 0:
        raise ValueError("rank and per_rank must be non-negative")
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def aggregate(elapsed: float, work: float, world: int, device="cpu") -> Tuple[float, float]:
    """(max over ranks of elapsed, sum over ranks of work); world == 1 needs no process group."""
    if world <= 1:
        return float(elapsed), float(work)
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def job_rate(elapsed_all: float, work_all: float) -> float:
    """Whole-job throughput: all ranks' work over the slowest rank's elapsed time."""
    if not elapsed_all > 0.0:
        raise ValueError("elapsed time must be positive")
    return work_all / elapsed_all


def pair_shard(M: int, rank: int, world: int) -> range:
    """Pairs of one level a rank solves: indices rank, rank + world, ... (level-stratified,
    so every rank holds a share of every level)."""
    if world < 1 or not 0 <= rank < world or M < 0:
        raise ValueError("bad shard arguments")
    return range(rank, M, world)


def distributed_estimate(local_pairs, W, world: int, device="cpu", fit: bool = False) -> dict:
    """The OF-MLMC estimate of all ranks' pairs: each rank summarises its own
    pairs per level (ofm_level_moments_of), the summaries are all-gathered
    (6 doubles per level and rank), combined in rank order (ofm_merge_moments)
    and evaluated (ofm_estimate_moments, or with fit the fitted estimator);
    every rank returns the same result."""
    from . import api
    local = [api.level_moments(p) for p in local_pairs]
    if world <= 1:
        return api.estimate_moments(local, W, fit=fit)
    import torch
    import torch.distributed as dist
    t = torch.tensor([[float(x) for x in m] for m in local], dtype=torch.float64, device=device)
    parts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    merged = None
    for part in parts:
        rows = [(int(r[0]), *[float(x) for x in r[1:]]) for r in part.cpu().tolist()]
        merged = rows if merged is None else [api.merge_moments(a, b) for a, b in zip(merged, rows)]
    return api.estimate_moments(merged, W, fit=fit)
