"""Host-side logic of the multi-GPU ensemble run (one process per GPU).

Samples are independent (Sec. 2.4: every MLMC sample is its own solve), so
the ranks split the ensemble into disjoint blocks of sample ids and never
exchange data while solving.  After a timed region the job's throughput is
the work of all ranks divided by the slowest rank's time: one all-reduce of
the elapsed time (MAX) and one of the work (SUM).  The functions take the
process group's tensors on whatever device the backend uses (NCCL: CUDA,
gloo: CPU), so the same code runs in the benchmark and in CPU tests.
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
