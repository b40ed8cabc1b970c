"""Column sharding across ranks (one process per GPU).

Right-hand-side columns are independent solves, so the path shards by panels
of columns with no collective in the data path: step s on rank r solves panel
(s * world + r) mod n_panels (weak scaling: every rank solves one panel per
step).  The only collectives are the timing and counting reductions of the
benchmark (maximum of the times, sum of the converged pairs).
"""
from __future__ import annotations


def panel_for(step: int, rank: int, world: int, n_panels: int) -> int:
    return (step * world + rank) % n_panels


def reduce_step_stats(ms: float, pairs: float, launches: float, world: int, device=None):
    """(max time, total pairs, total launches) over the ranks."""
    if world <= 1:
        return ms, pairs, launches
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, pairs, launches], dtype=torch.float64, device=device)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(sm[2])
