"""Column sharding across ranks (one process per GPU).

Right-hand-side columns are independent solves, so the path shards by panels
of columns with no collective in the data path: step s on rank r solves panel
(s * world + r) mod n_panels (weak scaling: every rank solves one panel per
step).  The collectives are the timing and counting reductions of the
benchmark (maximum of the times, sum of the converged pairs) and, for a caller
that wants every column's results on one rank, one gather of the outputs by
global column index (gather_columns).
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


def assemble_columns(parts):
    """Merge per-rank solver outputs into the single-rank layout, by global column index.

    parts: list of dicts with keys
      cols     int64 [c]         global indices of the columns the rank solved
      out_ptr  int64 [c+1]       kept-row offsets of those columns (as shifted_cocg_solve takes them)
      G        complex [n_out, n_z]
      ldos     float [c, n_z]    (optional)
      dm       float [n_out]     (optional)
    Returns the same keys for all columns in ascending global order, out_ptr
    rebuilt; every column must appear exactly once."""
    import numpy as np

    per_col = {}
    for p in parts:
        ptr = np.asarray(p["out_ptr"])
        for i, c in enumerate(np.asarray(p["cols"]).tolist()):
            if c in per_col:
                raise ValueError(f"column {c} solved by more than one rank")
            sl = slice(int(ptr[i]), int(ptr[i + 1]))
            per_col[c] = (p["G"][sl], None if p.get("ldos") is None else p["ldos"][i],
                          None if p.get("dm") is None else p["dm"][sl])
    cols = np.array(sorted(per_col), dtype=np.int64)
    ptr = np.zeros(len(cols) + 1, np.int64)
    ptr[1:] = np.cumsum([per_col[c][0].shape[0] for c in cols])
    out = {"cols": cols, "out_ptr": ptr, "G": np.concatenate([per_col[c][0] for c in cols])}
    if all(per_col[c][1] is not None for c in cols):
        out["ldos"] = np.stack([per_col[c][1] for c in cols])
    if all(per_col[c][2] is not None for c in cols):
        out["dm"] = np.concatenate([per_col[c][2] for c in cols])
    return out


def gather_columns(part, world: int, dst: int = 0):
    """Gathers every rank's outputs (a dict as in assemble_columns, numpy arrays)
    to rank `dst` and returns the merged single-rank layout there (None on the
    other ranks).  The one exchange of the sharded solve: columns are
    independent, so nothing else crosses ranks."""
    if world <= 1:
        return assemble_columns([part])
    import torch.distributed as dist
    parts = [None] * world if dist.get_rank() == dst else None
    dist.gather_object(part, parts, dst=dst)
    return assemble_columns(parts) if dist.get_rank() == dst else None
