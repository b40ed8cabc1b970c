"""Multi-rank column sharding on CPU (gloo, world size 2): disjoint panels,
every panel covered, the max/sum reductions of the benchmark, and the gather
of per-rank outputs (G, LDOS, DM of a test-only stub solver) into the layout
a single rank produces."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import numpy as np

from paper_1402_7285_gb300.sharding import assemble_columns, gather_columns, panel_for, reduce_step_stats


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


N_PANELS, W, NZ = 6, 4, 3


def _stub_panel(k):
    """Outputs a solve of panel k would give (deterministic stand-in, no GPU):
    column c keeps 2 + c % 3 rows, G = c + i*row + 1j*m, LDOS = c + m, DM = c - row."""
    cols = np.arange(k * W, (k + 1) * W, dtype=np.int64)
    rows = [np.arange(2 + c % 3) for c in cols]
    ptr = np.zeros(W + 1, np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    G = np.concatenate([(c + 10.0 * r)[:, None] + 1j * np.arange(NZ)[None, :] for c, r in zip(cols, rows)])
    ldos = np.stack([c + np.arange(NZ, dtype=np.float64) for c in cols])
    dm = np.concatenate([c - r.astype(np.float64) for c, r in zip(cols, rows)])
    return {"cols": cols, "out_ptr": ptr, "G": G, "ldos": ldos, "dm": dm}


def _local_part(rank, world):
    mine = sorted({panel_for(s, rank, world, N_PANELS) for s in range(N_PANELS // world)})
    parts = [_stub_panel(k) for k in mine]
    return assemble_columns(parts)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [panel_for(s, rank, world, 256) for s in range(6)]
    allp = [None] * world
    dist.all_gather_object(allp, mine)
    ms, pairs, launches = reduce_step_stats(10.0 + rank, 100.0 * (rank + 1), 7.0, world)
    merged = gather_columns(_local_part(rank, world), world)
    if rank == 0:
        q.put((allp, ms, pairs, launches, merged))
    else:
        assert merged is None
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allp, ms, pairs, launches, merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = [x for per in allp for x in per]
    assert len(set(flat)) == len(flat) == 12          # disjoint panels
    assert sorted(flat) == list(range(12))           # steps 0..5 cover panels 0..11
    assert ms == 11.0 and pairs == 300.0 and launches == 14.0
    single = assemble_columns([_stub_panel(k) for k in range(N_PANELS)])   # what one rank would hold
    for key in ("cols", "out_ptr", "G", "ldos", "dm"):
        assert np.array_equal(merged[key], single[key]), key


def test_assemble_rejects_a_column_solved_twice():
    with pytest.raises(ValueError):
        assemble_columns([_stub_panel(0), _stub_panel(0)])


def test_single_rank_is_identity():
    assert reduce_step_stats(5.0, 3.0, 2.0, 1) == (5.0, 3.0, 2.0)
    assert [panel_for(s, 0, 1, 4) for s in range(6)] == [0, 1, 2, 3, 0, 1]
