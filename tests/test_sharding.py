"""Multi-rank column sharding on CPU (gloo, world size 2): disjoint panels,
every panel covered, and the max/sum reductions of the benchmark."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1402_7285_gb300.sharding import panel_for, reduce_step_stats


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [panel_for(s, rank, world, 256) for s in range(6)]
    allp = [None] * world
    dist.all_gather_object(allp, mine)
    ms, pairs, launches = reduce_step_stats(10.0 + rank, 100.0 * (rank + 1), 7.0, world)
    if rank == 0:
        q.put((allp, ms, pairs, launches))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allp, ms, pairs, launches = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = [x for per in allp for x in per]
    assert len(set(flat)) == len(flat) == 12          # disjoint panels
    assert sorted(flat) == list(range(12))           # steps 0..5 cover panels 0..11
    assert ms == 11.0 and pairs == 300.0 and launches == 14.0


def test_single_rank_is_identity():
    assert reduce_step_stats(5.0, 3.0, 2.0, 1) == (5.0, 3.0, 2.0)
    assert [panel_for(s, 0, 1, 4) for s in range(6)] == [0, 1, 2, 3, 0, 1]
