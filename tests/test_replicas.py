"""Host logic of `bench.py --gpus N` (replicas, one process per GPU) on CPU: two gloo
ranks rendezvous, every rank reports its own time and rank 0 reads the maximum; the
reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w, local = bench.dist_init(world)
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + rank, w)   # rank 1 is the slowest replica
    ref = bench.run_reference(type("A", (), {"config": "q1_64"})(), r, w) if r == 1 else None
    out.put((rank, t, ref))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [t for _, t, _ in res] == [2.0, 2.0]
    assert res[1][2] is None   # no oracle work on a non-zero rank
