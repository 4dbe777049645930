"""The multi-GPU path is replicas only: every rank advances its own case and
bench.py reports the units of all ranks over the slowest rank's time.  This
checks that aggregation with two CPU ranks over gloo, and that a rank which
dies between steps is noticed by the survivor (an error from its next
collective within the process-group timeout), not waited for forever."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist("gloo")
    units = 1000.0 * (rank + 1)          # rank 0: 1000 units, rank 1: 2000
    seconds = 0.5 + rank                 # rank 1 is the slowest: 1.5 s
    value, tmax, total = bench.aggregate(d, units, seconds)
    d.barrier()
    d.close()
    out.put((rank, value, tmax, total))


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax, total in res:
        assert total == 3000.0 and tmax == 1.5
        assert value == pytest.approx(2000.0)


def _dying_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import time

    import bench
    d = bench.Dist("gloo", timeout_s=5.0)
    d.barrier()                              # both ranks joined
    if rank == 1:
        os._exit(3)                          # dies between steps, no collective in flight
    t0 = time.perf_counter()
    try:
        bench.aggregate(d, 1000.0, 0.5)
        out.put((rank, "no error", time.perf_counter() - t0))
    except Exception as e:                   # noqa: BLE001 - the failure is the result
        out.put((rank, type(e).__name__, time.perf_counter() - t0))


def test_dead_rank_is_reported_not_waited_for():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    rank, what, waited = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
    assert rank == 0 and what != "no error"
    assert waited < 60.0
    assert ps[1].exitcode == 3
