"""The multi-process path of bench.py on CPU (gloo, world size 2): each rank runs an independent
replica of the workload, the timed region ends with an element-wise max over ranks, and the
whole-job throughput counts every rank's units over the slowest time.  No collective touches
the data path; this checks the rank bookkeeping, the max and the aggregate, and that a rank
that leaves makes the others' next collective end with an error instead of waiting."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    w, r, local = bench._dist()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        # per-rank step times (seconds) and a second value that is larger on rank 0
        vals = bench._max_over_ranks([1.0 + rank, 10.0 - rank], w)
        dist.barrier()
        out.put((r, w, local, vals, bench._replica_rate(w, 1000, vals[0])))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 and g[2] == g[0] for g in got)
    for _, _, _, vals, rate in got:
        assert vals == [2.0, 10.0]                 # the slowest rank's time, element by element
        assert rate == pytest.approx(2 * 1000 / 2.0)


def test_single_process_defaults(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist() == (1, 0, 0)
    assert bench._max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench._replica_rate(1, 500, 2.0) == 250.0


def _leaver(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    bench._init_group("gloo", timeout_s=5.0)
    if rank == 1:
        out.put((rank, "left"))          # leaves between steps, with no collective in flight
        return
    import time
    t0 = time.time()
    try:
        bench._max_over_ranks([1.0], world)
        out.put((rank, "no error"))
    except Exception as e:               # the group's timeout ends the collective
        out.put((rank, "error after %.1f s: %s" % (time.time() - t0, type(e).__name__)))


def test_a_rank_that_leaves_ends_the_others_collective():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaver, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert got[1] == "left"
    assert got[0].startswith("error after"), got[0]
