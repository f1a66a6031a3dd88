"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank simulates its own problem,
the only collectives are a barrier and a max over ranks, and the whole-job value counts every rank's work
divided by the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    ws, r, local = bench.dist_env()
    dist = bench.dist_init(ws)
    bench.barrier(dist)
    t_local = 100.0 + 50.0 * r          # rank 1 is the slow one
    t_max = bench.allmax(dist, t_local)
    gates, steps = 1780, 3
    value = gates * steps * ws / (t_max / 1000.0)
    out.put((r, ws, local, t_max, value))
    dist.destroy_process_group()


def test_two_rank_barrier_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 150.0 for r in res)  # every rank sees the slowest rank's time
    assert res[0][4] == pytest.approx(1780 * 3 * 2 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    ws, r, _ = bench.dist_env()
    assert (ws, r) == (1, 0)
    assert bench.dist_init(1) is None
    assert bench.allmax(None, 3.5) == 3.5
