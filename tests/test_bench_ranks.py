"""Multi-rank logic of bench.py on CPU (gloo, world size 2): replicas only, so
the group carries just the barrier and the max / sum of per-rank numbers."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    w, r, local, pg = bench.dist_setup(backend="gloo")
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(pg, local)
    mx = bench.max_over_ranks(pg, float(10 * (rank + 1)), local)
    sm = bench.sum_over_ranks(pg, float(rank + 1), local)
    out.put((rank, mx, sm))
    pg.destroy_process_group()


def test_two_gloo_ranks_reduce_timings():
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
    assert res == [(0, 20.0, 3.0), (1, 20.0, 3.0)]


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, mode, steps, warmup = "sbm8192", "async", 1, 3
    assert bench.bench_reference(A()) is None
    assert capsys.readouterr().out == ""
