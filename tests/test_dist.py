"""The N > 1 path of bench.py on CPU (gloo, world size 2): replicas only, so the one collective is
the aggregation of the timed results -- the slowest rank's time and the eigenpairs of all ranks --
and the reference arm runs on rank 0 alone."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # rank r: 100 + 50 r ms, 64 (r + 1) converged eigenpairs
    ms, conv = bench.aggregate_replicas(100.0 + 50.0 * rank, 64.0 * (rank + 1), "cpu")
    tdist.barrier()
    q.put((rank, ms, conv))
    tdist.destroy_process_group()


def test_replica_aggregation_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest time and the sum of the eigenpairs: value = 192 / 0.150 s
    assert out == [(0, 150.0, 192.0), (1, 150.0, 192.0)]


def test_single_process_aggregation_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(12.5, 64, "cpu") == (12.5, 64.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class A:
        steps, warmup, workload = 1, 0, "medium"
    assert bench.run_reference(A()) is None        # returns at once: no oracle work, no output
    assert capsys.readouterr().out == ""
    assert bench.dist() == (2, 1, 1)
