"""The N > 1 host path of bench.py (replicas: one independently seeded lattice per rank, no
collective on the data path) on two gloo ranks on CPU: the job time is the slowest rank's,
the whole-job value counts every rank's cells, the ranks' stirring seeds differ, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) x 10 ms for its steps
    total_ms = bench.slowest(10.0 * (rank + 1), world, "cpu")
    value = bench.replica_mlups(world, 1024 * 1024, 20, total_ms / 1e3)
    q.put((rank, total_ms, value, bench.workload(None, rank)["seed"]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]
    assert all(abs(o[2] - 2 * 1024 * 1024 * 20 / 0.020 / 1e6) < 1e-6 for o in out)
    assert out[0][3] != out[1][3]


def test_single_rank_is_its_own_job_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest(12.5, 1, "cpu") == 12.5
    assert bench.replica_mlups(1, 1000, 10, 2.0) == 1000 * 10 / 2.0 / 1e6


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(None) is None
    assert capsys.readouterr().out == ""
