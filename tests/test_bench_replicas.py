"""The multi-rank paths of bench.py on CPU with the gloo backend (world size 2):
whole-job throughput of independent replicas is the units all ranks completed
over the slowest rank's time, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank 0 took 10 ms for 3 good solves, rank 1 took 25 ms for 2
    ms, ok, rate = bench.job_rate([10.0, 25.0][rank], [3, 2][rank], world, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, ok, rate))


def test_job_rate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, ok, rate in res:
        assert ms == 25.0 and ok == 5
        assert rate == pytest.approx(5 / 0.025)


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_rate(20.0, 4, 1, None, "cpu") == (20.0, 4, 200.0)


def test_reference_arm_other_ranks_do_nothing(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""
