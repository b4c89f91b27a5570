"""The multi-process path of the benchmark (one replica per rank, no
collective on the data path): two gloo ranks on the CPU check the
reduction of the timed milliseconds to the slowest rank's and the whole-job
rate built from it, and that the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        ms = 100.0 + 37.5 * rank  # rank 1 is the slow one
        mx = bench.max_over_ranks(ms, dist, "cpu")
        rate = bench.job_throughput(4096 * 1024, 50, ws, mx)
        out.put((r, ws, local, mx, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units():
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
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 and r[2] == r[0] for r in res)
    for r in res:
        assert r[3] == 137.5  # the slower rank's milliseconds on every rank
        assert r[4] == pytest.approx(4096 * 1024 * 50 * 2 / 0.1375, rel=1e-12)


def test_single_process_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(10, 4, 1, 2.0) == pytest.approx(20000.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the oracle on the host cores) prints
    from rank 0; the other ranks return without work."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        warmup, steps, gpus = 3, 1, 2
    bench.run_reference(A, None)  # rank 1: no oracle, no output
    assert capsys.readouterr().out == ""
