"""The replica path of bench.py (one box per rank, no collective on the data
path) with two gloo ranks on the CPU: the environment the launcher sets, the
maximum over ranks that gives the job's time, the whole-job throughput, and
the reference arm, whose ranks other than 0 exit without work."""
import multiprocessing as mp
import os
import socket
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    # each rank's time of its own replica; the job's time is the slowest one
    ms = 10.0 + 5.0 * r
    slowest = bench.max_over_ranks_of(ms, w, "cpu")
    value = bench.job_mlups(128 ** 3, 50, w, slowest)
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, w, local, slowest, value))


def test_two_gloo_ranks_agree_on_the_job_time_and_throughput():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    # both ranks see the slower rank's 15 ms
    assert all(r[3] == 15.0 for r in res)
    # two replicas of 128^3 nodes, 50 steps each, in 15 ms
    assert all(abs(r[4] - 2 * 128 ** 3 * 50 / 0.015 / 1e6) < 1e-6 * r[4] for r in res)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup, gpus = 3, 1, 2

    t0 = time.time()
    assert bench.run_reference(Args, workloads.workload("single")) == 0
    assert time.time() - t0 < 1.0  # no oracle step of the 128^3 box was run
    assert capsys.readouterr().out == ""  # rank 0 alone prints the line
