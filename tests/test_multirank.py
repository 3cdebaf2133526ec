"""The N > 1 path of bench.py on CPU: two gloo ranks launched as torchrun would launch them.

The path shards by replicas (each rank solves its own independent instances, no collective on
the data path), so what is tested is the host logic around it: rendezvous, the barrier, the
maximum of the ranks' timed intervals, the whole-job rate computed from it, and that the ranks
run distinct problem instances.  A rank that fails raises on the host; the test sees it."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q, fail_rank):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank), POGS_DIST_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    try:
        dist, r, w, local = bench._dist()
        assert (r, w, local) == (rank, ws, rank)
        if rank == fail_rank:
            raise RuntimeError(f"rank {rank} failed before its first step")
        bench._barrier(dist)
        t_ms = 100.0 + 50.0 * rank          # each rank's own timed interval
        t_max = bench._max_over_ranks(dist, t_ms)
        rate = bench.job_rate(10, w, t_max)
        bench._barrier(dist)
        q.put((rank, t_max, rate, bench.problem_seeds(rank)))
        dist.destroy_process_group()
    except Exception as e:   # report to the parent instead of hanging it
        q.put((rank, "error", repr(e), None))


def _run(ws, fail_rank=-1, timeout=60):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q, fail_rank)) for r in range(ws)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(ws if fail_rank < 0 else 1):
            rank, a, b, c = q.get(timeout=timeout)
            out[rank] = (a, b, c)
    finally:
        for p in procs:
            p.join(timeout=5 if fail_rank >= 0 else timeout)
            if p.is_alive():
                p.kill()
                p.join()
    return out


def test_two_gloo_ranks_report_the_max_interval_and_whole_job_rate():
    out = _run(2)
    assert sorted(out) == [0, 1]
    for rank, (t_max, rate, seeds) in out.items():
        assert t_max == 150.0                         # max over ranks, seen by every rank
        assert rate == pytest.approx(10 * 2 / 0.150)  # all ranks' units over the slowest time
    assert out[0][2] != out[1][2]                     # replicas run distinct instances
    assert out[0][2] == (10_000, 10_001)              # rank 0 runs the named workload


def test_a_failing_rank_is_reported_on_the_host():
    out = _run(2, fail_rank=1, timeout=60)
    assert out[1][0] == "error" and "failed before its first step" in out[1][1]
