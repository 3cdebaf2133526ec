"""The serving workload's oracle check (bench.oracle_sample_check), on the CPU: it solves a
bounded sample of the distinct payloads with the oracle, times that as the CPU baseline, and
compares every served objective for a sampled payload with the oracle's."""
import workloads as W
from oracle import admm as OA


def test_oracle_sample_check_bookkeeping():
    import bench
    pool = [W.lasso(60, 30, seed=1), W.nnls(50, 20, seed=2), W.huber(40, 25, seed=3)]
    ref = [OA.solve(p.A, p.f, p.g, OA.Params()).obj for p in pool]
    served = {0: [ref[0], ref[0]], 1: [ref[1] * (1 + 5e-3)], 2: [ref[2]]}
    cpu, check = bench.oracle_sample_check(pool, served, seconds=60.0)
    assert check["payloads"] == 3 and check["oracle_converged"] == 3
    assert check["requests_checked"] == 4
    assert check["within_1e_3"] == 3 and check["within_1e_2"] == 4
    assert abs(check["max_rel_obj_err"] - 5e-3 * abs(ref[1]) / max(1.0, abs(ref[1]))) < 1e-12
    assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["cores"] >= 1
    assert cpu["cpu_count"] >= 1 and "value_1thread" not in cpu
    # one BLAS thread: a child process rebuilds the pool from the expression it is given
    cpu1, _ = bench.oracle_sample_check(
        pool, served, seconds=60.0, one_thread_seconds=60.0,
        one_thread_pool="[W.lasso(60, 30, seed=1), W.nnls(50, 20, seed=2), W.huber(40, 25, seed=3)]")
    assert cpu1["value_1thread"] > 0 and "first 3 " in cpu1["sample_1thread"]
    # the sample is bounded: with no time allowed, only the first payload is solved
    cpu0, check0 = bench.oracle_sample_check(pool, served, seconds=0.0)
    assert check0["payloads"] == 1 and check0["requests_checked"] == 2
