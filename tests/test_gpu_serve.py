"""Continuous-batching server: each request's result is the same alone and in the mix,
requests admitted while others are on the GPU join and finish, admission respects the memory
budget, and results match the FP64 oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import admm as OA

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_08366_b300 as P
    return P


def _mix():
    """Small (batched engine) and large (min(m, n) > 512, single-problem path) requests."""
    probs = [W.CLASSES[c](m, n, seed=90_000 + i) for i, (c, m, n) in enumerate([
        ("lasso", 400, 120), ("huber", 900, 60), ("svm", 300, 90), ("nnls", 120, 300), ("logistic", 500, 80),
        ("lasso", 1300, 700), ("nnls", 800, 600), ("huber", 250, 40), ("logistic", 150, 400), ("svm", 2000, 300),
        ("lasso", 700, 520), ("nnls", 64, 32),
        # longest side past the shared-memory vector staging, not a multiple of four (arena vectors)
        ("lasso", 2501, 301), ("nnls", 150, 2403)])]
    return probs


def _serve(P, probs, budget=8 << 30, iters=25, stagger=False):
    out = {}
    with P.Server(budget, large_workers=3, max_resident=64, params=P.pogs_default_params(max_iter=5000)) as srv:
        half = len(probs) // 2 if stagger else len(probs)
        for i in range(half):
            srv.submit(probs[i], i)
        if stagger:            # the rest arrive while the first half is running on the GPU
            srv.step(iters)
            for i in range(half, len(probs)):
                srv.submit(probs[i], i)
        guard = 0
        while srv.pending() > 0:
            srv.step(iters)
            for tag, info, *_times, x, y, mu, nu in srv.poll():
                out[tag] = (info, x, y, mu, nu)
            guard += 1
            assert guard < 100000
        for tag, info, *_times, x, y, mu, nu in srv.poll():
            out[tag] = (info, x, y, mu, nu)
    return out


def test_each_result_is_the_same_alone_and_in_the_mix(P):
    probs = _mix()
    mix = _serve(P, probs, stagger=True)
    assert sorted(mix) == list(range(len(probs)))
    for i, prob in enumerate(probs):
        alone = _serve(P, [prob])[0]
        a, b = mix[i], alone
        assert a[0].status == 0 and b[0].status == 0, (i, a[0].status, b[0].status)
        assert a[0].iters == b[0].iters and a[0].obj == b[0].obj, (i, a[0].iters, b[0].iters)
        for u, v in zip(a[1:], b[1:]):
            assert np.array_equal(u, v), i


def test_served_results_match_oracle(P):
    probs = _mix()
    res = _serve(P, probs)
    for i in (0, 2, 3, 5, 7, 10, 12, 13):
        ref = OA.solve(probs[i].A, probs[i].f, probs[i].g, OA.Params(abs_tol=1e-9, rel_tol=1e-7, max_iter=50000))
        assert abs(res[i][0].obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj)), (i, res[i][0].obj, ref.obj)


def test_budget_limits_admission_and_oversized_requests_are_refused(P):
    probs = [W.lasso(300, 100, seed=s) for s in range(6)]
    # a budget that holds about one request at a time still completes them all, in order
    res = _serve(P, probs, budget=3 << 20, iters=10)
    assert sorted(res) == list(range(6)) and all(r[0].status == 0 for r in res.values())
    with P.Server(1 << 20, large_workers=0, max_resident=4) as srv:
        with pytest.raises(P.PogsError) as ei:
            srv.submit(W.lasso(2000, 400, seed=1), 0)
        assert ei.value.code == -7
