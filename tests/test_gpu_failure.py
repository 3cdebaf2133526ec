"""Failure detection without a GPU fault: a bounded device wait that nothing completes reports
POGS_ERR_TIMEOUT to the host, and the context stays usable (a solve right after it succeeds)."""
import time

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


def test_bounded_wait_times_out_and_the_context_stays_usable(P):
    t0 = time.perf_counter()
    rc = P.lib.pogs_check_bounded_wait(None)
    waited = time.perf_counter() - t0
    assert rc == -5, rc                   # POGS_ERR_TIMEOUT
    assert 0.2 < waited < 30.0, waited    # the budget, not a hang
    prob = W.lasso(300, 120, seed=81)
    with P.Solver(prob.A, P.pogs_default_params(max_iter=5000)) as s:
        info, *_ = s.solve(prob.f, prob.g)
    assert info.status == 0
    ref = OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=1e-9, rel_tol=1e-7, max_iter=100000))
    assert abs(info.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj))
