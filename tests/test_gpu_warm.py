"""Warm start and factor reuse (Section 5) on the CUDA path, against the FP64 oracle.

A handle keeps A^, its equilibration and the factor of I + A^T A; pogs_solve_warm starts the
iteration from a given x0 and/or nu0.  Tolerances as the solve parity tests:
|obj - p*| <= 1e-3 max(1, |p*|) with p* from the oracle at eps_rel = 1e-7."""
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


def _tight(prob):
    return OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=1e-9, rel_tol=1e-7, max_iter=100000))


@pytest.mark.parametrize("cls,shape", [("lasso", (600, 250)), ("logistic", (300, 700)), ("huber", (800, 200))])
def test_warm_start_at_the_oracle_solution_converges_at_once(P, cls, shape):
    prob = W.CLASSES[cls](*shape, seed=41)
    ref = _tight(prob)
    prm = P.pogs_default_params(max_iter=2000)
    with P.Solver(prob.A, prm) as s:
        cold, *_ = s.solve(prob.f, prob.g)
        warm, x, y, mu, nu = s.solve(prob.f, prob.g, x0=ref.x.astype(np.float32), nu0=ref.nu.astype(np.float32))
    assert cold.status == 0 and warm.status == 0
    assert warm.iters <= 3 < cold.iters, (warm.iters, cold.iters)
    assert abs(warm.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj)), (warm.obj, ref.obj)


def test_lasso_path_reuses_the_factor_and_warm_starts(P):
    """One setup, five regularisation weights, each solve started from the previous solution."""
    base = W.lasso(900, 400, seed=43)
    lam_max = float(np.max(np.abs(base.A.astype(np.float64).T @ base.f.b.astype(np.float64))))
    prm = P.pogs_default_params(max_iter=5000)
    warm_iters = cold_iters = 0
    with P.Solver(base.A, prm) as s:
        x0 = nu0 = None
        for frac in (0.5, 0.3, 0.2, 0.1, 0.05):
            g = W.FnParams.make(base.n, W.H["ABS"], c=frac * lam_max)
            prob = W.Problem("lasso", base.A, base.f, g, {})
            info, x, y, mu, nu = s.solve(prob.f, prob.g, x0=x0, nu0=nu0)
            cold, *_ = s.solve(prob.f, prob.g)
            ref = _tight(prob)
            assert info.status == 0 and cold.status == 0
            assert abs(info.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj)), (frac, info.obj, ref.obj)
            warm_iters += info.iters
            cold_iters += cold.iters
            x0, nu0 = x, nu
    assert warm_iters < cold_iters, (warm_iters, cold_iters)


@pytest.mark.parametrize("which", ["x0", "nu0"])
def test_one_part_of_the_warm_start_estimates_the_other(P, which):
    prob = W.lasso(500, 200, seed=45)
    ref = _tight(prob)
    prm = P.pogs_default_params(max_iter=5000)
    kw = dict(x0=ref.x.astype(np.float32)) if which == "x0" else dict(nu0=ref.nu.astype(np.float32))
    with P.Solver(prob.A, prm) as s:
        info, *_ = s.solve(prob.f, prob.g, **kw)
    assert info.status == 0
    assert abs(info.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj))


def test_device_and_host_warm_inputs_agree(P):
    import torch
    prob = W.logistic(400, 300, seed=47)
    prm = P.pogs_default_params(max_iter=5000)
    with P.Solver(prob.A, prm) as s:
        _, x, y, mu, nu = s.solve(prob.f, prob.g)
        a = s.solve(prob.f, prob.g, x0=0.9 * x, nu0=0.9 * nu)
        b = s.solve(prob.f, prob.g, x0=torch.from_numpy(0.9 * x).cuda(), nu0=torch.from_numpy(0.9 * nu).cuda())
    assert a[0].iters == b[0].iters
    for u, v in zip(a[1:], b[1:]):
        assert np.array_equal(u, v)
