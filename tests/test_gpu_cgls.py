"""Indirect projection (CGLS on the reduced update, Section 3.5) on the CUDA path.

  * step fidelity: k CGLS steps from zero on the GPU equal the oracle's k steps (FP64) on
    the GPU's own A^, within 1e-5 relative (FP32 arithmetic over a few steps);
  * convergence: run to a tight tolerance, the projection equals the exact (Cholesky)
    projection within 1e-5;
  * solves: with proj_mode CGLS (no Gram, no factorization) the objective is within 1e-3 of
    the oracle's tight optimum and both residuals meet their tolerances.
"""
import numpy as np
import pytest

import workloads as W
from oracle import admm as OA
from oracle import project as OPJ

pytestmark = pytest.mark.gpu

SHAPES = [(900, 300), (300, 900), (1100, 1030), (257, 600)]


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_08366_b300 as P
    return P


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("steps", [1, 3])
def test_cgls_steps_match_the_oracle_steps(P, shape, steps):
    m, n = shape
    prob = W.nnls(m, n, seed=61)
    prm = P.pogs_default_params(proj_mode="CGLS", cg_max_iter=steps, cg_tol=0.0)
    with P.Solver(prob.A, prm) as s:
        rep = P.pogs_get_setup_report(s.handle)
        Ah = s.ahat().astype(np.float64)
        rng = np.random.default_rng(4)
        c = rng.normal(size=n).astype(np.float32)
        d = rng.normal(size=m).astype(np.float32)
        x, y = s.project(c, d, prm)
    assert rep.factor_ms < 1.0 and rep.gram_ms < 1.0   # no Gram, no factorization
    xr, yr, _, k = OPJ.cgls(Ah, c.astype(np.float64), d.astype(np.float64), iters=steps, tol=0.0)
    assert k == steps
    assert _rel(x, xr) < 1e-5 and _rel(y, yr) < 1e-5, (_rel(x, xr), _rel(y, yr))


@pytest.mark.parametrize("shape", SHAPES)
def test_cgls_converges_to_the_exact_projection(P, shape):
    m, n = shape
    prob = W.lasso(m, n, seed=62)
    prm = P.pogs_default_params(proj_mode="CGLS", cg_max_iter=200, cg_tol=1e-7)
    with P.Solver(prob.A, prm) as s:
        Ah = s.ahat().astype(np.float64)
        rng = np.random.default_rng(5)
        c = rng.normal(size=n).astype(np.float32)
        d = rng.normal(size=m).astype(np.float32)
        x, y = s.project(c, d, prm)
    xr, yr = OPJ.Projector(Ah)(c.astype(np.float64), d.astype(np.float64))
    assert _rel(x, xr) < 1e-5 and _rel(y, yr) < 1e-5, (_rel(x, xr), _rel(y, yr))


@pytest.mark.parametrize("shape", [(1100, 1030), (1030, 1100)])
def test_cgls_past_the_fp32_floor_stops_instead_of_diverging(P, shape):
    """With no tolerance and many steps, FP32 CGLS would pass its rounding floor and grow
    without bound; the divergence test stops it near the best point it reached."""
    m, n = shape
    prob = W.lasso(m, n, seed=62)
    prm = P.pogs_default_params(proj_mode="CGLS", cg_max_iter=400, cg_tol=0.0)
    with P.Solver(prob.A, prm) as s:
        Ah = s.ahat().astype(np.float64)
        rng = np.random.default_rng(6)
        c = rng.normal(size=n).astype(np.float32)
        d = rng.normal(size=m).astype(np.float32)
        x, y = s.project(c, d, prm)
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(y))
    xr, yr = OPJ.Projector(Ah)(c.astype(np.float64), d.astype(np.float64))
    assert _rel(x, xr) < 1e-5 and _rel(y, yr) < 1e-5, (_rel(x, xr), _rel(y, yr))


@pytest.mark.parametrize("cls,shape", [("lasso", (800, 300)), ("logistic", (300, 900)), ("nnls", (600, 250)),
                                       ("huber", (700, 200))])
def test_solve_with_indirect_projection_matches_oracle(P, cls, shape):
    prob = W.CLASSES[cls](*shape, seed=63)
    prm = P.pogs_default_params(proj_mode="CGLS", max_iter=5000)
    with P.Solver(prob.A, prm) as s:
        info, x, y, mu, nu = s.solve(prob.f, prob.g)
    assert info.status == 0, info.as_dict()
    assert info.r_pri < info.eps_pri and info.r_dual < info.eps_dual
    ref = OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=1e-9, rel_tol=1e-7, max_iter=100000))
    assert abs(info.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj)), (info.obj, ref.obj)


def test_direct_handle_can_project_indirectly(P):
    """A handle set up with the factor may still solve with proj_mode CGLS (same optimum)."""
    prob = W.lasso(500, 200, seed=64)
    with P.Solver(prob.A, P.pogs_default_params(max_iter=5000)) as s:
        a, *_ = s.solve(prob.f, prob.g)
        b, *_ = s.solve(prob.f, prob.g, params=P.pogs_default_params(proj_mode="CGLS", max_iter=5000))
    assert a.status == 0 and b.status == 0
    assert abs(a.obj - b.obj) <= 1e-3 * max(1.0, abs(a.obj))
