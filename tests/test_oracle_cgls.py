"""Pins of the oracle's indirect projection (CGLS on the reduced update, Section 3.5)."""
import numpy as np
import pytest

import workloads as W
from oracle import admm as OA
from oracle import project as OPJ


@pytest.mark.parametrize("shape", [(40, 15), (15, 40)])
def test_cgls_converges_to_the_direct_projection(shape):
    rng = np.random.default_rng(1)
    A = rng.standard_normal(shape) / np.sqrt(shape[1])
    c, d = rng.standard_normal(shape[1]), rng.standard_normal(shape[0])
    x, y, _, steps = OPJ.cgls(A, c, d, iters=200, tol=1e-14)
    xr, yr = OPJ.Projector(A)(c, d)
    assert np.allclose(x, xr, atol=1e-10) and np.allclose(y, yr, atol=1e-10)


@pytest.mark.parametrize("shape", [(30, 12), (12, 30)])
def test_cgls_terminates_in_as_many_steps_as_distinct_singular_values(shape):
    """B^T B = M^T M + I has as many distinct eigenvalues as M has distinct singular values
    (here 2): conjugate gradients are exact after that many steps and not before."""
    rng = np.random.default_rng(2)
    m, n = shape
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    k = min(m, n)
    S = np.zeros((m, n))
    S[np.arange(k), np.arange(k)] = np.where(np.arange(k) % 2 == 0, 1.0, 3.0)
    A = U @ S @ V.T
    c, d = rng.standard_normal(n), rng.standard_normal(m)
    xr, yr = OPJ.Projector(A)(c, d)
    x1, y1, _, _ = OPJ.cgls(A, c, d, iters=1)
    x2, y2, _, _ = OPJ.cgls(A, c, d, iters=2)
    assert np.linalg.norm(x1 - xr) > 1e-3
    assert np.allclose(x2, xr, atol=1e-10) and np.allclose(y2, yr, atol=1e-10)


def test_cgls_from_the_solution_takes_no_step():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((25, 10))
    c, d = rng.standard_normal(10), rng.standard_normal(25)
    xr, _ = OPJ.Projector(A)(c, d)
    x, _, _, steps = OPJ.cgls(A, c, d, u0=xr, iters=10, tol=1e-10)
    assert steps == 0 and np.allclose(x, xr)


@pytest.mark.parametrize("cls,shape", [("lasso", (200, 80)), ("logistic", (80, 200))])
def test_admm_with_indirect_projection_reaches_the_same_optimum(cls, shape):
    prob = W.CLASSES[cls](*shape, seed=11)
    direct = OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=1e-8, rel_tol=1e-6, max_iter=20000))
    indirect = OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=1e-8, rel_tol=1e-6, max_iter=20000,
                                                         proj="cgls", cg_iters=100, cg_tol=1e-9))
    assert direct.status == 0 and indirect.status == 0
    assert abs(indirect.obj - direct.obj) <= 1e-5 * max(1.0, abs(direct.obj))
