"""Pins for oracle.admm (Algorithm 1 + over-relaxation + Algorithm 3, half-tuple output)
against closed forms, exhaustive enumeration and optimality conditions."""
import numpy as np
import pytest

import workloads as W
from oracle import admm as OA
from oracle import equil as OE
from oracle import prox as OP
from tests import _brute as B

TIGHT = OA.Params(abs_tol=1e-10, rel_tol=1e-8, max_iter=50000)


def _fp(k, code, **kw):
    return W.FnParams.make(k, code, **kw)


def test_least_squares_matches_normal_equations():
    """f = 1/2||y - b||^2, g = 0: the solution solves A^T A x = A^T b."""
    rng = np.random.default_rng(10)
    m, n = 40, 12
    A = rng.normal(size=(m, n))
    b = rng.normal(size=m)
    r = OA.solve(A, _fp(m, OP.SQUARE, b=b), _fp(n, OP.ZERO), TIGHT)
    x_ne = np.linalg.solve(A.T @ A, A.T @ b)
    assert r.status == 0
    assert np.allclose(r.x, x_ne, atol=1e-6)


def test_lasso_orthonormal_columns_is_soft_threshold():
    """With A^T A = I, argmin 1/2||Ax - b||^2 + lam||x||_1 = soft(A^T b, lam)."""
    rng = np.random.default_rng(11)
    m, n = 30, 10
    Q, _ = np.linalg.qr(rng.normal(size=(m, n)))
    b = rng.normal(size=m) * 2
    lam = 0.6
    r = OA.solve(Q, _fp(m, OP.SQUARE, b=b), _fp(n, OP.ABS, c=lam), TIGHT)
    z = Q.T @ b
    x_ref = np.sign(z) * np.maximum(np.abs(z) - lam, 0)
    assert np.allclose(r.x, x_ref, atol=1e-6)


def test_lasso_critical_lambda_gives_zero():
    """Appendix A.4: for lambda >= ||A^T b||_inf the Lasso solution is x = 0."""
    P = W.lasso(60, 20, seed=5)
    lam = 1.01 * float(np.max(np.abs(P.A.T.astype(float) @ P.f.b.astype(float))))
    g = _fp(P.n, OP.ABS, c=lam)
    r = OA.solve(P.A, P.f, g, TIGHT)
    assert np.max(np.abs(r.x)) < 1e-6


def test_logistic_critical_lambda_gives_zero():
    """Appendix A.5: for lambda >= ||A^T (1/2 - b)||_inf the l1-logistic solution is x = 0."""
    P = W.logistic(60, 15, seed=6)
    b = -P.f.d.astype(float)
    lam = 1.01 * float(np.max(np.abs(P.A.T.astype(float) @ (0.5 - b))))
    r = OA.solve(P.A, P.f, _fp(P.n, OP.ABS, c=lam), OA.Params(abs_tol=1e-9, rel_tol=1e-7, max_iter=50000))
    assert np.max(np.abs(r.x)) < 1e-5


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_lp_matches_vertex_enumeration(seed):
    """min c^T x s.t. Ax <= b, x >= 0 (Appendix A.6 construction) vs exhaustive vertices."""
    P = W.lp(6, 3, seed=seed, density=1.0)
    A = P.A.astype(float)
    b = P.f.b.astype(float)
    c = P.g.d.astype(float)
    best, _ = B.lp_vertex_enumeration(A, b, c)
    r = OA.solve(P.A, P.f, P.g, OA.Params(abs_tol=1e-9, rel_tol=1e-8, max_iter=200000))
    assert abs(r.obj - best) <= 1e-5 * max(1.0, abs(best))
    assert np.all(r.x >= -1e-7) and np.all(A @ r.x <= b + 1e-5)


@pytest.mark.parametrize("seed", [0, 1])
def test_tiny_nnls_matches_support_enumeration(seed):
    P = W.nnls(12, 6, seed=seed)
    best, xb = B.nnls_support_enumeration(P.A.astype(float), P.f.b.astype(float))
    r = OA.solve(P.A, P.f, P.g, TIGHT)
    assert abs(r.obj - best) <= 1e-7 * max(1.0, best)
    assert np.allclose(r.x, xb, atol=1e-5)


@pytest.mark.parametrize("cls,shape", [("lasso", (50, 20)), ("huber", (50, 20)), ("svm", (40, 15)),
                                        ("nnls", (50, 20)), ("logistic", (50, 20)), ("lasso", (20, 50)),
                                        ("logistic", (15, 40))])
def test_kkt_at_tight_solution(cls, shape):
    """Section 2.2: primal feasibility (Eq. 4), dual feasibility (Eq. 5) and the Fenchel
    conditions (Eq. 8) hold at the tight-tolerance solution (in the original variables)."""
    P = W.CLASSES[cls](*shape, seed=3)
    # fat logistic converges slowly (linear rate): a looser tight run keeps the suite fast
    slow = cls == "logistic" and shape[0] < shape[1]
    tol = 1e-4 if slow else 1e-6
    r = OA.solve(P.A, P.f, P.g, OA.Params(abs_tol=1e-8 if slow else 1e-10, rel_tol=1e-7 if slow else 1e-9,
                                          max_iter=100000))
    A = P.A.astype(float)
    rp, rd = OA.unscaled_residuals(A, r.x, r.y, r.mu, r.nu)
    assert rp < tol * (1 + np.linalg.norm(r.y)) and rd < tol * (1 + np.linalg.norm(r.mu))
    for fp, z, w in ((P.f, r.y, r.nu), (P.g, r.x, r.mu)):
        for i in range(0, len(z), max(1, len(z) // 10)):
            assert B.subgradient_ok(int(fp.h[i]), float(fp.a[i]), float(fp.b[i]), float(fp.c[i]),
                                    float(fp.d[i]), float(fp.e[i]), float(z[i]), float(w[i]),
                                    tol=100 * tol)
    # the half-tuple gap y^T nu + x^T mu vanishes at optimality (Eqs. 6, 7)
    assert abs(r.gap) < 10 * tol * (1 + abs(r.obj))


def test_dual_feasibility_invariant_every_iteration():
    """Section 3.3 (with the tilde terms Algorithm 1 projects): x~^k + A^T y~^k = 0 for all k,
    including under over-relaxation and rho rescaling."""
    P = W.lasso(80, 30, seed=4)
    r = OA.solve(P.A, P.f, P.g, OA.Params(max_iter=300), record=True)
    assert max(h["dual_inv"] for h in r.history) < 1e-10


def test_de_scaling_equals_rho_scaling():
    """Section 4.1: multiplying D by a and dividing E by a scales rho by a^2 and leaves the
    projection unchanged -- the original-space iterates are identical."""
    P = W.huber(60, 25, seed=2)
    A = P.A.astype(float)
    eq = OE.equilibrate(A, 10)
    a = 1.7
    base = OA.Params(max_iter=40, adaptive_rho=False, abs_tol=0, rel_tol=0, gap_stop=False)
    r1 = OA.solve(A, P.f, P.g, OA.Params(**{**base.__dict__, "rho0": 0.8}),
                  eq=OE.Equilibration(a * eq.D, eq.E / a, eq.Ahat))
    r2 = OA.solve(A, P.f, P.g, OA.Params(**{**base.__dict__, "rho0": 0.8 * a * a}), eq=eq)
    for u, v in ((r1.x, r2.x), (r1.y, r2.y), (r1.mu, r2.mu), (r1.nu, r2.nu)):
        assert np.allclose(u, v, rtol=1e-9, atol=1e-11)


def test_equilibration_does_not_change_the_solution():
    P = W.nnls(50, 20, seed=8)
    r1 = OA.solve(P.A, P.f, P.g, TIGHT)
    r2 = OA.solve(P.A, P.f, P.g, OA.Params(**{**TIGHT.__dict__, "equil": False}))
    assert np.allclose(r1.x, r2.x, atol=1e-6)


def test_small_lasso_converges_with_default_tolerances():
    P = W.lasso_small(0)
    r = OA.solve(P.A, P.f, P.g, OA.Params(max_iter=2000))
    assert r.status == 0 and r.iters < 2000
    assert r.r_pri < r.eps_pri and r.r_dual < r.eps_dual
    rt = OA.solve(P.A, P.f, P.g, TIGHT)
    assert abs(r.obj - rt.obj) <= 1e-3 * max(1, abs(rt.obj))


# ---- warm start (Section 5) -----------------------------------------------------------------
@pytest.mark.parametrize("cls,shape", [("lasso", (120, 60)), ("logistic", (80, 150)), ("nnls", (90, 40))])
def test_warm_start_at_the_solution_is_a_fixed_point(cls, shape):
    """Started from the optimal (x*, nu*) of a tight solve, the first iteration reproduces them:
    x* = prox_g(x* + mu*/rho) and y* = prox_f(y* + nu*/rho) are exactly the optimality
    conditions.  A wrong sign or a missing D/E scaling of the warm start breaks this."""
    prob = W.CLASSES[cls](*shape, seed=13)
    tight = OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=1e-10, rel_tol=1e-9, max_iter=50000))
    assert tight.status == 0
    warm = OA.solve(prob.A, prob.f, prob.g, OA.Params(max_iter=1, adaptive_rho=False), x0=tight.x, nu0=tight.nu)
    assert np.linalg.norm(warm.x - tight.x) <= 1e-6 * max(1.0, np.linalg.norm(tight.x))
    assert np.linalg.norm(warm.nu - tight.nu) <= 1e-6 * max(1.0, np.linalg.norm(tight.nu))
    # and a perturbed start converges to the same optimum
    rng = np.random.default_rng(1)
    pert = OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=1e-8, rel_tol=1e-7, max_iter=50000),
                    x0=tight.x + 0.1 * rng.standard_normal(prob.n), nu0=tight.nu + 0.1 * rng.standard_normal(prob.m))
    assert abs(pert.obj - tight.obj) <= 1e-5 * max(1.0, abs(tight.obj))


@pytest.mark.parametrize("which", ["x0", "nu0"])
def test_warm_start_with_one_part_estimates_the_other(which):
    """Only x^0 (or only nu^0) of the optimum: the solve converges to the same optimum, no slower
    than from zero (strictly faster from x^0), and the invariant x~ + A^T y~ = 0 holds from the
    first iteration."""
    prob = W.lasso(150, 70, seed=21)
    prm = OA.Params(abs_tol=1e-7, rel_tol=1e-6, max_iter=50000)
    cold = OA.solve(prob.A, prob.f, prob.g, prm, record=True)
    kw = dict(x0=cold.x) if which == "x0" else dict(nu0=cold.nu)
    warm = OA.solve(prob.A, prob.f, prob.g, prm, record=True, **kw)
    assert warm.status == 0 and warm.iters <= cold.iters
    if which == "x0":
        assert warm.iters < cold.iters
    assert abs(warm.obj - cold.obj) <= 1e-5 * max(1.0, abs(cold.obj))
    assert max(h["dual_inv"] for h in warm.history) < 1e-9
