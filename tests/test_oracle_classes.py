"""The oracle on the remaining problem classes of Appendix A (basis pursuit, entropy
maximization, portfolio optimization), each pinned to an independent solver of the same
problem: an LP solver, a general constrained minimiser, and exact support enumeration."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import admm as OA

TIGHT = OA.Params(abs_tol=1e-10, rel_tol=1e-8, max_iter=400000)


def test_basis_pursuit_matches_linprog():
    """min ||x||_1 s.t. A x = b as the LP min 1^T t, -t <= x <= t, A x = b (HiGHS)."""
    from scipy.optimize import linprog
    prob = W.basis_pursuit(20, 50, seed=3)
    A, b = prob.A.astype(np.float64), prob.f.b.astype(np.float64)
    m, n = A.shape
    c = np.concatenate([np.zeros(n), np.ones(n)])
    I = np.eye(n)
    res = linprog(c, A_ub=np.block([[I, -I], [-I, -I]]), b_ub=np.zeros(2 * n),
                  A_eq=np.hstack([A, np.zeros((m, n))]), b_eq=b, bounds=[(None, None)] * (2 * n), method="highs")
    r = OA.solve(prob.A, prob.f, prob.g, TIGHT)
    assert r.status == 0
    assert abs(r.obj - res.fun) <= 1e-5 * max(1.0, abs(res.fun)), (r.obj, res.fun)
    assert np.linalg.norm(A @ r.x - b) <= 1e-5 * max(1.0, np.linalg.norm(b))


def test_entropy_maximization_matches_slsqp():
    """min sum x log x s.t. F x <= b, 1^T x = 1 with scipy's SLSQP from the feasible point."""
    from scipy.optimize import minimize
    prob = W.entropy(5, 14, seed=4)
    F, b = prob.A[:-1].astype(np.float64), prob.f.b[:-1].astype(np.float64)
    n = F.shape[1]
    obj = lambda x: float(np.sum(x * np.log(x)))
    grad = lambda x: np.log(x) + 1.0
    cons = [dict(type="ineq", fun=lambda x: b - F @ x, jac=lambda x: -F),
            dict(type="eq", fun=lambda x: np.sum(x) - 1.0, jac=lambda x: np.ones((1, n)))]
    res = minimize(obj, np.full(n, 1.0 / n), jac=grad, constraints=cons, bounds=[(1e-12, 1.0)] * n,
                   method="SLSQP", options=dict(ftol=1e-14, maxiter=2000))
    assert res.success
    r = OA.solve(prob.A, prob.f, prob.g, TIGHT)
    assert r.status == 0
    assert abs(r.obj - res.fun) <= 1e-6 * max(1.0, abs(res.fun)), (r.obj, res.fun)
    assert abs(r.x.sum() - 1.0) < 1e-6 and np.all(F @ r.x <= b + 1e-6)


def _portfolio_by_support_enumeration(F, Dd, mu, gamma):
    """min -mu^T x + gamma x^T (F F^T + D) x s.t. x >= 0, 1^T x = 1: on each support S solve the
    KKT system of the equality-constrained QP and keep the point that is primal feasible and
    satisfies the multiplier signs off the support."""
    n = len(mu)
    Q = 2.0 * gamma * (F @ F.T + np.diag(Dd))
    best = (np.inf, None)
    for r in range(1, n + 1):
        for S in itertools.combinations(range(n), r):
            S = list(S)
            K = np.zeros((r + 1, r + 1))
            K[:r, :r] = Q[np.ix_(S, S)]
            K[:r, r] = 1.0
            K[r, :r] = 1.0
            rhs = np.concatenate([mu[S], [1.0]])
            try:
                sol = np.linalg.solve(K, rhs)
            except np.linalg.LinAlgError:
                continue
            x = np.zeros(n)
            x[S] = sol[:r]
            nu = sol[r]
            if np.any(x[S] < -1e-12):
                continue
            slack = Q @ x - mu + nu
            if np.any(np.delete(slack, S) < -1e-9):
                continue
            val = float(-mu @ x + 0.5 * x @ Q @ x)
            if val < best[0]:
                best = (val, x)
    return best


def test_portfolio_matches_support_enumeration():
    prob = W.portfolio(9, 2, seed=5)
    k = prob.A.shape[0] - 1
    F = prob.A[:k].T.astype(np.float64)            # n x k factor loadings
    mu = -prob.g.d.astype(np.float64)
    Dd = prob.g.e.astype(np.float64) / 2.0          # e = 2 gamma D, gamma = 1
    pstar, xstar = _portfolio_by_support_enumeration(F, Dd, mu, 1.0)
    r = OA.solve(prob.A, prob.f, prob.g, TIGHT)
    assert r.status == 0
    assert abs(r.obj - pstar) <= 1e-6 * max(1.0, abs(pstar)), (r.obj, pstar)
    assert np.linalg.norm(r.x - xstar) <= 1e-4
