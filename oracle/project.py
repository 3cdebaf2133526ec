"""Projection onto the graph {(x, y) : y = A x}, FP64.

Two independent statements of the same operator:
  * ``project_kkt``: the KKT system of Eq. 9,  K [x; y] = [c + A^T d; 0],
    K = [[I, A^T], [A, -I]]  (dense solve; tiny problems only);
  * ``Projector``: the reduced updates of Section 3.5 (dense block elimination) with a
    cached FP64 Cholesky factor (factorization caching):
        m >= n:  x = (A^T A + I)^{-1} (c + A^T d),   y = A x
        m <  n:  y = d + (A A^T + I)^{-1} (A c - d), x = c + A^T (d - y).
The paper prints the last update as x = c - A^T (d - y); the first block row of Eq. 9,
x + A^T y = c + A^T d, gives the plus sign, and Eq. 9 is taken as the authority (the
KKT solve pins it in the tests).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl


def project_kkt(A: np.ndarray, c: np.ndarray, d: np.ndarray):
    A = np.asarray(A, np.float64)
    m, n = A.shape
    K = np.block([[np.eye(n), A.T], [A, -np.eye(m)]])
    rhs = np.concatenate([np.asarray(c, np.float64) + A.T @ np.asarray(d, np.float64), np.zeros(m)])
    sol = np.linalg.solve(K, rhs)
    return sol[:n], sol[n:]


class Projector:
    """Factor once (I + A^T A if m >= n, else I + A A^T), then apply per call."""

    def __init__(self, A: np.ndarray):
        self.A = np.asarray(A, np.float64)
        m, n = self.A.shape
        self.tall = m >= n
        G = self.A.T @ self.A if self.tall else self.A @ self.A.T
        G[np.diag_indices_from(G)] += 1.0
        self.L = np.linalg.cholesky(G)   # lower, FP64

    def solve(self, r: np.ndarray) -> np.ndarray:
        """(I + G)^{-1} r with the cached factor: L^{-T} L^{-1} r."""
        z = sl.solve_triangular(self.L, r, lower=True)
        return sl.solve_triangular(self.L.T, z, lower=False)

    def __call__(self, c: np.ndarray, d: np.ndarray):
        A = self.A
        c = np.asarray(c, np.float64)
        d = np.asarray(d, np.float64)
        if self.tall:
            x = self.solve(c + A.T @ d)
            y = A @ x
        else:
            y = d + self.solve(A @ c - d)
            x = c + A.T @ (d - y)
        return x, y


def cgls(A: np.ndarray, c: np.ndarray, d: np.ndarray, u0=None, iters: int = 50, tol: float = 0.0):
    """Indirect projection (Section 3.5): CGLS on the reduced least-squares problem, started
    from a previous iterate u0 (the paper's suggestion for very large problems).

        m >= n:  x = argmin_u ||A u - d||^2 + ||u - c||^2,  y = A x;
        m <  n:  z = argmin_u ||A^T u - c||^2 + ||u + d||^2, y = d + z, x = c - A^T z
    (the normal equations of these are the two reduced updates).  Both are min ||B u - b||
    with B = [M; I]; the iteration is textbook CGLS (Hestenes-Stiefel conjugate gradients on
    the least-squares problem, residual kept as r = b - B u), run until the least-squares
    optimality test ||B^T r|| <= tol ||r|| (LSQR's first stopping rule with ||B|| taken as 1,
    the scale of an equilibrated matrix; ||r|| is the distance of (c, d) from the graph and
    stays away from zero) or `iters` steps.  Returns (x, y, u, steps)."""
    A = np.asarray(A, np.float64)
    c = np.asarray(c, np.float64)
    d = np.asarray(d, np.float64)
    m, n = A.shape
    tall = m >= n
    M, top, bot = (A, d, c) if tall else (A.T, c, -d)   # min ||M u - top||^2 + ||u - bot||^2
    u = np.zeros(M.shape[1]) if u0 is None else np.array(u0, np.float64)
    r_top = top - M @ u
    r_bot = bot - u
    s = M.T @ r_top + r_bot
    p = s.copy()
    gamma = float(s @ s)
    steps = 0
    while steps < iters and gamma > 0.0 and np.sqrt(gamma) > tol * np.sqrt(float(r_top @ r_top + r_bot @ r_bot)):
        q = M @ p
        alpha = gamma / float(q @ q + p @ p)
        u = u + alpha * p
        r_top = r_top - alpha * q
        r_bot = r_bot - alpha * p
        s = M.T @ r_top + r_bot
        gamma_new = float(s @ s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        steps += 1
    if tall:
        x, y = u, A @ u
    else:
        x, y = c - A.T @ u, d + u
    return x, y, u, steps
