"""Brute-force reference computations used to pin the oracle (no shared code with it).

Each helper computes a quantity from its definition by exhaustive or derivative-free
search, so that a mistake in a closed form (a dropped term, a wrong sign, a swapped
operand) shows up as a mismatch.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# Base functions written out independently of oracle.prox (value only).
def base_value(code: int, z: float) -> float:
    if code == 0:
        return 0.0
    if code == 1:
        return abs(z)
    if code == 2:
        return 0.5 * z * z
    if code == 3:
        return 0.5 * z * z if abs(z) <= 1 else abs(z) - 0.5
    if code == 4:
        return math.log1p(math.exp(z)) if z < 30 else z + math.log1p(math.exp(-z))
    if code == 5:
        return max(0.0, 1.0 - z)
    if code == 6:
        return max(0.0, z)
    if code == 7:
        return 0.0 if z >= 0 else math.inf
    if code == 8:
        return 0.0 if z <= 0 else math.inf
    if code == 9:
        return 0.0 if z == 0 else math.inf
    if code == 10:
        return 0.0 if 0 <= z <= 1 else math.inf
    if code == 11:
        if z < 0:
            return math.inf
        return 0.0 if z == 0 else z * math.log(z)
    raise ValueError(code)


# Feasible set of z for the indicator codes, as an interval [lo, hi].
IND_SET = {7: (0.0, math.inf), 8: (-math.inf, 0.0), 9: (0.0, 0.0), 10: (0.0, 1.0)}


def _golden(phi, lo, hi, iters=300):
    """Golden-section minimisation of a convex function on [lo, hi]."""
    gr = (math.sqrt(5) - 1) / 2
    a, b = lo, hi
    c = b - gr * (b - a)
    d = a + gr * (b - a)
    fc, fd = phi(c), phi(d)
    for _ in range(iters):
        if fc <= fd:
            b, d, fd = d, c, fc
            c = b - gr * (b - a)
            fc = phi(c)
        else:
            a, c, fc = c, d, fd
            d = a + gr * (b - a)
            fd = phi(d)
        if b - a < 1e-15 * (1 + abs(a)):
            break
    return 0.5 * (a + b)


def prox_bruteforce(code, a, b, c, d, e, rho, v):
    """argmin_y c h(a y - b) + d y + (e/2) y^2 + (rho/2)(y - v)^2 by golden section.

    For indicators the search runs over the interval {y : a y - b in S}."""
    def smooth(y):
        return d * y + 0.5 * e * y * y + 0.5 * rho * (y - v) ** 2
    if code in IND_SET and c > 0:
        zlo, zhi = IND_SET[code]
        ylo, yhi = sorted(((zlo + b) / a, (zhi + b) / a))
        if ylo == yhi:
            return ylo
        # bound the infinite side by a window around the unconstrained minimiser
        ystar = (rho * v - d) / (e + rho)
        span = 10 * (1 + abs(ystar) + abs(v))
        lo = ylo if math.isfinite(ylo) else min(yhi, ystar) - span
        hi = yhi if math.isfinite(yhi) else max(ylo, ystar) + span
        return _golden(smooth, lo, hi)

    def phi(y):
        return (c * base_value(code, a * y - b) if c > 0 else 0.0) + smooth(y)
    # the minimiser lies within a window around v scaled by the slopes involved
    span = 10 * (1 + abs(v) + abs(d) / rho + c * abs(a) / rho + abs(b / a))
    lo, hi = v - span, v + span
    if code == 11 and c > 0:
        # domain a y - b >= 0, and log z grows only slowly: widen the window on that side
        edge = b / a
        span = 10 * (1 + abs(v) + abs(d) / rho + c * abs(a) / rho * (1 + abs(math.log(1 + abs(v) + abs(edge))))
                     + abs(edge))
        lo, hi = (edge, max(edge, v) + span) if a > 0 else (min(edge, v) - span, edge)
    return _golden(phi, lo, hi)


def f_scalar(code, a, b, c, d, e, y, tol=0.0):
    z = a * y - b
    if code in IND_SET:
        lo, hi = IND_SET[code]
        inside = (z >= lo - tol) and (z <= hi + tol)
        hv = 0.0 if inside else math.inf
    else:
        hv = base_value(code, z)
    return (c * hv if c > 0 else 0.0) + d * y + 0.5 * e * y * y


def subgradient_ok(code, a, b, c, d, e, y, nu, tol=1e-7, grid=None) -> bool:
    """Check nu in the subdifferential of f at y: f(z) >= f(y) + nu (z - y) for z on a grid."""
    fy = f_scalar(code, a, b, c, d, e, y, tol=1e-9)
    if not math.isfinite(fy):
        return False
    if grid is None:
        grid = y + np.concatenate([-np.logspace(-6, 2, 40), np.logspace(-6, 2, 40)])
    for z in grid:
        fz = f_scalar(code, a, b, c, d, e, float(z))
        if not math.isfinite(fz):
            continue
        if fz < fy + nu * (z - y) - tol * (1 + abs(fy) + abs(nu * (z - y))):
            return False
    return True


def lp_vertex_enumeration(A, b, c):
    """min c^T x s.t. A x <= b, x >= 0 by enumerating every vertex (tiny problems)."""
    A = np.asarray(A, float)
    m, n = A.shape
    G = np.vstack([A, -np.eye(n)])
    h = np.concatenate([b, np.zeros(n)])
    best, arg = math.inf, None
    for rows in itertools.combinations(range(m + n), n):
        Gs = G[list(rows)]
        if abs(np.linalg.det(Gs)) < 1e-12:
            continue
        x = np.linalg.solve(Gs, h[list(rows)])
        if np.all(G @ x <= h + 1e-9):
            val = float(c @ x)
            if val < best:
                best, arg = val, x
    return best, arg


def nnls_support_enumeration(A, b):
    """min 1/2 ||A x - b||^2 s.t. x >= 0 by trying every support (tiny n)."""
    A = np.asarray(A, float)
    m, n = A.shape
    best, arg = 0.5 * float(b @ b), np.zeros(n)
    for k in range(1, n + 1):
        for S in itertools.combinations(range(n), k):
            S = list(S)
            xs, *_ = np.linalg.lstsq(A[:, S], b, rcond=None)
            if np.all(xs >= -1e-12):
                x = np.zeros(n)
                x[S] = np.maximum(xs, 0)
                val = 0.5 * float(np.sum((A @ x - b) ** 2))
                if val < best:
                    best, arg = val, x
    return best, arg
