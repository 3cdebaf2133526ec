"""Proximal operators of the separable functions (Section 5), FP64.

A separable function is sum_i f_i(y_i) with the parametric form of Section 5

    f_i(y) = c_i h_i(a_i y - b_i) + d_i y + (e_i/2) y^2,   a_i != 0, c_i >= 0, e_i >= 0,

and prox_f(v) = argmin_y f(y) + (rho/2)(y - v)^2 (Section 3.1).

The base functions h are identified by the integer codes of ``workloads.H``; the
oracle keeps its own table of them below (it does not import the C enum).
"""
from __future__ import annotations

import numpy as np
from scipy.special import expit

ZERO, ABS, SQUARE, HUBER, LOGISTIC, HINGE, MAXPOS, IND_GE0, IND_LE0, IND_EQ0, IND_BOX01, XLOGX = range(12)
ALL_H = (ZERO, ABS, SQUARE, HUBER, LOGISTIC, HINGE, MAXPOS, IND_GE0, IND_LE0, IND_EQ0, IND_BOX01, XLOGX)
INDICATORS = (IND_GE0, IND_LE0, IND_EQ0, IND_BOX01)


def h_value(h: int, z: np.ndarray, tol: float = 0.0) -> np.ndarray:
    """Value of base function h at z (elementwise). Indicators return 0 inside the set
    (up to an absolute slack `tol`) and +inf outside."""
    z = np.asarray(z, np.float64)
    inf = np.inf
    if h == ZERO:
        return np.zeros_like(z)
    if h == ABS:
        return np.abs(z)
    if h == SQUARE:
        return 0.5 * z * z
    if h == HUBER:
        return np.where(np.abs(z) <= 1.0, 0.5 * z * z, np.abs(z) - 0.5)
    if h == LOGISTIC:
        return np.logaddexp(0.0, z)
    if h == HINGE:
        return np.maximum(0.0, 1.0 - z)
    if h == MAXPOS:
        return np.maximum(0.0, z)
    if h == IND_GE0:
        return np.where(z >= -tol, 0.0, inf)
    if h == IND_LE0:
        return np.where(z <= tol, 0.0, inf)
    if h == IND_EQ0:
        return np.where(np.abs(z) <= tol, 0.0, inf)
    if h == IND_BOX01:
        return np.where((z >= -tol) & (z <= 1.0 + tol), 0.0, inf)
    if h == XLOGX:
        # z log z (entropy term, Appendix A.2): 0 at z = 0, +inf for z < 0
        with np.errstate(divide="ignore", invalid="ignore"):
            val = np.where(z > 0.0, z * np.log(np.where(z > 0.0, z, 1.0)), 0.0)
        return np.where(z >= -tol, val, inf)
    raise ValueError(f"unknown h code {h}")


def _prox_xlogx(v: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """argmin_{z > 0} z log z + (rho/2)(z-v)^2.

    Optimality: log z + 1 + rho (z - v) = 0.  In t = log z the left side
    psi(t) = t + 1 + rho e^t - rho v is increasing; with hi = max(v, 1), psi(log hi) > 0 and
    psi(rho (v - hi) - 1) = rho (e^{rho(v-hi)-1} - hi) < 0, so the root is bracketed there;
    plain bisection in t to full FP64 resolution, then z = e^t.
    """
    hi_z = np.maximum(v, 1.0)
    hi = np.log(hi_z)
    lo = rho * (v - hi_z) - 1.0
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        psi = mid + 1.0 + rho * np.exp(mid) - rho * v
        neg = psi < 0.0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
        if np.all((hi - lo) <= 1e-15 * (1.0 + np.abs(hi))):
            break
    return np.exp(0.5 * (lo + hi))


def _prox_logistic(v: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """argmin_z log(1+e^z) + (rho/2)(z-v)^2.

    Optimality: sigma(z) + rho (z - v) = 0.  The left side is increasing in z, negative at
    z = v - 1/rho and positive at z = v (sigma lies in (0,1)), so the root is bracketed
    there; plain bisection to full FP64 resolution.
    """
    lo = v - 1.0 / rho
    hi = v.copy()
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        phi = expit(mid) + rho * (mid - v)
        neg = phi < 0.0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
        if np.all((hi - lo) <= 1e-15 * (1.0 + np.abs(hi))):
            break
    return 0.5 * (lo + hi)


def prox_h(h: int, v: np.ndarray, rho) -> np.ndarray:
    """argmin_z h(z) + (rho/2)(z - v)^2 for base function h (textbook forms; the paper
    defers to the proximal-algorithms monograph, Section 3.5 'Proximal operators')."""
    v = np.asarray(v, np.float64)
    rho = np.broadcast_to(np.asarray(rho, np.float64), v.shape)
    if h == ZERO:
        return v.copy()
    if h == ABS:
        return np.sign(v) * np.maximum(np.abs(v) - 1.0 / rho, 0.0)
    if h == SQUARE:
        return rho * v / (1.0 + rho)
    if h == HUBER:
        # quadratic piece while |z| <= 1, i.e. |v| <= 1 + 1/rho; linear piece beyond
        return np.where(np.abs(v) <= 1.0 + 1.0 / rho, rho * v / (1.0 + rho), v - np.sign(v) / rho)
    if h == LOGISTIC:
        return _prox_logistic(v, rho)
    if h == HINGE:
        # max(0, 1 - z): slope -1 left of 1, flat right of 1
        return np.where(v < 1.0 - 1.0 / rho, v + 1.0 / rho, np.where(v > 1.0, v, 1.0))
    if h == MAXPOS:
        # max(0, z): flat left of 0, slope 1 right of 0
        return np.where(v > 1.0 / rho, v - 1.0 / rho, np.where(v < 0.0, v, 0.0))
    if h == IND_GE0:
        return np.maximum(v, 0.0)
    if h == IND_LE0:
        return np.minimum(v, 0.0)
    if h == IND_EQ0:
        return np.zeros_like(v)
    if h == IND_BOX01:
        return np.clip(v, 0.0, 1.0)
    if h == XLOGX:
        return _prox_xlogx(v, rho)
    raise ValueError(f"unknown h code {h}")


def _as64(p):
    return (np.asarray(p.h, np.int64), np.asarray(p.a, np.float64), np.asarray(p.b, np.float64),
            np.asarray(p.c, np.float64), np.asarray(p.d, np.float64), np.asarray(p.e, np.float64))


def prox_f(params, v: np.ndarray, rho) -> np.ndarray:
    """Parametric prox of Section 5:

        prox_f(v) = (1/a) ( prox_{h, (e+rho)/(c a^2)} ( a (v rho - d)/(e + rho) - b ) + b ).

    When c = 0 the h term vanishes and the inner prox is the identity (the paper does not
    state this case; it is the limit of the formula as c -> 0).
    `params` has per-element arrays h, a, b, c, d, e; `rho` is a scalar or per-element.
    """
    h, a, b, c, d, e = _as64(params)
    v = np.asarray(v, np.float64)
    rho = np.broadcast_to(np.asarray(rho, np.float64), v.shape)
    w = a * (v * rho - d) / (e + rho) - b
    out = np.empty_like(v)
    for code in np.unique(h):
        k = h == code
        z = w[k].copy()
        active = c[k] > 0.0
        if np.any(active):
            rho_h = (e[k][active] + rho[k][active]) / (c[k][active] * a[k][active] ** 2)
            z[active] = prox_h(int(code), w[k][active], rho_h)
        out[k] = (z + b[k]) / a[k]
    return out


def f_value(params, y: np.ndarray, tol: float = 0.0) -> np.ndarray:
    """Elementwise f_i(y_i) = c_i h_i(a_i y_i - b_i) + d_i y_i + (e_i/2) y_i^2 (Section 5).
    A zero weight c_i contributes nothing (also for indicators)."""
    h, a, b, c, d, e = _as64(params)
    y = np.asarray(y, np.float64)
    z = a * y - b
    hv = np.empty_like(y)
    for code in np.unique(h):
        k = h == code
        hv[k] = h_value(int(code), z[k], tol * (1.0 + np.abs(b[k])))
    with np.errstate(invalid="ignore"):
        ch = np.where(c > 0.0, c * hv, 0.0)
    return ch + d * y + 0.5 * e * y * y
