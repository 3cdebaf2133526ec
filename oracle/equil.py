"""Diagonal pre-conditioning (Section 4), FP64.

Regularized Sinkhorn-Knopp (Algorithm 2, objective Eq. 14) with p = 2, the Frobenius
rescale of Section 4.1.2 / Section 5, and the pre-conditioned functions of Eq. 12.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def default_gamma(m: int, n: int) -> float:
    """gamma = (m + n) sqrt(eps) (Section 5).  Reading: eps is the FP32 machine epsilon
    2^-23, since the paper's runs are single precision (Section 6)."""
    return (m + n) * float(np.sqrt(2.0 ** -23))


def sinkhorn_knopp(A: np.ndarray, sweeps: int, gamma: float):
    """Algorithm 2 with p = 2, run for a fixed number of sweeps.

    e^0 = 1;  d^k = n / (|A|^2 e^{k-1} + gamma/m),  e^k = m / (|A^T|^2 d^k + gamma/n).
    (The paper's stopping rule has an unspecified absolute epsilon; a fixed sweep count
    is used on both sides.)  Returns (d, e) -- the squares of the diagonals of D and E.
    """
    A = np.asarray(A, np.float64)
    m, n = A.shape
    A2 = A * A
    e = np.ones(n)
    d = np.ones(m)
    for _ in range(sweeps):
        d = n / (A2 @ e + gamma / m)
        e = m / (A2.T @ d + gamma / n)
    return d, e


@dataclasses.dataclass
class Equilibration:
    D: np.ndarray      # diagonal of D (length m)
    E: np.ndarray      # diagonal of E (length n)
    Ahat: np.ndarray   # D A E, FP64


def equilibrate(A: np.ndarray, sweeps: int = 10, gamma: float | None = None) -> Equilibration:
    """D = diag(d)^(1/2), E = diag(e)^(1/2) from Algorithm 2, then both rescaled evenly so
    that ||D A E||_F / sqrt(min(m, n)) = 1 (Section 4.1.2, Section 5): with
    s = ||D A E||_F / sqrt(min(m,n)), D <- D / sqrt(s), E <- E / sqrt(s).
    `sweeps = 0` gives D = E = I followed by the rescale."""
    A = np.asarray(A, np.float64)
    m, n = A.shape
    if gamma is None:
        gamma = default_gamma(m, n)
    if sweeps > 0:
        d, e = sinkhorn_knopp(A, sweeps, gamma)
        D, E = np.sqrt(d), np.sqrt(e)
    else:
        D, E = np.ones(m), np.ones(n)
    Ahat = D[:, None] * A * E[None, :]
    s = np.linalg.norm(Ahat) / np.sqrt(min(m, n))
    if s == 0.0:
        s = 1.0      # A = 0: there is no norm to rescale to (the rescale is skipped)
    D = D / np.sqrt(s)
    E = E / np.sqrt(s)
    Ahat = D[:, None] * A * E[None, :]
    return Equilibration(D, E, Ahat)


@dataclasses.dataclass
class Params64:
    h: np.ndarray
    a: np.ndarray
    b: np.ndarray
    c: np.ndarray
    d: np.ndarray
    e: np.ndarray


def fold_f(params, D: np.ndarray) -> Params64:
    """f_hat(y_hat) = f(D^{-1} y_hat) (Eq. 12):
    c h(a y_hat / D - b) + (d / D) y_hat + (e / D^2) y_hat^2 / 2."""
    D = np.asarray(D, np.float64)
    return Params64(np.asarray(params.h, np.int64), np.asarray(params.a, np.float64) / D,
                    np.asarray(params.b, np.float64), np.asarray(params.c, np.float64),
                    np.asarray(params.d, np.float64) / D, np.asarray(params.e, np.float64) / D ** 2)


def fold_g(params, E: np.ndarray) -> Params64:
    """g_hat(x_hat) = g(E x_hat) (Eq. 12): c h(a E x_hat - b) + (d E) x_hat + (e E^2) x_hat^2 / 2."""
    E = np.asarray(E, np.float64)
    return Params64(np.asarray(params.h, np.int64), np.asarray(params.a, np.float64) * E,
                    np.asarray(params.b, np.float64), np.asarray(params.c, np.float64),
                    np.asarray(params.d, np.float64) * E, np.asarray(params.e, np.float64) * E ** 2)
