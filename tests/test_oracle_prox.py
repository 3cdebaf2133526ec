"""Pins for oracle.prox: every base function, through the parametric formula of
Section 5, against brute-force 1-D minimisation and subgradient membership."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import prox as OP
from tests import _brute as B


def _params(rng, code, k):
    a = rng.uniform(0.3, 2.5, k) * rng.choice([-1.0, 1.0], k)
    b = rng.normal(0, 1.5, k)
    c = rng.uniform(0.2, 3.0, k)
    c[::5] = 0.0                           # zero weight: h drops out
    d = rng.normal(0, 1.0, k)
    e = rng.uniform(0.0, 2.0, k)
    e[::3] = 0.0
    return W.FnParams(np.full(k, code, np.uint8), a, b, c, d, e)


def test_codes_match_workload_table():
    for name, code in W.H.items():
        assert getattr(OP, name) == code


@pytest.mark.parametrize("code", OP.ALL_H, ids=[W.H_NAMES[c] for c in OP.ALL_H])
def test_parametric_prox_vs_bruteforce(code):
    rng = np.random.default_rng(100 + code)
    k = 160
    p = _params(rng, code, k)
    v = rng.normal(0, 3.0, k)
    rho = np.exp(rng.uniform(np.log(0.02), np.log(50.0), k))   # log-uniform: every regime
    got = OP.prox_f(p, v, rho)
    for i in range(k):
        ref = B.prox_bruteforce(code, p.a[i], p.b[i], p.c[i], p.d[i], p.e[i], rho[i], v[i])
        assert abs(got[i] - ref) <= 1e-6 * (1 + abs(ref)), (i, got[i], ref)


@pytest.mark.parametrize("code", OP.ALL_H, ids=[W.H_NAMES[c] for c in OP.ALL_H])
def test_prox_output_is_fenchel_feasible(code):
    """Section 3.3: y = prox_f(v) implies nu = rho (v - y) lies in the subdifferential of f at y."""
    rng = np.random.default_rng(200 + code)
    k = 25
    p = _params(rng, code, k)
    v = rng.normal(0, 3.0, k)
    rho = rng.uniform(0.1, 10.0, k)
    y = OP.prox_f(p, v, rho)
    nu = rho * (v - y)
    for i in range(k):
        assert B.subgradient_ok(code, p.a[i], p.b[i], p.c[i], p.d[i], p.e[i], y[i], nu[i]), i


def test_textbook_values():
    """Hand-computed values of the base proxes at rho = 1 (soft threshold, clip, ...)."""
    v = np.array([3.0, 0.5, -2.0])
    assert np.allclose(OP.prox_h(OP.ABS, v, 1.0), [2.0, 0.0, -1.0])
    assert np.allclose(OP.prox_h(OP.SQUARE, v, 1.0), [1.5, 0.25, -1.0])
    assert np.allclose(OP.prox_h(OP.HUBER, v, 1.0), [2.0, 0.25, -1.0])
    assert np.allclose(OP.prox_h(OP.MAXPOS, v, 1.0), [2.0, 0.0, -2.0])
    assert np.allclose(OP.prox_h(OP.HINGE, v, 1.0), [3.0, 1.0, -1.0])
    assert np.allclose(OP.prox_h(OP.IND_BOX01, v, 1.0), [1.0, 0.5, 0.0])
    # logistic at v = 0, rho = 1: z = -sigma(z) has the root z ~ -0.401058 (fixed point)
    z = OP.prox_h(OP.LOGISTIC, np.array([0.0]), 1.0)[0]
    assert abs(z + 1.0 / (1.0 + math.exp(-z))) < 1e-12
    assert abs(z - (-0.4010577)) < 1e-6


def test_xlogx_prox_is_lambert_w():
    """log z + 1 + rho (z - v) = 0 has the closed form rho z = W(rho e^{rho v - 1}) with the
    principal branch of Lambert's W (scipy), a pin independent of the oracle's bisection."""
    from scipy.special import lambertw
    v = np.linspace(-6.0, 8.0, 57)
    for rho in (0.05, 0.7, 3.0, 40.0):
        ref = np.real(lambertw(rho * np.exp(rho * v - 1.0))) / rho
        got = OP.prox_h(OP.XLOGX, v, rho)
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-300), rho


def test_value_matches_bruteforce_table():
    rng = np.random.default_rng(7)
    for code in OP.ALL_H:
        if code in OP.INDICATORS:
            continue
        z = rng.normal(0, 3, 30)
        got = OP.h_value(code, z)
        ref = [B.base_value(code, float(t)) for t in z]
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
