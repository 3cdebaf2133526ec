"""Pins for oracle.equil (Algorithm 2, Section 4.1.2 rescale, Eq. 12 folding) and
oracle.project (Eq. 9 and the reduced updates of Section 3.5)."""
import numpy as np
import pytest

import workloads as W
from oracle import equil as OE
from oracle import project as OPJ
from oracle import prox as OP


@pytest.mark.parametrize("shape", [(30, 12), (12, 30), (25, 25)])
def test_sk_optimality_conditions_at_convergence(shape):
    """Section 4.2: at the optimum of Eq. 14 (p = 2),
    |DAE|^2 1 + (gamma/m) d = n 1  and  1^T |DAE|^2 + (gamma/n) e = m 1^T."""
    rng = np.random.default_rng(1)
    m, n = shape
    A = rng.normal(size=shape) * rng.uniform(0.1, 10, size=(m, 1)) * rng.uniform(0.1, 10, size=(1, n))
    gamma = 20.0  # the common-scale mode contracts at a rate set by gamma
    d, e = OE.sinkhorn_knopp(A, 4000, gamma)
    S = d[:, None] * A * A * e[None, :]
    assert np.allclose(S.sum(1) + gamma / m * d, n, rtol=1e-8)
    assert np.allclose(S.sum(0) + gamma / n * e, m, rtol=1e-8)
    # derived consequence: the average entries of d and e agree
    assert abs(d.mean() - e.mean()) <= 1e-8 * d.mean()


def test_sk_large_gamma_limit():
    """Section 4.2: as gamma -> infinity, d and e tend to (mn/gamma) 1."""
    rng = np.random.default_rng(2)
    m, n = 20, 9
    A = rng.normal(size=(m, n))
    gamma = 1e9
    d, e = OE.sinkhorn_knopp(A, 50, gamma)
    assert np.allclose(d, m * n / gamma, rtol=1e-5)
    assert np.allclose(e, m * n / gamma, rtol=1e-5)


def test_sk_non_equilibratable_matrix_stays_finite():
    """gamma > 0 keeps Eq. 14 bounded even when A cannot be equilibrated (zero row/col)."""
    A = np.array([[1.0, 0.0, 2.0], [0.0, 0.0, 0.0], [3.0, 0.0, 1.0], [0.0, 0.0, 0.5]])
    d, e = OE.sinkhorn_knopp(A, 500, OE.default_gamma(4, 3))
    assert np.all(np.isfinite(d)) and np.all(np.isfinite(e)) and np.all(d > 0) and np.all(e > 0)


def test_sk_already_equilibrated_is_uniform():
    """A with all |A_ij| equal is equilibrated: d and e come out constant."""
    m, n = 8, 5
    A = np.where(np.random.default_rng(3).random((m, n)) < 0.5, -2.0, 2.0)
    eq = OE.equilibrate(A, 20)
    assert np.allclose(eq.D, eq.D[0]) and np.allclose(eq.E, eq.E[0])
    assert np.allclose(np.abs(eq.Ahat), np.abs(eq.Ahat[0, 0]))


@pytest.mark.parametrize("shape", [(40, 15), (15, 40)])
def test_rescale_frobenius(shape):
    """Section 4.1.2 / Section 5: ||D A E||_F / sqrt(min(m,n)) = 1, and Ahat = D A E."""
    rng = np.random.default_rng(4)
    A = rng.normal(size=shape) * 7.0
    eq = OE.equilibrate(A, 10)
    assert abs(np.linalg.norm(eq.Ahat) / np.sqrt(min(shape)) - 1.0) < 1e-12
    assert np.allclose(eq.Ahat, eq.D[:, None] * A * eq.E[None, :])


def test_zero_matrix_skips_the_rescale():
    """A = 0 has no Frobenius norm to rescale to: D and E stay the finite Algorithm 2 factors
    (for A = 0 those are d = n m / gamma, e = m n / gamma in closed form) and A^ = 0; the
    projection is then (c, 0) for the tall form, the closed form with G = 0."""
    m, n = 9, 4
    eq = OE.equilibrate(np.zeros((m, n)), 10)
    gamma = OE.default_gamma(m, n)
    assert np.all(np.isfinite(eq.D)) and np.all(np.isfinite(eq.E))
    assert np.allclose(eq.D ** 2, n * m / gamma) and np.allclose(eq.E ** 2, m * n / gamma)
    assert np.all(eq.Ahat == 0)
    c, d = np.arange(n, dtype=float), np.arange(m, dtype=float)
    x, y = OPJ.Projector(eq.Ahat)(c, d)
    assert np.allclose(x, c) and np.allclose(y, 0)


def test_folding_matches_composed_function():
    """Eq. 12: f_hat(yh) = f(yh / D) and g_hat(xh) = g(E xh), evaluated pointwise."""
    rng = np.random.default_rng(5)
    for code in OP.ALL_H:
        if code in OP.INDICATORS:
            continue
        k = 12
        p = W.FnParams(np.full(k, code, np.uint8), rng.uniform(0.5, 2, k), rng.normal(size=k),
                       rng.uniform(0.5, 2, k), rng.normal(size=k), rng.uniform(0, 2, k))
        D = rng.uniform(0.3, 3, k)
        yh = rng.normal(size=k)
        assert np.allclose(OP.f_value(OE.fold_f(p, D), yh), OP.f_value(p, yh / D))
        assert np.allclose(OP.f_value(OE.fold_g(p, D), yh), OP.f_value(p, D * yh))


def test_folded_prox_equals_weighted_prox():
    """Section 4.1: the pre-conditioned prox is the original prox with rho_i^D = rho D_ii^2
    (y side) -- prox_{f_hat}(D v) = D prox_f(v) at parameter rho D^2."""
    rng = np.random.default_rng(6)
    for code in OP.ALL_H:
        k = 15
        p = W.FnParams(np.full(k, code, np.uint8), rng.uniform(0.5, 2, k) * rng.choice([-1, 1], k),
                       rng.normal(size=k), rng.uniform(0.5, 2, k), rng.normal(size=k), rng.uniform(0, 2, k))
        D = rng.uniform(0.3, 3, k)
        v = rng.normal(size=k) * 2
        rho = 0.7
        lhs = OP.prox_f(OE.fold_f(p, D), D * v, rho)
        rhs = D * OP.prox_f(p, v, rho * D ** 2)
        assert np.allclose(lhs, rhs, rtol=1e-9, atol=1e-9), code


@pytest.mark.parametrize("shape", [(9, 5), (5, 9), (7, 7)])
def test_diagonal_sigma_projection_closed_form(shape):
    """Section 4.1.1: for A = Sigma (non-negative diagonal) the projection is explicit:
    x_i = (c_i + s_i d_i)/(1+s_i^2), y_i = s_i (c_i + s_i d_i)/(1+s_i^2) for i < min(m,n);
    x_i = c_i beyond, y_i = 0 beyond."""
    rng = np.random.default_rng(7)
    m, n = shape
    q = min(m, n)
    s = rng.uniform(0.1, 3.0, q)
    S = np.zeros((m, n))
    S[np.arange(q), np.arange(q)] = s
    c, d = rng.normal(size=n), rng.normal(size=m)
    x, y = OPJ.Projector(S)(c, d)
    xe = c.copy()
    ye = np.zeros(m)
    xe[:q] = (c[:q] + s * d[:q]) / (1 + s ** 2)
    ye[:q] = s * (c[:q] + s * d[:q]) / (1 + s ** 2)
    assert np.allclose(x, xe, atol=1e-13) and np.allclose(y, ye, atol=1e-13)
    # sigma = 1 averages (Section 4.1.1)
    S1 = np.zeros((m, n))
    S1[np.arange(q), np.arange(q)] = 1.0
    x1, y1 = OPJ.Projector(S1)(c, d)
    assert np.allclose(x1[:q], 0.5 * (c[:q] + d[:q])) and np.allclose(y1[:q], x1[:q])


@pytest.mark.parametrize("shape", [(12, 5), (5, 12), (6, 6), (1, 4), (4, 1)])
def test_reduced_updates_match_kkt(shape):
    """Section 3.5 reduced updates (tall and fat) equal the KKT solve of Eq. 9."""
    rng = np.random.default_rng(8)
    A = rng.normal(size=shape)
    c, d = rng.normal(size=shape[1]), rng.normal(size=shape[0])
    x1, y1 = OPJ.Projector(A)(c, d)
    x2, y2 = OPJ.project_kkt(A, c, d)
    assert np.allclose(x1, x2, atol=1e-12) and np.allclose(y1, y2, atol=1e-12)


@pytest.mark.parametrize("shape", [(30, 8), (8, 30)])
def test_projection_properties(shape):
    """Projection onto a subspace: lands on the graph, is idempotent, and its residual is
    orthogonal to the graph: (c - x) + A^T (d - y) = 0."""
    rng = np.random.default_rng(9)
    A = rng.normal(size=shape)
    P = OPJ.Projector(A)
    c, d = rng.normal(size=shape[1]), rng.normal(size=shape[0])
    x, y = P(c, d)
    assert np.allclose(y, A @ x, atol=1e-12)
    x2, y2 = P(x, y)
    assert np.allclose(x2, x, atol=1e-12) and np.allclose(y2, y, atol=1e-12)
    assert np.allclose((c - x) + A.T @ (d - y), 0, atol=1e-11)
