"""Seeded synthetic problem generators shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the solver itself: it only draws problem data
(a matrix A and the per-element parameters of the separable functions f and g) the
way the paper's appendix describes its random problem classes (Appendix A), with the
matrix distributions and sizes of the workloads used here.

Every function is encoded in the parametric form of Section 5,

    f_i(y_i) = c_i * h_i(a_i * y_i - b_i) + d_i * y_i + (e_i / 2) * y_i**2,

and likewise g_j(x_j).  ``H`` below lists the integer codes of the base functions h;
they are the values of the ``pogs_h`` enum of the C interface.

Seeds: ``numpy.random.Generator(PCG64(seed))``.  Data is drawn and stored in FP32
(``A`` row-major m x n, parameters as FP32 arrays) -- the oracle upcasts exactly these
FP32 values to FP64, so data rounding is never counted as solver error.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Base-function codes h (values of the C enum ``pogs_h``).
H = dict(
    ZERO=0,        # h(z) = 0
    ABS=1,         # |z|
    SQUARE=2,      # z^2 / 2
    HUBER=3,       # z^2/2 if |z| <= 1 else |z| - 1/2
    LOGISTIC=4,    # log(1 + e^z)
    HINGE=5,       # max(0, 1 - z)
    MAXPOS=6,      # max(0, z)
    IND_GE0=7,     # indicator of z >= 0
    IND_LE0=8,     # indicator of z <= 0
    IND_EQ0=9,     # indicator of z == 0
    IND_BOX01=10,  # indicator of 0 <= z <= 1
    XLOGX=11,      # z log z (0 at z = 0, +inf for z < 0)
)
H_NAMES = {v: k for k, v in H.items()}


@dataclasses.dataclass
class FnParams:
    """Parameters (h, a, b, c, d, e) of a separable function, one entry per element."""
    h: np.ndarray  # uint8
    a: np.ndarray  # float32
    b: np.ndarray
    c: np.ndarray
    d: np.ndarray
    e: np.ndarray

    @staticmethod
    def make(k: int, h: int, a=1.0, b=0.0, c=1.0, d=0.0, e=0.0) -> "FnParams":
        def arr(v):
            out = np.empty(k, np.float32)
            out[...] = v
            return out
        return FnParams(np.full(k, h, np.uint8), arr(a), arr(b), arr(c), arr(d), arr(e))

    def __len__(self):
        return len(self.h)


@dataclasses.dataclass
class Problem:
    """minimize f(y) + g(x) subject to y = A x (Eq. 1)."""
    name: str
    A: np.ndarray          # float32, (m, n), C-contiguous
    f: FnParams            # length m
    g: FnParams            # length n
    meta: dict

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _normal32(rng, shape, mean=0.0, std=1.0) -> np.ndarray:
    A = rng.standard_normal(shape, dtype=np.float32)
    if std != 1.0:
        A *= np.float32(std)
    if mean != 0.0:
        A += np.float32(mean)
    return A


def _sparse_vector(rng, n, frac, std=1.0) -> np.ndarray:
    """frac*n nonzeros (at least 1) drawn N(0, std^2) at uniformly chosen positions."""
    k = max(1, int(round(frac * n)))
    v = np.zeros(n)
    idx = rng.choice(n, size=k, replace=False)
    v[idx] = rng.standard_normal(k) * std
    return v


def lasso(m: int, n: int, seed: int, nnz_frac=0.1, noise_std=0.01, lam_frac=0.1) -> Problem:
    """Lasso (Appendix A.4): f(y) = 1/2 ||y - b||^2, g(x) = lambda ||x||_1.

    A ~ N(0, 1/n); x_true has nnz_frac nonzeros ~ N(0, 1); b = A x_true + N(0, noise_std^2);
    lambda = lam_frac * ||A^T b||_inf.
    """
    rng = _rng(seed)
    A = _normal32(rng, (m, n), std=1.0 / math.sqrt(n))
    x_true = _sparse_vector(rng, n, nnz_frac)
    b = (A.astype(np.float64) @ x_true + rng.standard_normal(m) * noise_std).astype(np.float32)
    lam = float(lam_frac * np.max(np.abs(A.T.astype(np.float64) @ b.astype(np.float64))))
    f = FnParams.make(m, H["SQUARE"], b=b)
    g = FnParams.make(n, H["ABS"], c=lam)
    return Problem("lasso", A, f, g, dict(lam=lam, seed=seed))


def logistic(m: int, n: int, seed: int, nnz_frac=0.05, lam_frac=0.05) -> Problem:
    """l1-regularised logistic regression (Appendix A.5).

    f_i(y) = log(1 + e^y) - b_i y  (LOGISTIC with d = -b_i), g(x) = lambda ||x||_1,
    labels b_i in {0,1} with P(b_i = 1) = sigma(a_i^T x_true),
    lambda = lam_frac * ||A^T (1/2 - b)||_inf.
    """
    rng = _rng(seed)
    A = _normal32(rng, (m, n), std=1.0 / math.sqrt(n))
    x_true = _sparse_vector(rng, n, nnz_frac)
    z = A.astype(np.float64) @ x_true
    p1 = 1.0 / (1.0 + np.exp(-z))
    b = (rng.random(m) < p1).astype(np.float32)
    lam = float(lam_frac * np.max(np.abs(A.T.astype(np.float64) @ (0.5 - b.astype(np.float64)))))
    f = FnParams.make(m, H["LOGISTIC"], d=-b)
    g = FnParams.make(n, H["ABS"], c=lam)
    return Problem("logistic", A, f, g, dict(lam=lam, seed=seed))


def huber(m: int, n: int, seed: int) -> Problem:
    """Huber fitting (Appendix A.3): f_i(y) = huber(y_i - b_i) (M = 1), g = 0.

    b = A v + eps, v ~ N(0, 1/n), eps ~ N(0, 1/4) w.p. 0.95 else U[0, 10].
    """
    rng = _rng(seed)
    A = _normal32(rng, (m, n), std=1.0 / math.sqrt(n))
    v = rng.standard_normal(n) / math.sqrt(n)
    outlier = rng.random(m) >= 0.95
    eps = np.where(outlier, rng.uniform(0.0, 10.0, m), rng.standard_normal(m) * 0.5)
    b = (A.astype(np.float64) @ v + eps).astype(np.float32)
    f = FnParams.make(m, H["HUBER"], b=b)
    g = FnParams.make(n, H["ZERO"])
    return Problem("huber", A, f, g, dict(seed=seed))


def svm(m: int, n: int, seed: int, lam=1.0) -> Problem:
    """Support vector machine (Appendix A.9): f_i(y) = lambda max(0, y_i + 1), g(x) = x^T x,
    with y = diag(b) A x; the stored matrix is diag(b) A.

    Rows i < m/2 have label +1 and entries N(+1/n, 1/n); the rest label -1, N(-1/n, 1/n).
    """
    rng = _rng(seed)
    half = m // 2
    A = np.empty((m, n), np.float32)
    A[:half] = _normal32(rng, (half, n), mean=1.0 / n, std=1.0 / math.sqrt(n))
    A[half:] = _normal32(rng, (m - half, n), mean=-1.0 / n, std=1.0 / math.sqrt(n))
    A[half:] *= -1.0   # diag(b) A with b = -1 on the second class
    f = FnParams.make(m, H["MAXPOS"], a=1.0, b=-1.0, c=lam)
    g = FnParams.make(n, H["SQUARE"], c=2.0)
    return Problem("svm", A, f, g, dict(lam=lam, seed=seed))


def nnls(m: int, n: int, seed: int) -> Problem:
    """Non-negative least squares (Appendix A.7): f = 1/2 ||y - b||^2, g = indicator(x >= 0).

    A ~ N(0, 1/n); v ~ N(1/n, 1/n); b = A v + N(0, 1/4).
    """
    rng = _rng(seed)
    A = _normal32(rng, (m, n), std=1.0 / math.sqrt(n))
    v = 1.0 / n + rng.standard_normal(n) / math.sqrt(n)
    b = (A.astype(np.float64) @ v + rng.standard_normal(m) * 0.5).astype(np.float32)
    f = FnParams.make(m, H["SQUARE"], b=b)
    g = FnParams.make(n, H["IND_GE0"])
    return Problem("nnls", A, f, g, dict(seed=seed))


def lp(m: int, n: int, seed: int, density=0.1) -> Problem:
    """Inequality-form LP (Appendix A.6 with x >= 0): minimize c^T x s.t. A x <= b, x >= 0.

    A has `density` nonzeros ~ N(0,1) (stored dense); v = |N(0, 1/n)|; b = A v + U[0, 0.1];
    c = -A^T u with u ~ U[0,1]^m, which makes the problem feasible (x = v) and bounded.
    f_i = indicator(y_i - b_i <= 0), g_j(x_j) = c_j x_j + indicator(x_j >= 0).
    """
    rng = _rng(seed)
    A = _normal32(rng, (m, n))
    A *= (rng.random((m, n), dtype=np.float32) < density)
    v = np.abs(rng.standard_normal(n) / math.sqrt(n))
    A64 = A.astype(np.float64)
    b = (A64 @ v + rng.uniform(0.0, 0.1, m)).astype(np.float32)
    u = rng.uniform(0.0, 1.0, m)
    c = (-(A64.T @ u)).astype(np.float32)
    f = FnParams.make(m, H["IND_LE0"], b=b)
    g = FnParams.make(n, H["IND_GE0"], d=c)
    return Problem("lp", A, f, g, dict(seed=seed))


def basis_pursuit(m: int, n: int, seed: int) -> Problem:
    """Basis pursuit (Appendix A.1): minimize ||x||_1 s.t. A x = b, in graph form
    f = indicator(y = b), g = |x|.  A ~ N(0, 1/n); v has each entry 0 with probability 1/2,
    else N(0, 1/n); b = A v.  Underdetermined (m < n), as the problem is described."""
    rng = _rng(seed)
    A = _normal32(rng, (m, n), std=1.0 / math.sqrt(n))
    v = np.where(rng.random(n) < 0.5, 0.0, rng.standard_normal(n) / math.sqrt(n))
    b = (A.astype(np.float64) @ v).astype(np.float32)
    f = FnParams.make(m, H["IND_EQ0"], b=b)
    g = FnParams.make(n, H["ABS"])
    return Problem("basis_pursuit", A, f, g, dict(seed=seed))


def entropy(m: int, n: int, seed: int) -> Problem:
    """Entropy maximization (Appendix A.2): minimize sum_j x_j log x_j s.t. F x <= b,
    1^T x = 1.  Graph form with the (m+1) x n matrix [F; 1^T]: f_i = indicator(y_i <= b_i)
    for i < m, f_m = indicator(y_m = 1), g_j = x_j log x_j.  F ~ N(0, 1/n); v ~ U[0, 1]^n;
    b = F v / (1^T v), so x = v / (1^T v) is feasible.  m < n."""
    rng = _rng(seed)
    F = _normal32(rng, (m, n), std=1.0 / math.sqrt(n))
    v = rng.uniform(0.0, 1.0, n)
    b = (F.astype(np.float64) @ v / v.sum()).astype(np.float32)
    A = np.vstack([F, np.ones((1, n), np.float32)])
    f = FnParams.make(m + 1, H["IND_LE0"], b=np.concatenate([b, [1.0]]).astype(np.float32))
    f.h[m] = H["IND_EQ0"]
    g = FnParams.make(n, H["XLOGX"])
    return Problem("entropy", A, f, g, dict(seed=seed))


def portfolio(n: int, k: int, seed: int, gamma: float = 1.0) -> Problem:
    """Portfolio optimization with a k-factor risk model (Appendix A.7): maximize
    mu^T x - gamma x^T (F F^T + D) x s.t. x >= 0, 1^T x = 1.  Graph form with the (k+1) x n
    matrix [F^T; 1^T]: f_i = gamma y_i^2 (SQUARE with c = 2 gamma) for i < k,
    f_k = indicator(y_k = 1), g_j(x) = -mu_j x + gamma D_jj x^2 + indicator(x >= 0).
    F ~ N(0, 1), D_jj ~ U[0, sqrt(k)], mu ~ N(0, 1), gamma = 1; n > k."""
    rng = _rng(seed)
    F = _normal32(rng, (n, k))
    Dd = rng.uniform(0.0, math.sqrt(k), n)
    mu = rng.standard_normal(n)
    A = np.vstack([np.ascontiguousarray(F.T), np.ones((1, n), np.float32)])
    f = FnParams.make(k + 1, H["SQUARE"], c=2.0 * gamma, b=np.concatenate([np.zeros(k), [1.0]]).astype(np.float32))
    f.h[k] = H["IND_EQ0"]
    f.c[k] = 1.0
    g = FnParams.make(n, H["IND_GE0"], d=(-mu).astype(np.float32), e=(2.0 * gamma * Dd).astype(np.float32))
    return Problem("portfolio", A, f, g, dict(seed=seed, gamma=gamma))


def sparse_lasso(m: int, n: int, seed: int, per_row: int = 100, nnz_frac=0.1, noise_std=0.01,
                 lam_frac=0.1) -> Problem:
    """Lasso (Appendix A.4) on a sparse A, returned in CSR form (scipy.sparse, float32, sorted
    unique column indices): each row has `per_row` column positions drawn uniformly (repeats
    dropped), values N(0, 1/per_row) so that rows have the dense generator's expected norm;
    x_true has nnz_frac nonzeros ~ N(0, 1); b = A x_true + N(0, noise_std^2);
    lambda = lam_frac * ||A^T b||_inf.  Built row-block by row-block without a dense copy."""
    import scipy.sparse as sp
    rng = _rng(seed)
    cols = np.sort(rng.integers(0, n, size=(m, per_row), dtype=np.int64), axis=1)
    keep = np.ones_like(cols, dtype=bool)
    keep[:, 1:] = cols[:, 1:] != cols[:, :-1]
    vals = _normal32(rng, (m, per_row), std=1.0 / math.sqrt(per_row))
    counts = keep.sum(axis=1)
    indptr = np.zeros(m + 1, np.int64)
    np.cumsum(counts, out=indptr[1:])
    A = sp.csr_matrix((vals[keep], cols[keep].astype(np.int32), indptr), shape=(m, n), dtype=np.float32)
    x_true = _sparse_vector(rng, n, nnz_frac)
    A64 = A.astype(np.float64)
    b = (A64 @ x_true + rng.standard_normal(m) * noise_std).astype(np.float32)
    lam = float(lam_frac * np.max(np.abs(A64.T @ b.astype(np.float64))))
    f = FnParams.make(m, H["SQUARE"], b=b)
    g = FnParams.make(n, H["ABS"], c=lam)
    return Problem("sparse_lasso", A, f, g, dict(lam=lam, seed=seed, nnz=int(A.nnz)))


def _csr_lasso(name, rows, cols, vals, m, n, rng, nnz_frac, noise_std, lam_frac, meta) -> Problem:
    """Lasso data (the Appendix A.4 recipe) on a sparse A given as COO triples."""
    import scipy.sparse as sp
    A = sp.csr_matrix((np.asarray(vals, np.float32), (rows, cols)), shape=(m, n), dtype=np.float32)
    A.sum_duplicates()
    A.sort_indices()
    x_true = _sparse_vector(rng, n, nnz_frac)
    A64 = A.astype(np.float64)
    b = (A64 @ x_true + rng.standard_normal(m) * noise_std).astype(np.float32)
    lam = float(lam_frac * np.max(np.abs(A64.T @ b.astype(np.float64))))
    return Problem(name, A, FnParams.make(m, H["SQUARE"], b=b), FnParams.make(n, H["ABS"], c=lam),
                   dict(meta, lam=lam, nnz=int(A.nnz)))


def banded_lasso(m: int, n: int, seed: int, half_band: int = 8, nnz_frac=0.1, noise_std=0.01,
                 lam_frac=0.1) -> Problem:
    """Lasso on a banded sparse A (CSR, float32): row i has nonzeros in the 2 * half_band + 1
    columns around c_i = round(i (n - 1) / (m - 1)) (clipped to [0, n)), values
    N(0, 1 / (2 half_band + 1)), so that rows have the dense generator's expected norm."""
    rng = _rng(seed)
    w = 2 * half_band + 1
    centre = np.rint(np.arange(m) * (n - 1) / max(1, m - 1)).astype(np.int64)
    cols = centre[:, None] + np.arange(-half_band, half_band + 1)[None, :]
    keep = (cols >= 0) & (cols < n)
    rows = np.repeat(np.arange(m), w).reshape(m, w)
    vals = _normal32(rng, (m, w), std=1.0 / math.sqrt(w))
    return _csr_lasso("banded_lasso", rows[keep], cols[keep], vals[keep], m, n, rng, nnz_frac, noise_std,
                      lam_frac, dict(seed=seed, half_band=half_band))


def block_angular_lasso(blocks: int, mb: int, nb: int, coupling: int, seed: int, density=0.2,
                        coupling_density=0.05, nnz_frac=0.1, noise_std=0.01, lam_frac=0.1) -> Problem:
    """Lasso on a block-angular sparse A (CSR, float32): `blocks` diagonal blocks of mb x nb with
    `density` nonzeros each, then `coupling` linking rows over all blocks * nb columns with
    `coupling_density` nonzeros; values N(0, 1 / (nonzeros per row))."""
    rng = _rng(seed)
    m, n = blocks * mb + coupling, blocks * nb
    R, Cc, V = [], [], []
    per = max(1, int(round(density * nb)))
    for k in range(blocks):
        for i in range(mb):
            c = np.sort(rng.choice(nb, size=per, replace=False)) + k * nb
            R.append(np.full(per, k * mb + i))
            Cc.append(c)
            V.append(_normal32(rng, (per,), std=1.0 / math.sqrt(per)))
    perc = max(1, int(round(coupling_density * n)))
    for i in range(coupling):
        c = np.sort(rng.choice(n, size=perc, replace=False))
        R.append(np.full(perc, blocks * mb + i))
        Cc.append(c)
        V.append(_normal32(rng, (perc,), std=1.0 / math.sqrt(perc)))
    return _csr_lasso("block_angular_lasso", np.concatenate(R), np.concatenate(Cc), np.concatenate(V), m, n, rng,
                      nnz_frac, noise_std, lam_frac,
                      dict(seed=seed, blocks=blocks, mb=mb, nb=nb, coupling=coupling))


CLASSES = dict(lasso=lasso, logistic=logistic, huber=huber, svm=svm, nnls=nnls, lp=lp,
               basis_pursuit=basis_pursuit, entropy=entropy, portfolio=portfolio)


def nnls_precision_large(seed: int = 30_000) -> Problem:
    """Dense NNLS, 30000 x 15000 (1.8 GB FP32), for the Gram-precision study."""
    return nnls(30000, 15000, seed)


def lp_precision_large(seed: int = 30_001) -> Problem:
    """Inequality-form LP, 30000 x 15000, 10% nonzeros stored dense, for the Gram-precision study."""
    return lp(30000, 15000, seed, density=0.1)


def _log_uniform_int(rng, lo, hi) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def lasso_small(seed: int = 0) -> Problem:
    """Plain single Lasso solve: 200 x 100, A ~ N(0, 1/100), 10% nonzeros, noise N(0, 0.01^2)."""
    return lasso(200, 100, seed, nnz_frac=0.1, noise_std=0.01, lam_frac=0.1)


def lasso_tall_large(seed: int = 10_000) -> Problem:
    """Large dense tall Lasso: 40000 x 10000 (1.6 GB FP32)."""
    return lasso(40000, 10000, seed, nnz_frac=0.1, noise_std=0.01, lam_frac=0.1)


def logistic_fat_large(seed: int = 10_001) -> Problem:
    """Large dense fat l1-logistic regression: 2000 x 40000."""
    return logistic(2000, 40000, seed, nnz_frac=0.05, lam_frac=0.05)


def batch_mix_instance(i: int, base_seed: int = 20_000, m_range=(64, 2048), n_range=(32, 512),
                       classes=("lasso", "huber", "svm", "nnls")) -> Problem:
    """Instance i of `batch_mix`, built on its own from its seed."""
    rng = _rng(base_seed + i)
    cls = classes[int(rng.integers(len(classes)))]
    m = _log_uniform_int(rng, *m_range)
    n = _log_uniform_int(rng, *n_range)
    return CLASSES[cls](m, n, base_seed + 100_000 + i)


def batch_mix(count: int = 2048, base_seed: int = 20_000, m_range=(64, 2048), n_range=(32, 512),
              classes=("lasso", "huber", "svm", "nnls")) -> list:
    """Many small independent instances: class uniform over `classes`, m and n log-uniform."""
    return [batch_mix_instance(i, base_seed, m_range, n_range, classes) for i in range(count)]


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    cls: str
    m: int
    n: int
    seed: int

    def problem(self) -> Problem:
        return CLASSES[self.cls](self.m, self.n, self.seed)


def serve_trace(count: int = 20000, rate_hz: float = 2000.0, base_seed: int = 40_000,
                m_range=(100, 8000), n_range=(50, 4000),
                classes=("lasso", "logistic", "huber", "svm", "nnls")) -> list:
    """Poisson arrival stream of mixed-size requests (exponential inter-arrival gaps)."""
    rng = _rng(base_seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        cls = classes[int(rng.integers(len(classes)))]
        m = _log_uniform_int(rng, *m_range)
        n = _log_uniform_int(rng, *n_range)
        out.append(Request(i, t, cls, m, n, base_seed + 100_000 + i))
    return out
