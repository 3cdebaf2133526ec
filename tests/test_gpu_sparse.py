"""Sparse A through the CSR entry point (Section 3.5's sparse case) against the FP64 oracle.

The oracle is format-agnostic: it runs on the dense array of the same matrix.  Checks:
  * equilibration over the nonzeros: A^ = D A E equals the oracle's within the dense test's
    1e-5 bound, and the dense handle's A^ within FP32 summation-order differences;
  * the projection (direct: factor of the Gram of A^; the passes are CSR kernels) equals the
    oracle's exact projection on the handle's A^;
  * solves, direct and indirect (CGLS), tall and fat, several classes: objective within 1e-3
    of the oracle's tight optimum, both residuals under tolerance;
  * structure: empty rows and columns, a row with every column, malformed input rejected
    with POGS_ERR_ARG / POGS_ERR_NONFINITE; host and device arrays agree; runs repeat bit for
    bit (the transposed copy is built by a stable multi-split).
"""
import numpy as np
import pytest

import workloads as W
from oracle import admm as OA
from oracle import equil as OE
from oracle import project as OPJ

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_08366_b300 as P
    return P


def _csr(A):
    import scipy.sparse as sp
    M = sp.csr_matrix(np.asarray(A, np.float32))
    M.sort_indices()
    return M


def _sparse(cls, shape, seed, frac):
    """The class's generator with its A masked to about `frac` nonzeros (seeded); f and g as
    generated (any f, g pose a valid problem on the masked A)."""
    prob = W.CLASSES[cls](*shape, seed=seed)
    keep = np.random.default_rng(seed + 1).random(prob.A.shape) < frac
    return W.Problem(prob.name, (prob.A * keep).astype(np.float32), prob.f, prob.g, {})


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _tight(prob):
    return OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=1e-9, rel_tol=1e-7, max_iter=100000))


@pytest.mark.parametrize("shape,frac", [((700, 300), 0.05), ((300, 900), 0.02), ((1200, 1100), 0.01)])
def test_sparse_equilibration_matches_oracle_and_dense(P, shape, frac):
    prob = _sparse("lasso", shape, 71, frac)
    A = prob.A.astype(np.float32)
    assert (A != 0).mean() < 2 * frac
    prm = P.pogs_default_params()
    with P.Solver(_csr(A), prm) as s:
        Ahat_s = s.ahat()
    with P.Solver(A, prm) as d:
        Ahat_d = d.ahat()
    ref = OE.equilibrate(A.astype(np.float64)).Ahat
    assert np.array_equal(Ahat_s != 0, A != 0)                 # same pattern, no fill
    assert _rel(Ahat_s, ref) < 1e-5, _rel(Ahat_s, ref)
    assert _rel(Ahat_s, Ahat_d) < 1e-5, _rel(Ahat_s, Ahat_d)


@pytest.mark.parametrize("shape,frac", [((900, 300), 0.05), ((300, 900), 0.05), ((1030, 1100), 0.01)])
def test_sparse_projection_matches_oracle(P, shape, frac):
    m, n = shape
    prob = _sparse("nnls", shape, 72, frac)
    prm = P.pogs_default_params()
    with P.Solver(_csr(prob.A), prm) as s:
        Ah = s.ahat().astype(np.float64)
        rng = np.random.default_rng(8)
        c = rng.normal(size=n).astype(np.float32)
        d = rng.normal(size=m).astype(np.float32)
        x, y = s.project(c, d, prm)
    xr, yr = OPJ.Projector(Ah)(c.astype(np.float64), d.astype(np.float64))
    assert _rel(x, xr) < 1e-5 and _rel(y, yr) < 1e-5, (_rel(x, xr), _rel(y, yr))


@pytest.mark.parametrize("mode", ["DIRECT", "CGLS"])
@pytest.mark.parametrize("cls,shape,frac", [("lasso", (800, 300), 0.1), ("logistic", (300, 900), 0.1),
                                            ("nnls", (600, 250), 0.05), ("huber", (700, 200), 0.2)])
def test_sparse_solve_matches_oracle(P, mode, cls, shape, frac):
    prob = _sparse(cls, shape, 73, frac)
    prm = P.pogs_default_params(max_iter=5000, proj_mode=mode)
    with P.Solver(_csr(prob.A), prm) as s:
        info, x, y, mu, nu = s.solve(prob.f, prob.g)
    assert info.status == 0, info.as_dict()
    assert info.r_pri < info.eps_pri and info.r_dual < info.eps_dual
    ref = _tight(prob)
    assert abs(info.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj)), (info.obj, ref.obj)
    Ad = prob.A.astype(np.float64)
    assert np.linalg.norm(Ad @ x - y) <= 1e-2 * max(1.0, np.linalg.norm(y))


@pytest.mark.parametrize("mode", ["DIRECT", "CGLS"])
@pytest.mark.parametrize("shape,per_row", [((3000, 800), 20), ((600, 2500), 40)])
def test_sparse_lasso_generator_solve(P, mode, shape, per_row):
    """The CSR workload generator (row-wise random pattern) end to end, tall and fat."""
    prob = W.sparse_lasso(*shape, seed=77, per_row=per_row)
    prm = P.pogs_default_params(max_iter=5000, proj_mode=mode)
    with P.Solver(prob.A, prm) as s:
        info, x, y, mu, nu = s.solve(prob.f, prob.g)
    assert info.status == 0, info.as_dict()
    dense = W.Problem(prob.name, prob.A.toarray(), prob.f, prob.g, {})
    ref = _tight(dense)
    assert abs(info.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj)), (info.obj, ref.obj)


def test_empty_rows_columns_and_a_full_row(P):
    rng = np.random.default_rng(74)
    m, n = 400, 150
    A = (rng.normal(size=(m, n)) * (rng.random((m, n)) < 0.05)).astype(np.float32)
    A[[3, 77, 399], :] = 0.0          # empty rows (the last one too)
    A[:, [0, 50, 149]] = 0.0          # empty columns (the first and the last)
    A[10, :] = rng.normal(size=n)     # one row with every column
    A[10, [0, 50, 149]] = 0.0
    b = rng.normal(size=m).astype(np.float32)
    f = W.FnParams.make(m, W.H["SQUARE"], b=b)
    g = W.FnParams.make(n, W.H["ABS"], c=0.1)
    prob = W.Problem("lasso", A, f, g, {})
    prm = P.pogs_default_params(max_iter=5000)
    with P.Solver(_csr(A), prm) as s:
        Ahat = s.ahat()
        info, x, *_ = s.solve(f, g)
    ref_hat = OE.equilibrate(A.astype(np.float64)).Ahat
    assert _rel(Ahat, ref_hat) < 1e-5
    assert info.status == 0
    ref = _tight(prob)
    assert abs(info.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj)), (info.obj, ref.obj)


def test_malformed_csr_is_rejected(P):
    import ctypes
    h = ctypes.c_void_p()

    def setup(rp, ci, va, m=3, n=4):
        rp = np.asarray(rp, np.int32)
        ci = np.asarray(ci, np.int32)
        va = np.asarray(va, np.float32)
        return P.lib.pogs_setup_csr(m, n, len(ci), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, None, None,
                                    ctypes.byref(h))

    assert setup([0, 1, 2, 3], [0, 1, 2], [1, 2, 3]) == 0
    P.lib.pogs_free(h)
    assert setup([0, 2, 2, 3], [1, 0, 2], [1, 2, 3]) == -1       # columns not increasing in a row
    assert setup([0, 2, 2, 3], [1, 1, 2], [1, 2, 3]) == -1       # duplicate entry
    assert setup([0, 1, 2, 3], [0, 4, 2], [1, 2, 3]) == -1       # column index out of range
    assert setup([0, 1, 2, 3], [0, -1, 2], [1, 2, 3]) == -1      # negative column index
    assert setup([0, 2, 1, 3], [0, 1, 2], [1, 2, 3]) == -1       # decreasing row pointers
    assert setup([1, 1, 2, 3], [0, 1, 2], [1, 2, 3]) == -1       # rowptr[0] != 0
    assert setup([0, 1, 2, 2], [0, 1, 2], [1, 2, 3]) == -1       # rowptr[m] != nnz
    assert setup([0, 1, 2, 9], [0, 1, 2], [1, 2, 3]) == -1       # row pointer beyond nnz
    assert setup([0, 1, 2, 3], [0, 1, 2], [1, np.nan, 3]) == -3  # non-finite value


def test_host_and_device_arrays_agree_and_runs_repeat(P):
    import torch
    prob = _sparse("logistic", (500, 400), 75, 0.05)
    M = _csr(prob.A)
    prm = P.pogs_default_params(max_iter=5000)
    outs = []
    for dev in (False, True, True):
        arrs = (M.indptr, M.indices, M.data)
        if dev:
            arrs = tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs)
        h = P.pogs_setup_csr(*arrs, M.shape, prm)
        x = np.empty(prob.n, np.float32)
        y = np.empty(prob.m, np.float32)
        info = P.pogs_solve(h, prob.f, prob.g, prm, x, y)
        P.pogs_free(h)
        outs.append((info.iters, x, y))
    for it, x, y in outs[1:]:
        assert it == outs[0][0]
        assert np.array_equal(x, outs[0][1]) and np.array_equal(y, outs[0][2])


def test_empty_matrix_of_nonzeros(P):
    """nnz = 0: A = 0, the projection is (c, 0) for the tall case; a Lasso solve returns x = 0
    and the half-step y (the prox output, within the primal residual of A x = 0) near 0."""
    m, n = 50, 20
    rp = np.zeros(m + 1, np.int32)
    ci = np.zeros(0, np.int32)
    va = np.zeros(0, np.float32)
    prm = P.pogs_default_params(max_iter=5000)
    h = P.pogs_setup_csr(rp, ci, va, (m, n), prm)
    b = np.random.default_rng(76).normal(size=m).astype(np.float32)
    f = W.FnParams.make(m, W.H["SQUARE"], b=b)
    g = W.FnParams.make(n, W.H["ABS"], c=0.1)
    x = np.empty(n, np.float32)
    y = np.empty(m, np.float32)
    info = P.pogs_solve(h, f, g, prm, x, y)
    P.pogs_free(h)
    assert info.status == 0
    assert np.all(x == 0) and np.max(np.abs(y)) <= info.eps_pri
