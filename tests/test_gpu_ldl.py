"""The sparse direct projection (Section 3.5): LDL^T of the quasi-definite K = [I A^T; A -I],
ordered for sparsity on the host, factored once on the GPU and cached in the handle
(proj_mode LDL, CSR input), against the FP64 oracle on the dense array of the same matrix.

Checks (tolerances as the dense path's):
  * one projection of random (c, d) equals the oracle's exact projection on the handle's own A^
    within 1e-5 relative in x and in y -- banded (tall and fat), block-angular (whose coupling
    rows make frontal matrices of more than 96 rows, assembled in global memory) and uniformly
    scattered patterns, with and without one refinement step;
  * solves: objective within 1e-3 of the oracle's tight optimum with both residuals under
    tolerance; the same iterates' objective as the dense factor of the reduced update;
  * the cached factor serves warm-started re-solves with new weights;
  * dense input with proj_mode LDL is rejected (POGS_ERR_ARG); runs repeat bit for bit.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import admm as OA
from oracle import project as OPJ

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_08366_b300 as P
    return P


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _scattered(m, n, seed, per_row):
    return W.sparse_lasso(m, n, seed=seed, per_row=per_row)


CASES = {
    "banded_tall": lambda: W.banded_lasso(3000, 1200, seed=81, half_band=6),
    "banded_fat": lambda: W.banded_lasso(900, 2500, seed=82, half_band=5),
    "block_angular": lambda: W.block_angular_lasso(6, 150, 80, 120, seed=83, density=0.08, coupling_density=0.05),
    "scattered": lambda: _scattered(700, 400, 84, per_row=4),
}


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_ldl_projection_matches_oracle(P, name, refine):
    prob = CASES[name]()
    A = prob.A
    m, n = A.shape
    prm = P.pogs_default_params(proj_mode="LDL", refine_steps=refine)
    with P.Solver(A, prm) as s:
        Ah = s.ahat().astype(np.float64)
        proj = OPJ.Projector(Ah)
        rng = np.random.default_rng(7)
        for _ in range(2):
            c = rng.normal(size=n).astype(np.float32)
            d = rng.normal(size=m).astype(np.float32)
            x, y = s.project(c, d, prm)
            xr, yr = proj(c.astype(np.float64), d.astype(np.float64))
            assert _rel(x, xr) < 1e-5 and _rel(y, yr) < 1e-5, (name, _rel(x, xr), _rel(y, yr))


def test_block_angular_case_has_global_fronts(P):
    A = CASES["block_angular"]().A
    stats, _, _ = P.pogs_ldl_analyze(A.indptr, A.indices, A.shape)
    assert stats["max_front"] > 96, stats


@pytest.mark.parametrize("name", ["banded_tall", "banded_fat", "block_angular"])
def test_ldl_solve_matches_oracle_and_dense_factor(P, name):
    prob = CASES[name]()
    A = prob.A
    ref = OA.solve(A.toarray(), prob.f, prob.g, OA.Params(abs_tol=1e-9, rel_tol=1e-7, max_iter=100000))
    out = {}
    for mode in ("LDL", "DIRECT"):
        prm = P.pogs_default_params(proj_mode=mode, max_iter=5000)
        with P.Solver(A, prm) as s:
            info, x, y, mu, nu = s.solve(prob.f, prob.g)
        assert info.status == 0, (mode, info.as_dict())
        assert info.r_pri < info.eps_pri and info.r_dual < info.eps_dual
        assert abs(info.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj)), (mode, info.obj, ref.obj)
        out[mode] = info
    assert abs(out["LDL"].obj - out["DIRECT"].obj) <= 1e-4 * max(1.0, abs(ref.obj))


def test_ldl_factor_is_cached_for_warm_restarts(P):
    prob = CASES["banded_tall"]()
    A = prob.A
    lam_max = float(np.max(np.abs(A.T.astype(np.float64) @ prob.f.b.astype(np.float64))))
    prm = P.pogs_default_params(proj_mode="LDL", max_iter=5000)
    with P.Solver(A, prm) as s:
        x0 = nu0 = None
        for frac in (0.3, 0.1, 0.05):
            g = W.FnParams.make(A.shape[1], W.H["ABS"], c=frac * lam_max)
            info, x, y, mu, nu = s.solve(prob.f, g, x0=x0, nu0=nu0)
            ref = OA.solve(A.toarray(), prob.f, g, OA.Params(abs_tol=1e-9, rel_tol=1e-7, max_iter=100000))
            assert info.status == 0
            assert abs(info.obj - ref.obj) <= 1e-3 * max(1.0, abs(ref.obj))
            x0, nu0 = x, nu


def test_ldl_runs_repeat_bit_for_bit(P):
    prob = CASES["block_angular"]()
    outs = []
    for _ in range(2):
        with P.Solver(prob.A, P.pogs_default_params(proj_mode="LDL")) as s:
            outs.append(s.solve(prob.f, prob.g))
    (i0, *v0), (i1, *v1) = outs
    assert i0.iters == i1.iters and i0.obj == i1.obj
    for a, b in zip(v0, v1):
        assert np.array_equal(a, b)


def test_ldl_degenerate_patterns(P):
    """Empty rows and columns, a single row, a single column."""
    rng = np.random.default_rng(9)
    for shape, dens in (((40, 30), 0.05), ((1, 20), 0.5), ((25, 1), 0.5)):
        A = sp.random(*shape, density=dens, random_state=rng, format="csr", dtype=np.float32)
        A.sort_indices()
        b = rng.normal(size=shape[0]).astype(np.float32)
        f = W.FnParams.make(shape[0], W.H["SQUARE"], b=b)
        g = W.FnParams.make(shape[1], W.H["ABS"], c=0.1)
        prm = P.pogs_default_params(proj_mode="LDL", max_iter=5000)
        with P.Solver(A, prm) as s:
            Ah = s.ahat().astype(np.float64)
            c = rng.normal(size=shape[1]).astype(np.float32)
            d = rng.normal(size=shape[0]).astype(np.float32)
            x, y = s.project(c, d, prm)
            info, *_ = s.solve(f, g)
        xr, yr = OPJ.Projector(Ah)(c.astype(np.float64), d.astype(np.float64))
        assert _rel(x, xr) < 1e-5 and _rel(y, yr) < 1e-5
        assert info.status in (0, 1)


def test_ldl_needs_sparse_input(P):
    prob = W.lasso(60, 30, seed=1)
    with pytest.raises(P.PogsError) as ei:
        P.Solver(prob.A, P.pogs_default_params(proj_mode="LDL"))
    assert ei.value.code == -1
