"""Gram precision x refinement on dense NNLS and inequality-form LP (the precision study).

BF16 and TF32 tensor-core Gram with one refinement step against A per projection (the
configuration of the study) and the default BF16x3 Gram must converge and reach the oracle's
optimum:
  * NNLS: |obj - p*| <= 1e-3 max(1, |p*|), p* from the oracle run to eps_rel = 1e-7;
  * LP: |obj - p_same| <= 1e-3 max(1, |p_same|), p_same from the FP64 oracle stopped by the
    same test (eps_abs = 1e-4, eps_rel = 1e-3), and |obj - p*| <= 1e-2 max(1, |p*|).  At
    eps_rel = 1e-3 the residual test bounds the LP objective only loosely: the FP64 oracle
    itself, stopped by that test, lands about 1e-3 from p* on these instances.
Without refinement the BF16 and TF32 modes project only to their Gram's accuracy and ADMM can
stall at that level (BF16 on NNLS does); for them only the projection bound is asserted.
Projections of the same input on the GPU's own A^ (FP64 oracle projection of the upcast A^):
  * with one refinement step (BF16, TF32) or the BF16x3 Gram: within 1e-5 relative;
  * without refinement: BF16 within 1e-2 and TF32 within 2e-3 (the Gram's own error bound).
At the full 30000 x 15000 size, objectives are checked against the oracle results stored by
tests/golden/make_precision_refs.py, and projections through the normal equations that the
exact projection satisfies, (I + A^T A) x = c + A^T d, evaluated in FP64.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import admm as OA
from oracle import project as OPJ

pytestmark = pytest.mark.gpu

MODES = [("BF16", 0), ("BF16", 1), ("TF32", 0), ("TF32", 1), ("BF16X3", 0)]
CONVERGE = {("BF16", 1), ("TF32", 1), ("BF16X3", 0)}
PROJ_TOL = {("BF16", 0): 1e-2, ("TF32", 0): 2e-3}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


@pytest.fixture(scope="module")
def small():
    probs = {"nnls": W.nnls(3000, 1500, seed=31_000), "lp": W.lp(1200, 600, seed=31_001)}
    refs = {}
    for k, prob in probs.items():
        tol = (1e-9, 1e-7) if k == "nnls" else (1e-7, 1e-5)
        refs[k] = OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=tol[0], rel_tol=tol[1], max_iter=40000))
    refs["lp_same"] = OA.solve(probs["lp"].A, probs["lp"].f, probs["lp"].g, OA.Params(max_iter=20000))
    return probs, refs


@pytest.mark.parametrize("cls", ["nnls", "lp"])
@pytest.mark.parametrize("gram,refine", MODES)
def test_every_precision_reaches_the_oracle_optimum(P, small, cls, gram, refine):
    probs, refs = small
    prob, ref = probs[cls], refs[cls]
    prm = P.pogs_default_params(gram_prec=gram, refine_steps=refine,
                                max_iter=20000 if (gram, refine) in CONVERGE else 500)
    with P.Solver(prob.A, prm) as s:
        info, x, y, mu, nu = s.solve(prob.f, prob.g)
        assert P.pogs_get_setup_report(s.handle).gram_prec_used == P.GRAM[gram]
        Ah = s.ahat().astype(np.float64)
        rng = np.random.default_rng(8)
        c = rng.normal(size=prob.n).astype(np.float32)
        d = rng.normal(size=prob.m).astype(np.float32)
        xp, yp = s.project(c, d, prm)
    if (gram, refine) in CONVERGE:
        assert info.status == 0, info.as_dict()
        assert info.r_pri < info.eps_pri and info.r_dual < info.eps_dual
        bound = 1e-3 if cls == "nnls" else 1e-2
        assert abs(info.obj - ref.obj) <= bound * max(1.0, abs(ref.obj)), (info.obj, ref.obj)
        if cls == "lp":
            same = refs["lp_same"]
            assert same.status == 0
            assert abs(info.obj - same.obj) <= 1e-3 * max(1.0, abs(same.obj)), (info.obj, same.obj)
    else:
        assert info.status in (0, 1) and np.isfinite(info.obj)
    xr, yr = OPJ.Projector(Ah)(c.astype(np.float64), d.astype(np.float64))
    tol = PROJ_TOL.get((gram, refine), 1e-5)
    assert _rel(xp, xr) < tol and _rel(yp, yr) < tol, (gram, refine, _rel(xp, xr), _rel(yp, yr))


def test_refinement_improves_low_precision_projections(P, small):
    probs, _ = small
    prob = probs["nnls"]
    rng = np.random.default_rng(9)
    c = rng.normal(size=prob.n).astype(np.float32)
    d = rng.normal(size=prob.m).astype(np.float32)
    for gram in ("BF16", "TF32"):
        errs = []
        for refine in (0, 1):
            prm = P.pogs_default_params(gram_prec=gram, refine_steps=refine)
            with P.Solver(prob.A, prm) as s:
                xr, _ = OPJ.Projector(s.ahat().astype(np.float64))(c.astype(np.float64), d.astype(np.float64))
                xp, _ = s.project(c, d, prm)
            errs.append(_rel(xp, xr))
        assert errs[1] < 0.1 * errs[0], (gram, errs)


def test_full_size_nnls_against_stored_oracle(P):
    """30000 x 15000 dense NNLS, every mode, against the stored oracle optimum."""
    import torch
    path = os.path.join(GOLDEN, "precision_nnls_30000x15000.json")
    ref = json.load(open(path))
    prob = W.nnls_precision_large()
    assert (prob.m, prob.n, int(prob.meta["seed"])) == (ref["m"], ref["n"], ref["seed"])
    pstar = ref["tight"]["obj"]
    Adev = torch.from_numpy(prob.A).cuda()
    rng = np.random.default_rng(77)
    c = rng.standard_normal(prob.n).astype(np.float32)
    d = rng.standard_normal(prob.m).astype(np.float32)
    for gram, refine in MODES:
        conv = (gram, refine) in CONVERGE
        prm = P.pogs_default_params(gram_prec=gram, refine_steps=refine, max_iter=20000 if conv else 300)
        with P.Solver(Adev, prm) as s:
            info, *_ = s.solve(prob.f, prob.g)
            xp, _ = s.project(c, d, prm)
            Ah = s.ahat().astype(np.float64)
        if conv:
            assert info.status == 0, (gram, refine, info.as_dict())
            assert abs(info.obj - pstar) <= 1e-3 * max(1.0, abs(pstar)), (gram, refine, info.obj, pstar)
        rhs = c.astype(np.float64) + Ah.T @ d.astype(np.float64)
        x64 = xp.astype(np.float64)
        kkt = np.linalg.norm(rhs - (x64 + Ah.T @ (Ah @ x64))) / np.linalg.norm(rhs)
        assert kkt < PROJ_TOL.get((gram, refine), 1e-5), (gram, refine, kkt)
        del Ah


def test_full_size_lp_against_stored_oracle(P):
    """30000 x 15000 inequality-form LP (10% nonzeros stored dense), every converging mode,
    against the stored oracle results: within 1e-3 of the oracle stopped by the same test, and
    within the LP bound 1e-2 of p* (the oracle itself stops 1.1e-3 from p* at eps_rel = 1e-3)."""
    import torch
    path = os.path.join(GOLDEN, "precision_lp_30000x15000.json")
    ref = json.load(open(path))
    prob = W.lp_precision_large()
    assert (prob.m, prob.n, int(prob.meta["seed"])) == (ref["m"], ref["n"], ref["seed"])
    same, pstar = ref["same_tol"]["obj"], ref["tight"]["obj"]
    Adev = torch.from_numpy(prob.A).cuda()
    for gram, refine in sorted(CONVERGE):
        prm = P.pogs_default_params(gram_prec=gram, refine_steps=refine, max_iter=20000)
        with P.Solver(Adev, prm) as s:
            info, *_ = s.solve(prob.f, prob.g)
        assert info.status == 0, (gram, refine, info.as_dict())
        assert abs(info.obj - same) <= 1e-3 * max(1.0, abs(same)), (gram, refine, info.obj, same)
        assert abs(info.obj - pstar) <= 1e-2 * max(1.0, abs(pstar)), (gram, refine, info.obj, pstar)
