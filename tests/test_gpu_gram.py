"""Gram formation on the tensor cores (tcgen05) and in FP32 SIMT vs the FP64 Gram of the
same FP32 matrix, lower triangle.  Shapes span one and several 128-tiles, ragged edges and
K not a multiple of the TMA box, tall (A^T A) and fat (A A^T).

Tolerance on ||G - G_ref||_F / ||G_ref||_F, from each mode's input rounding (unit roundoff u
of the operand format; products of rounded inputs have relative error ~2u, FP32 accumulation
adds ~sqrt(K) 2^-24):
  BF16 (u = 2^-9):  1e-2      TF32 (u = 2^-11): 2e-3
  BF16x3 (hi + lo, error ~2^-17 per product): 2e-5      FP32: 1e-5
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"BF16": 1e-2, "TF32": 2e-3, "BF16X3": 2e-5, "FP32": 1e-5}
SHAPES = [(300, 200), (200, 300), (1000, 600), (130, 2500), (4096, 256), (257, 129), (64, 33)]


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_08366_b300 as P
    return P


@pytest.mark.parametrize("prec", ["BF16X3", "BF16", "TF32", "FP32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_gram_matches_fp64(P, prec, shape):
    import torch
    m, n = shape
    rng = np.random.default_rng(m * 7 + n)
    A = (rng.standard_normal((m, n)) / np.sqrt(n)).astype(np.float32)
    G = P.pogs_gram(torch.from_numpy(A).cuda(), prec).cpu().numpy().astype(np.float64)
    A64 = A.astype(np.float64)
    ref = A64.T @ A64 if m >= n else A64 @ A64.T
    lo = np.tril_indices(ref.shape[0])
    err = np.linalg.norm(G[lo] - ref[lo]) / np.linalg.norm(ref[lo])
    assert err <= TOL[prec], (prec, shape, err)


def test_setup_with_tensor_gram_projects_within_tolerance(P):
    """BF16x3 Gram (the default) meets the 1e-5 projection bound without refinement; BF16
    and TF32 meet it with one refinement step against A (approximate projection, Section 3.2)."""
    import workloads as W
    from oracle import project as OPJ
    prob = W.nnls(3000, 700, seed=19)
    rng = np.random.default_rng(1)
    c = rng.normal(size=700).astype(np.float32)
    d = rng.normal(size=3000).astype(np.float32)
    for prec, refine in (("BF16X3", 0), ("BF16", 1), ("TF32", 1)):
        prm = P.pogs_default_params(gram_prec=prec, refine_steps=refine)
        with P.Solver(prob.A, prm) as s:
            assert P.pogs_get_setup_report(s.handle).gram_prec_used == P.GRAM[prec]
            proj = OPJ.Projector(s.ahat().astype(np.float64))
            x, y = s.project(c, d, prm)
        xr, yr = proj(c.astype(np.float64), d.astype(np.float64))
        ex = np.linalg.norm(x - xr) / np.linalg.norm(xr)
        ey = np.linalg.norm(y - yr) / np.linalg.norm(yr)
        assert ex < 1e-5 and ey < 1e-5, (prec, ex, ey)
