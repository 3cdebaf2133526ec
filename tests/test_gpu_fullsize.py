"""The two large solves of the default benchmark step at full size (tall Lasso 40000 x 10000,
fat l1-logistic 2000 x 40000), in the configuration the benchmark times (default parameters,
inputs resident on the device, the device-side graph loop):

  * objective within 1e-3 of the FP64 oracle stopped by the same test (stored values written
    by tests/golden/make_bench_refs.py, which runs only the oracle);
  * primal and dual feasibility of the returned unscaled tuple, ||A x - y|| and ||A^T nu + mu||,
    recomputed in FP64 on the host;
  * one full-size projection of random (c, d) in the benchmark's configuration: within 1e-5
    relative, in x and in y, of the FP64 projection of the same input on the handle's A^
    (factored on the host in FP64), and its optimality conditions x - c + A^T(y - d) = 0 and
    y = A x.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import project as OPJ

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_08366_b300 as P
    return P


@pytest.mark.parametrize("gen", [W.lasso_tall_large, W.logistic_fat_large])
def test_benchmark_solves_at_full_size(P, gen):
    import torch
    prob = gen()
    m, n = prob.A.shape
    ref = json.load(open(os.path.join(GOLD, f"bench_{prob.name}_{m}x{n}.json")))
    A = torch.from_numpy(prob.A).cuda()
    prm = P.pogs_default_params()
    with P.Solver(A, prm) as s:
        info, x, y, mu, nu = s.solve(prob.f, prob.g)
        rng = np.random.default_rng(91)
        c = rng.normal(size=n).astype(np.float32)
        d = rng.normal(size=m).astype(np.float32)
        xp, yp = s.project(c, d, prm)
        Ah = s.ahat()
    del A
    assert info.status == 0, info.as_dict()
    assert abs(info.obj - ref["obj"]) <= 1e-3 * max(1.0, abs(ref["obj"])), (info.obj, ref["obj"])

    A64 = prob.A.astype(np.float64)
    x64, y64, mu64, nu64 = (v.astype(np.float64) for v in (x, y, mu, nu))
    r_pri = np.linalg.norm(A64 @ x64 - y64)
    r_dual = np.linalg.norm(A64.T @ nu64 + mu64)
    assert r_pri <= 1e-2 * max(1.0, np.linalg.norm(y64)), r_pri
    assert r_dual <= 1e-2 * max(1.0, np.linalg.norm(mu64)), r_dual
    # the solver's own unscaled residuals describe the same tuple
    assert abs(r_pri - info.r_pri_unscaled) <= 1e-2 * max(r_pri, 1e-6)
    assert abs(r_dual - info.r_dual_unscaled) <= 1e-2 * max(r_dual, 1e-6)
    del A64

    Ah = Ah.astype(np.float64)
    xp64, yp64 = xp.astype(np.float64), yp.astype(np.float64)
    c64, d64 = c.astype(np.float64), d.astype(np.float64)
    xr, yr = OPJ.Projector(Ah)(c64, d64)
    ex = np.linalg.norm(xp64 - xr) / np.linalg.norm(xr)
    ey = np.linalg.norm(yp64 - yr) / np.linalg.norm(yr)
    assert ex < 1e-5 and ey < 1e-5, (ex, ey)
    stat = xp64 - c64 + Ah.T @ (yp64 - d64)
    assert np.linalg.norm(stat) <= 1e-4 * np.linalg.norm(c64 + Ah.T @ d64), np.linalg.norm(stat)
    assert np.linalg.norm(yp64 - Ah @ xp64) <= 1e-5 * np.linalg.norm(yp64)
