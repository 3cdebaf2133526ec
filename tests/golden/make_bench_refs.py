"""Writes the FP64 oracle's results for the two large solves of the default benchmark step
(tall Lasso 40000 x 10000 and fat l1-logistic 2000 x 40000, the workload generators' seeds
10000 and 10001) to ``bench_<class>_<m>x<n>.json`` beside this file.  Only the oracle runs
here, stopped by the same test the GPU path uses (eps_abs = 1e-4, eps_rel = 1e-3); the
full-size GPU test compares its objective against these stored values.

Usage:  python tests/golden/make_bench_refs.py      (a few minutes on 16 CPU cores)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W            # noqa: E402
from oracle import admm as OA    # noqa: E402


def main():
    for gen in (W.lasso_tall_large, W.logistic_fat_large):
        prob = gen()
        m, n = prob.A.shape
        t0 = time.time()
        r = OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=1e-4, rel_tol=1e-3, max_iter=20000))
        rec = dict(problem=prob.name, m=m, n=n, seed=int(prob.meta["seed"]), generator=gen.__name__,
                   abs_tol=1e-4, rel_tol=1e-3, status=int(r.status), iters=int(r.iters), obj=float(r.obj),
                   r_pri=float(r.r_pri), r_dual=float(r.r_dual), eps_pri=float(r.eps_pri),
                   eps_dual=float(r.eps_dual), seconds=round(time.time() - t0, 1))
        out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"bench_{prob.name}_{m}x{n}.json")
        with open(out, "w") as fh:
            json.dump(rec, fh, indent=1)
        print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
