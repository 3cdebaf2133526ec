"""Writes the FP64 oracle's reference results for the Gram-precision study (dense NNLS and an
inequality-form LP, both 30000 x 15000) to ``precision_<class>_30000x15000.json`` beside this
file.  Only the oracle runs here; the GPU results are compared against these stored values.

Two oracle runs per problem:
  * ``same_tol``: the stopping tolerances the GPU path runs at (eps_abs = 1e-4, eps_rel = 1e-3),
    so the GPU and the oracle are the same algorithm stopped by the same test;
  * ``tight``: a much tighter run whose objective stands in for p*.

Usage:  python tests/golden/make_precision_refs.py nnls|lp [--tight-rel R] [--tight-abs A]
Takes about a quarter of an hour (NNLS) to a few hours (LP) on 8 CPU cores.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W            # noqa: E402
from oracle import admm as OA    # noqa: E402

GEN = {"nnls": W.nnls_precision_large, "lp": W.lp_precision_large}
TIGHT = {"nnls": (1e-9, 1e-7), "lp": (1e-7, 1e-5)}


def _run(prob, abs_tol, rel_tol, max_iter):
    t0 = time.time()
    r = OA.solve(prob.A, prob.f, prob.g, OA.Params(abs_tol=abs_tol, rel_tol=rel_tol, max_iter=max_iter))
    return dict(abs_tol=abs_tol, rel_tol=rel_tol, max_iter=max_iter, status=int(r.status),
                iters=int(r.iters), obj=float(r.obj), r_pri=float(r.r_pri), r_dual=float(r.r_dual),
                eps_pri=float(r.eps_pri), eps_dual=float(r.eps_dual), gap=float(r.gap),
                seconds=round(time.time() - t0, 1))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cls", choices=sorted(GEN))
    ap.add_argument("--tight-abs", type=float, default=None)
    ap.add_argument("--tight-rel", type=float, default=None)
    ap.add_argument("--max-iter", type=int, default=40000)
    a = ap.parse_args()
    prob = GEN[a.cls]()
    m, n = prob.A.shape
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"precision_{a.cls}_{m}x{n}.json")
    rec = dict(problem=prob.name, m=m, n=n, seed=int(prob.meta["seed"]),
               generator=GEN[a.cls].__name__, threads=os.environ.get("OMP_NUM_THREADS", "all"))
    rec["same_tol"] = _run(prob, 1e-4, 1e-3, a.max_iter)
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
    ta, tr = TIGHT[a.cls]
    rec["tight"] = _run(prob, a.tight_abs or ta, a.tight_rel or tr, a.max_iter)
    with open(out, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
