"""The mixed-workload input generators follow their stated recipes (no GPU):

  * the serving trace: Poisson arrivals at 2000/s (exponential gaps: mean 1/rate, coefficient
    of variation 1, a Kolmogorov-Smirnov test against the exponential law), the five classes
    in equal shares, m log-uniform on [100, 8000] and n on [50, 4000] (uniform in log m);
  * the batch mix: four classes, m log-uniform on [64, 2048], n on [32, 512];
  * both are reproducible from their seeds, and a request's payload matches its shape.
"""
import numpy as np
import pytest
from scipy import stats

import workloads as W


@pytest.fixture(scope="module")
def trace():
    return W.serve_trace(count=20000)


def _log_uniform_ok(v, lo, hi):
    v = np.asarray(v, np.float64)
    assert v.min() >= lo and v.max() <= hi
    u = (np.log(v) - np.log(lo)) / (np.log(hi) - np.log(lo))
    # rounding to integers distorts the low end slightly; the KS distance stays small
    return stats.kstest(u, "uniform").statistic


def test_serve_trace_arrivals_are_poisson_at_the_stated_rate(trace):
    t = np.array([r.arrival_s for r in trace])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() * 2000.0 - 1.0) < 0.03               # 20000 gaps: s.e. 0.7%
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03           # exponential: CV = 1
    assert stats.kstest(gaps * 2000.0, "expon").pvalue > 1e-3
    assert 9.5 < t[-1] < 10.5                                   # 20000 requests in ~10 s


def test_serve_trace_classes_and_shapes(trace):
    cls = [r.cls for r in trace]
    shares = {c: cls.count(c) / len(cls) for c in set(cls)}
    assert sorted(shares) == sorted(["lasso", "logistic", "huber", "svm", "nnls"])
    assert all(abs(s - 0.2) < 0.02 for s in shares.values()), shares
    assert _log_uniform_ok([r.m for r in trace], 100, 8000) < 0.02
    assert _log_uniform_ok([r.n for r in trace], 50, 4000) < 0.02


def test_serve_trace_is_reproducible_and_payloads_match(trace):
    again = W.serve_trace(count=50)
    assert [(r.arrival_s, r.cls, r.m, r.n, r.seed) for r in again] == \
           [(r.arrival_s, r.cls, r.m, r.n, r.seed) for r in trace[:50]]
    for r in trace[:3]:
        p = r.problem()
        assert p.A.shape == (r.m, r.n) and p.A.dtype == np.float32 and p.name == r.cls
        q = r.problem()
        assert np.array_equal(p.A, q.A)


def test_batch_mix_follows_its_recipe():
    probs = W.batch_mix(count=400, base_seed=20_000)
    names = [p.name for p in probs]
    assert set(names) == {"lasso", "huber", "svm", "nnls"}
    assert all(abs(names.count(c) / 400 - 0.25) < 0.08 for c in set(names))
    assert _log_uniform_ok([p.A.shape[0] for p in probs], 64, 2048) < 0.08
    assert _log_uniform_ok([p.A.shape[1] for p in probs], 32, 512) < 0.08
    again = W.batch_mix(count=5, base_seed=20_000)
    for p, q in zip(probs[:5], again):
        assert np.array_equal(p.A, q.A)
