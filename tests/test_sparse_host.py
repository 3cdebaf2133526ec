"""Host-side pieces of the sparse path (no GPU): the CSR workload generator produces canonical
CSR (sorted, unique, in-range column indices, float32 values, the stated row density), and the
Python binding marshals CSR input and surfaces the library's argument errors before any device
work."""
import numpy as np
import pytest

import workloads as W


def test_sparse_lasso_generator_is_canonical_csr():
    prob = W.sparse_lasso(500, 300, seed=5, per_row=20)
    A = prob.A
    assert A.shape == (500, 300) and A.dtype == np.float32
    assert A.has_sorted_indices
    rp, ci = A.indptr, A.indices
    assert rp[0] == 0 and rp[-1] == A.nnz and np.all(np.diff(rp) >= 0)
    for r in range(A.shape[0]):
        row = ci[rp[r]:rp[r + 1]]
        assert np.all(np.diff(row) > 0)            # strictly increasing: sorted, no duplicates
        assert 0 < len(row) <= 20                   # per_row draws, repeats dropped
    assert np.all((ci >= 0) & (ci < 300))
    assert 0.9 * 500 * 20 <= A.nnz <= 500 * 20
    assert np.isfinite(A.data).all()
    # rows have the dense generator's expected squared norm (values N(0, 1/per_row))
    assert abs(float(np.mean(np.asarray(A.multiply(A).sum(axis=1)))) - 1.0) < 0.1


def test_csr_binding_rejects_bad_sizes_without_device_work():
    import paper_1503_08366_b300 as P
    rp = np.zeros(1, np.int32)
    with pytest.raises(P.PogsError):
        P.pogs_setup_csr(rp, np.zeros(0, np.int32), np.zeros(0, np.float32), (0, 5))
    with pytest.raises(P.PogsError):
        P.pogs_setup_csr(np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32), (3, 0))
