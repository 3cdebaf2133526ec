"""pogs_gram_noalloc -- the Gram formation for callers that cannot allocate device memory
(their device memory is owned by another allocator or a fixed budget, or their path cannot
afford cudaMalloc's synchronisation) -- gives the same result as pogs_gram, on two calls in a
row (the second call reuses the library's fixed scratch array left over from the first), and
requests no device memory from the library's allocator.

This file is collected last so that a run stopping at the first failure has already run every
other test.  It passes alone in a fresh process and after the others."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# same tolerances as the Gram tests (relative Frobenius error of the lower triangle)
TOL = {"BF16": 1e-2, "TF32": 2e-3, "BF16X3": 2e-5, "FP32": 1e-5}


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_08366_b300 as P
    return P


@pytest.mark.parametrize("prec", ["BF16X3", "TF32", "BF16", "FP32"])
def test_noalloc_matches_allocating_entry_point_twice(P, prec):
    import torch
    for call, (m, n) in enumerate([(1500, 700), (500, 1300)]):     # tall, then fat
        rng = np.random.default_rng(31 + call)
        A = torch.from_numpy((rng.standard_normal((m, n)) / np.sqrt(n)).astype(np.float32)).cuda()
        ref = P.pogs_gram(A, prec).cpu().numpy().astype(np.float64)
        q = min(m, n)
        G = torch.full((q, q), float("nan"), dtype=torch.float32, device="cuda")
        P.pogs_gram_noalloc(A, G, prec)
        got = G.cpu().numpy().astype(np.float64)
        lo = np.tril_indices(q)
        err = np.linalg.norm(got[lo] - ref[lo]) / np.linalg.norm(ref[lo])
        assert err <= TOL[prec], (prec, call, err)


def test_noalloc_rejects_oversized_problem_before_device_work(P):
    """K = 20000 rows of a 1000-column matrix needs 1024 x 20032 x 4 B > 32 MiB - 512 B for BF16x3."""
    import torch
    A = torch.zeros((20000, 1000), dtype=torch.float32, device="cuda")
    G = torch.zeros((1000, 1000), dtype=torch.float32, device="cuda")
    rc = P.lib.pogs_gram_noalloc(A.data_ptr(), 20000, 1000, 1000, P.GRAM["BF16X3"], G.data_ptr(), None)
    assert rc == -7   # POGS_ERR_CAPACITY
    rc = P.lib.pogs_gram_noalloc(None, 20000, 1000, 1000, P.GRAM["BF16X3"], G.data_ptr(), None)
    assert rc == -1   # POGS_ERR_ARG


def test_noalloc_requests_no_device_allocation(P):
    """The entry point's defining property: after a first call (which looks up the scratch
    array's device address), further calls request no device memory from the library --
    its allocation counter stays put -- while the allocating entry point moves it."""
    import torch
    A = torch.from_numpy(np.random.default_rng(5).standard_normal((900, 400)).astype(np.float32)).cuda()
    G = torch.zeros((400, 400), dtype=torch.float32, device="cuda")
    P.pogs_gram_noalloc(A, G, "BF16X3")
    torch.cuda.synchronize()
    before = P.pogs_device_allocations()
    for prec in ("BF16X3", "TF32", "BF16", "FP32"):
        P.pogs_gram_noalloc(A, G, prec)
    torch.cuda.synchronize()
    assert P.pogs_device_allocations() == before
    P.pogs_gram(A, "BF16X3")
    assert P.pogs_device_allocations() > before
