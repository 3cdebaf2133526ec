"""Host logic of the sparse LDL^T of K = [I A^T; A -I] (Section 3.5, sparse direct method): the
symbolic analysis that runs on the CPU at setup (ordering, elimination tree, column counts,
supernodes), checked against brute-force symbolic elimination on the graph of K and against the
structure of a dense LDL^T of the permuted matrix.  No GPU needed."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W


@pytest.fixture(scope="module")
def P():
    import paper_1503_08366_b300 as P
    return P


def _graph(A):
    """Adjacency sets of the graph of K (unknowns x_0..x_{n-1}, then y_i = n + i)."""
    m, n = A.shape
    adj = [set() for _ in range(n + m)]
    coo = A.tocoo()
    for i, j in zip(coo.row, coo.col):
        adj[j].add(n + i)
        adj[n + i].add(j)
    return adj


def _brute_colcounts(adj, order):
    """Eliminate the unknowns in `order` on the graph: each one's later neighbours become a clique;
    the count of later neighbours at its elimination is its column count in L."""
    pos = {v: k for k, v in enumerate(order)}
    nbr = [set(s) for s in adj]
    out = []
    for k, v in enumerate(order):
        later = {u for u in nbr[v] if pos[u] > k}
        out.append(len(later))
        for a in later:
            nbr[a] |= later - {a}
    return np.array(out)


def _patterns():
    rng = np.random.default_rng(3)
    rand = sp.random(40, 25, density=0.12, random_state=rng, format="csr", dtype=np.float32)
    rand.sort_indices()
    return {
        "banded": W.banded_lasso(60, 40, seed=1, half_band=3).A,
        "banded_fat": W.banded_lasso(30, 70, seed=2, half_band=2).A,
        "block_angular": W.block_angular_lasso(4, 12, 9, 3, seed=4, density=0.3, coupling_density=0.2).A,
        "random": rand,
        "empty_rows_cols": sp.csr_matrix((np.ones(3, np.float32), ([0, 0, 5], [1, 7, 2])), shape=(8, 9)),
    }


@pytest.mark.parametrize("name", list(_patterns()))
def test_symbolic_counts_match_brute_force_elimination(P, name):
    A = _patterns()[name]
    A.sort_indices()
    m, n = A.shape
    stats, perm, cc = P.pogs_ldl_analyze(A.indptr, A.indices, A.shape)
    assert stats["N"] == m + n
    assert sorted(perm.tolist()) == list(range(m + n)), "the ordering is a permutation"
    want = _brute_colcounts(_graph(A), perm.tolist())
    assert np.array_equal(cc, want)
    assert stats["nnz_l"] >= int(cc.sum())          # supernodes may store explicit zeros
    assert stats["supernodes"] >= 1 and stats["levels"] >= 1


@pytest.mark.parametrize("name", ["banded", "block_angular", "random"])
def test_dense_ldl_of_permuted_K_stays_in_the_predicted_structure(P, name):
    """P K P^T = L D L^T with random values on the pattern: every entry of L that is not zero
    lies where the symbolic analysis predicts one, and D has the signs of quasi-definiteness
    (positive on x unknowns, negative on y unknowns)."""
    A = _patterns()[name]
    m, n = A.shape
    _, perm, cc = P.pogs_ldl_analyze(A.indptr, A.indices, A.shape)
    Ad = A.toarray().astype(np.float64)
    K = np.block([[np.eye(n), Ad.T], [Ad, -np.eye(m)]])
    Kp = K[np.ix_(perm, perm)]
    N = m + n
    L = np.eye(N)
    d = np.zeros(N)
    S = Kp.copy()
    for k in range(N):                         # right-looking LDL^T without pivoting
        d[k] = S[k, k]
        L[k + 1:, k] = S[k + 1:, k] / d[k]
        S[k + 1:, k + 1:] -= np.outer(L[k + 1:, k], L[k + 1:, k]) * d[k]
    assert np.allclose(L @ np.diag(d) @ L.T, Kp, atol=1e-10)
    assert np.all(d[perm < n] > 0) and np.all(d[perm >= n] < 0)
    nz = (np.abs(np.tril(L, -1)) > 1e-13).sum(axis=0)
    assert np.all(nz <= cc)


def test_nested_dissection_keeps_banded_fill_low(P):
    """A banded A keeps L sparse: far fewer entries than the dense triangle and within a small
    factor of the natural (band) ordering, whose fill is the band itself."""
    A = W.banded_lasso(3000, 2000, seed=5, half_band=4).A
    m, n = A.shape
    stats, perm, cc = P.pogs_ldl_analyze(A.indptr, A.indices, A.shape)
    N = m + n
    assert stats["nnz_l"] < 0.01 * N * (N - 1) / 2
    assert stats["levels"] < 80, stats


def test_block_angular_coupling_rows_are_ordered_last(P):
    """The coupling rows (dense in A) are taken out of the dissection and eliminated last, so the
    blocks factor independently."""
    A = W.block_angular_lasso(8, 200, 100, 10, seed=6, density=0.05, coupling_density=0.5).A
    m, n = A.shape
    stats, perm, _ = P.pogs_ldl_analyze(A.indptr, A.indices, A.shape)
    coupling = set(range(n + m - 10, n + m))
    assert set(perm[-10:].tolist()) == coupling


def test_malformed_pattern_is_rejected(P):
    rp = np.array([0, 2, 3], np.int32)
    with pytest.raises(P.PogsError):
        P.pogs_ldl_analyze(rp, np.array([1, 0, 2], np.int32), (2, 3))     # unsorted row
    with pytest.raises(P.PogsError):
        P.pogs_ldl_analyze(rp, np.array([0, 1, 3], np.int32), (2, 3))     # column out of range


def _colcounts_by_column_structures(A, perm):
    """Column counts of L for P K P^T by the column-structure recurrence: struct(j) = the later
    neighbours of j, together with struct(c) minus {j} for every child c of j in the elimination
    tree (the tree computed here with ancestor links)."""
    m, n = A.shape
    N = m + n
    adj = [[] for _ in range(N)]
    coo = A.tocoo()
    for i, j in zip(coo.row.tolist(), coo.col.tolist()):
        adj[j].append(n + i)
        adj[n + i].append(j)
    iperm = np.empty(N, np.int64)
    iperm[np.asarray(perm)] = np.arange(N)
    nadj = [[int(iperm[u]) for u in adj[perm[k]]] for k in range(N)]
    parent, anc = [-1] * N, [-1] * N
    for k in range(N):
        for i in nadj[k]:
            while i != -1 and i < k:
                nxt = anc[i]
                anc[i] = k
                if nxt == -1:
                    parent[i] = k
                i = nxt
    kids = [[] for _ in range(N)]
    for j in range(N):
        if parent[j] >= 0:
            kids[parent[j]].append(j)
    st, counts = [None] * N, np.zeros(N, np.int64)
    for j in range(N):
        s = {i for i in nadj[j] if i > j}
        for c in kids[j]:
            s |= st[c]
            st[c] = None            # a child's structure is read by its parent only
        s.discard(j)
        st[j], counts[j] = s, len(s)
    return counts


def test_large_pattern_counts_and_deterministic_ordering(P):
    """A pattern large enough that the ordering's halves are dissected on separate threads: the
    ordering is the same on every call, and the column counts agree with the column-structure
    recurrence evaluated independently here."""
    A = W.banded_lasso(40000, 20000, seed=9, half_band=2).A
    m, n = A.shape
    stats, perm, cc = P.pogs_ldl_analyze(A.indptr, A.indices, A.shape)
    _, perm2, cc2 = P.pogs_ldl_analyze(A.indptr, A.indices, A.shape)
    assert np.array_equal(perm, perm2) and np.array_equal(cc, cc2)
    assert np.array_equal(np.sort(perm), np.arange(m + n))
    assert np.array_equal(cc, _colcounts_by_column_structures(A, perm.tolist()))
    assert stats["nnz_l"] >= int(cc.sum())


_OOM_CHILD = r"""
import resource, sys
import numpy as np
import paper_1503_08366_b300 as P
import workloads as W
A = W.banded_lasso(200000, 100000, seed=1, half_band=8).A
rp = np.ascontiguousarray(A.indptr, np.int32)
ci = np.ascontiguousarray(A.indices, np.int32)
size = next(int(l.split()[1]) * 1024 for l in open('/proc/self/status') if l.startswith('VmSize'))
resource.setrlimit(resource.RLIMIT_AS, (size + 64 * 2**20, resource.RLIM_INFINITY))
try:
    P.pogs_ldl_analyze(rp, ci, A.shape)
    print('NO ERROR')
except P.PogsError as e:
    print('ERROR', e.code)
"""


def test_analysis_out_of_host_memory_returns_an_error():
    """With the process's address space capped just above its current size, the analysis of a
    large pattern runs out of host memory: it returns POGS_ERR_OOM (in a worker thread or the
    calling one) instead of ending the process."""
    import os
    import subprocess
    import sys
    from paper_1503_08366_b300 import _lib
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _OOM_CHILD], cwd=root, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, PYTHONPATH=root))
    assert r.returncode == 0, r.stderr[-2000:]
    oom = next(k for k, v in _lib.ERR.items() if v == "OOM")
    assert r.stdout.split() == ["ERROR", str(oom)], r.stdout
