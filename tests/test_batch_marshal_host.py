"""Host side of the batched binding (argument marshalling only, no GPU): the problem and result
tables that pogs_solve_batch hands to the C entry point.  The entry point is replaced by a
recorder for each test, which reads the memory behind every pointer while the call is in
progress and checks it against the caller's arrays: host parameter arrays may be gathered into
one block, matrices and torch tensors must be passed as they are, missing parameters as NULL,
and each instance's four outputs must be the consecutive host views the binding returns."""
import ctypes as C
from types import SimpleNamespace

import numpy as np
import pytest

import workloads as W


def _read(ptr, count, dtype):
    ct = C.c_uint8 if dtype == np.uint8 else C.c_float
    return np.array(np.ctypeslib.as_array((ct * count).from_address(int(ptr))), dtype=dtype)


@pytest.fixture
def L(monkeypatch):
    import paper_1503_08366_b300._lib as L
    seen = {}

    def recorder(n_p, probs, params, res, stream):
        seen["n"] = n_p
        seen["probs"] = [dict(A=probs[i].A, m=probs[i].m, n=probs[i].n, lda=probs[i].lda,
                              f=[getattr(probs[i].f, k) for k in "habcde"],
                              g=[getattr(probs[i].g, k) for k in "habcde"]) for i in range(n_p)]
        seen["res"] = [[getattr(res[i], k) for k in ("x", "y", "mu", "nu")] for i in range(n_p)]
        # the data behind every input pointer, read during the call
        seen["data"] = []
        for i in range(n_p):
            pr = seen["probs"][i]
            m, n = pr["m"], pr["n"]
            row = dict(A=_read(pr["A"], m * n, np.float32).reshape(m, n))
            for side, ln in (("f", m), ("g", n)):
                row[side] = [None if p is None else _read(p, ln, np.uint8 if t == 0 else np.float32)
                             for t, p in enumerate(pr[side])]
            seen["data"].append(row)
        for i in range(n_p):   # results the caller should find in the returned views
            for t, p in enumerate(seen["res"][i]):
                ln = seen["probs"][i]["n"] if t % 2 == 0 else seen["probs"][i]["m"]
                np.ctypeslib.as_array((C.c_float * ln).from_address(p))[:] = 100 * i + t
        return 0

    monkeypatch.setattr(L.lib, "pogs_solve_batch", recorder)
    return L, seen


def _mixed_problems():
    """Six instances of the batch mix, altered so that every marshalling case occurs: a float64
    parameter array, a strided one, a missing one (None) and a float64 matrix."""
    probs = W.batch_mix(count=6)
    out = []
    for i, p in enumerate(probs):
        f = SimpleNamespace(**{k: getattr(p.f, k) for k in "habcde"})
        g = SimpleNamespace(**{k: getattr(p.g, k) for k in "habcde"})
        A = p.A
        if i == 1:
            f.b = f.b.astype(np.float64)
        if i == 2:
            g.c = np.repeat(g.c, 2)[::2]            # strided view, same values
        if i == 3:
            g.e = None
        if i == 4:
            A = A.astype(np.float64)
        out.append(SimpleNamespace(A=A, f=f, g=g))
    return out


def _check_inputs(probs, seen):
    assert seen["n"] == len(probs)
    for p, pr, d in zip(probs, seen["probs"], seen["data"]):
        m, n = p.A.shape
        assert (pr["m"], pr["n"], pr["lda"]) == (m, n, n)
        assert np.array_equal(d["A"], np.asarray(p.A, np.float32))
        for side, fn in (("f", p.f), ("g", p.g)):
            for t, k in enumerate("habcde"):
                want = getattr(fn, k)
                if want is None:
                    assert pr[side][t] is None, (side, k)
                else:
                    assert np.array_equal(d[side][t], np.asarray(want, np.uint8 if t == 0 else np.float32)), (side, k)


def test_host_arrays_reach_the_entry_point_unchanged(L):
    Lm, seen = L
    probs = _mixed_problems()
    out = Lm.pogs_solve_batch(probs)
    _check_inputs(probs, seen)
    # matrices are passed in place when already float32 and C-contiguous
    for p, pr in zip(probs, seen["probs"]):
        if p.A.dtype == np.float32:
            assert pr["A"] == p.A.ctypes.data
    # outputs: x, y, mu, nu consecutive in one block, and the returned views are those regions
    prev_end = None
    for i, (p, ptrs, o) in enumerate(zip(probs, seen["res"], out)):
        m, n = p.A.shape
        assert [ptrs[1] - ptrs[0], ptrs[2] - ptrs[1], ptrs[3] - ptrs[2]] == [4 * n, 4 * m, 4 * n]
        if prev_end is not None:
            assert ptrs[0] == prev_end
        prev_end = ptrs[3] + 4 * m
        for t, view in enumerate(o[1:]):
            assert view.ctypes.data == ptrs[t] and view.dtype == np.float32
            assert np.all(view == 100 * i + t)


def test_tensors_are_passed_as_they_are(L):
    torch = pytest.importorskip("torch")
    Lm, seen = L
    probs = []
    for p in W.batch_mix(count=5):
        probs.append(SimpleNamespace(A=torch.from_numpy(p.A),
                                     f=SimpleNamespace(**{k: torch.from_numpy(getattr(p.f, k)) for k in "habcde"}),
                                     g=SimpleNamespace(**{k: torch.from_numpy(getattr(p.g, k)) for k in "habcde"})))
    Lm.pogs_solve_batch(probs)
    _check_inputs([SimpleNamespace(A=p.A.numpy(), f=SimpleNamespace(**{k: getattr(p.f, k).numpy() for k in "habcde"}),
                                   g=SimpleNamespace(**{k: getattr(p.g, k).numpy() for k in "habcde"})) for p in probs],
                  seen)
    for p, pr in zip(probs, seen["probs"]):
        assert pr["A"] == p.A.data_ptr()
        assert pr["f"] == [getattr(p.f, k).data_ptr() for k in "habcde"]
        assert pr["g"] == [getattr(p.g, k).data_ptr() for k in "habcde"]
    # a tensor of another dtype is converted (a copy with the same values)
    probs[0].f.b = probs[0].f.b.double()
    Lm.pogs_solve_batch(probs)
    assert np.array_equal(seen["data"][0]["f"][2], probs[0].f.b.float().numpy())


def test_empty_batch_is_handed_through(L):
    Lm, seen = L
    assert Lm.pogs_solve_batch([]) == []
    assert seen["n"] == 0
