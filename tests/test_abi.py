"""The C-ABI library loads and exports every entry point include/pogs.h declares (no GPU
needed: nothing is called except pogs_default_params, which touches no device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    names = set()
    for hp in HEADERS:
        src = open(hp).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|void|const char\s*\*|size_t|int64_t)\s+\**\s*(pogs_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("pogs_setup", "pogs_solve", "pogs_free", "pogs_default_params", "pogs_project",
                 "pogs_prox_eval"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_1503_08366_b300 as P
    lib = ctypes.CDLL(P.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params_match_paper():
    """Section 5: alpha = 1.7, (delta, tau) = (1.05, 0.8); Section 6.1: max_iter 1e4."""
    import paper_1503_08366_b300 as P
    p = P.pogs_default_params()
    assert (p.alpha, p.delta, p.tau, p.max_iter) == (1.7, 1.05, 0.8, 10000)
    assert (p.abs_tol, p.rel_tol, p.rho0) == (1e-4, 1e-3, 1.0)


def test_enum_values_match_workloads_and_header():
    import paper_1503_08366_b300 as P
    import workloads as W
    assert P.H == W.H
    hdr = open(os.path.join(ROOT, "include", "pogs.h")).read()
    for name, code in W.H.items():
        assert re.search(rf"POGS_{name}\s*=\s*{code}\b", hdr), name


def test_free_null_is_noop():
    import paper_1503_08366_b300 as P
    P.lib.pogs_free(None)


def test_setup_rejects_bad_arguments_without_device_work():
    """Argument checks happen before any CUDA call (ARG = -1)."""
    import paper_1503_08366_b300 as P
    h = ctypes.c_void_p()
    assert P.lib.pogs_setup(None, 10, 5, 5, b"R", None, None, ctypes.byref(h)) == -1
    buf = (ctypes.c_float * 50)()
    assert P.lib.pogs_setup(buf, 10, 5, 4, b"R", None, None, ctypes.byref(h)) == -1   # lda < n
    assert P.lib.pogs_setup(buf, 10, 5, 5, b"X", None, None, ctypes.byref(h)) == -1   # bad order
    assert P.lib.pogs_setup(buf, 0, 5, 5, b"R", None, None, ctypes.byref(h)) == -1    # empty
    p = P.pogs_default_params(alpha=2.5)
    assert P.lib.pogs_setup(buf, 10, 5, 5, b"R", ctypes.byref(p), None, ctypes.byref(h)) == -1


def test_setup_csr_rejects_bad_arguments_without_device_work():
    """Sizes, NULL arrays and out-of-range counts are refused before any CUDA call."""
    import paper_1503_08366_b300 as P
    h = ctypes.c_void_p()
    rp = (ctypes.c_int * 3)(0, 1, 2)
    ci = (ctypes.c_int * 2)(0, 1)
    va = (ctypes.c_float * 2)(1.0, 2.0)
    f = P.lib.pogs_setup_csr
    assert f(2, 2, 2, None, ci, va, None, None, ctypes.byref(h)) == -1          # no row pointers
    assert f(2, 2, 2, rp, None, va, None, None, ctypes.byref(h)) == -1          # nnz > 0, no indices
    assert f(2, 2, 2, rp, ci, None, None, None, ctypes.byref(h)) == -1          # nnz > 0, no values
    assert f(0, 2, 0, rp, ci, va, None, None, ctypes.byref(h)) == -1            # no rows
    assert f(2, 0, 0, rp, ci, va, None, None, ctypes.byref(h)) == -1            # no columns
    assert f(2, 2, -1, rp, ci, va, None, None, ctypes.byref(h)) == -1           # negative nnz
    assert f(2, 2, 1 << 31, rp, ci, va, None, None, ctypes.byref(h)) == -1      # nnz beyond int32
    p = P.pogs_default_params(alpha=2.5)
    assert f(2, 2, 2, rp, ci, va, ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert f(2, 2, 2, rp, ci, va, None, None, None) == -1                       # no output


def test_server_and_batch_reject_bad_arguments_without_device_work():
    """The server and batch entry points check their arguments before any CUDA call (ARG = -1);
    destroying a NULL server is a no-op."""
    import paper_1503_08366_b300 as P
    lib = P.lib
    s = ctypes.c_void_p()
    assert lib.pogs_server_create(0, 1, 4, None, None, ctypes.byref(s)) == -1          # no budget
    assert lib.pogs_server_create(1 << 20, -1, 4, None, None, ctypes.byref(s)) == -1   # workers < 0
    assert lib.pogs_server_create(1 << 20, 1, 0, None, None, ctypes.byref(s)) == -1    # no slots
    assert lib.pogs_server_create(1 << 20, 1, 4, None, None, None) == -1               # no out
    pr = P.pogs_problem()
    assert lib.pogs_server_submit(None, ctypes.byref(pr), None, None, None, None, 0) == -1
    assert lib.pogs_server_step(None, 25) == -1
    assert lib.pogs_server_poll(None, None, 0) == -1
    assert lib.pogs_server_pending(None) == -1
    lib.pogs_server_destroy(None)
    out = (P.pogs_result * 2)()
    probs = (P.pogs_problem * 2)()
    assert lib.pogs_solve_batch(-1, probs, None, out, None) == -1                      # count < 0
    assert lib.pogs_solve_batch(2, None, None, out, None) == -1                        # no problems
    assert lib.pogs_solve_batch(2, probs, None, None, None) == -1                      # no results
    buf = (ctypes.c_float * 12)()
    h = (ctypes.c_uint8 * 4)()
    for k in range(2):
        probs[k].A = ctypes.cast(buf, ctypes.c_void_p)
        probs[k].m, probs[k].n, probs[k].lda = 4, 3, 3
        probs[k].f.h = ctypes.cast(h, ctypes.c_void_p)
        probs[k].g.h = ctypes.cast(h, ctypes.c_void_p)
    probs[1].lda = 2                                                                  # lda < n
    assert lib.pogs_solve_batch(2, probs, None, out, None) == -1
    probs[1].lda, probs[1].m = 3, 0                                                   # empty
    assert lib.pogs_solve_batch(2, probs, None, out, None) == -1
    assert lib.pogs_solve_batch(0, probs, None, out, None) == 0                        # nothing to do


def test_handle_entry_points_reject_null_before_device_work():
    """Every entry point that takes a handle returns ARG (-1) for a NULL handle or a missing
    required array without touching the device; prox evaluation of zero elements is a no-op."""
    import paper_1503_08366_b300 as P
    lib = P.lib
    fn = P.pogs_fn()
    info = P.pogs_info()
    buf = (ctypes.c_float * 8)()
    assert lib.pogs_solve(None, ctypes.byref(fn), ctypes.byref(fn), None, None, None, None, None,
                          ctypes.byref(info)) == -1
    assert lib.pogs_solve_warm(None, ctypes.byref(fn), ctypes.byref(fn), None, None, None, None, None, None,
                               None, ctypes.byref(info)) == -1
    assert lib.pogs_get_equil(None, buf, buf) == -1
    assert lib.pogs_get_ahat(None, buf) == -1
    assert lib.pogs_project(None, buf, buf, buf, buf, None) == -1
    rep = P.pogs_setup_report()
    assert lib.pogs_get_setup_report(None, ctypes.byref(rep)) == -1
    ms = (ctypes.c_double * 8)()
    assert lib.pogs_time_kernels(None, 3, ms, ms) == -1
    h = (ctypes.c_uint8 * 4)()
    fn.h = ctypes.cast(h, ctypes.c_void_p)
    assert lib.pogs_prox_eval(None, 4, buf, None, ctypes.c_float(1.0), buf, None) == -1   # no function
    assert lib.pogs_prox_eval(ctypes.byref(fn), -1, buf, None, ctypes.c_float(1.0), buf, None) == -1
    assert lib.pogs_prox_eval(ctypes.byref(fn), 0, buf, None, ctypes.c_float(1.0), buf, None) == 0
