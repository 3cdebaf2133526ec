"""ctypes binding of include/pogs.h -- argument marshalling only; every step of the
solver runs inside libpogs_b300.so.  Fails loudly when the library has not been built."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpogs_b300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -m paper_1503_08366_b300.build)")

lib = C.CDLL(LIB_PATH)

# ---- enums -----------------------------------------------------------------------------
H = dict(ZERO=0, ABS=1, SQUARE=2, HUBER=3, LOGISTIC=4, HINGE=5, MAXPOS=6, IND_GE0=7, IND_LE0=8,
         IND_EQ0=9, IND_BOX01=10, XLOGX=11)
OK, MAX_ITER = 0, 1
ERR = {-1: "ARG", -2: "OOM", -3: "NONFINITE", -4: "NUMERIC", -5: "TIMEOUT", -6: "CUDA", -7: "CAPACITY"}
GRAM = dict(BF16=0, TF32=1, BF16X3=2, FP32=3)
CHOL = dict(FP64=0, MIXED=1)
PROJ = dict(DIRECT=0, CGLS=1, LDL=2)


class pogs_fn(C.Structure):
    _fields_ = [("h", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p), ("c", C.c_void_p),
                ("d", C.c_void_p), ("e", C.c_void_p)]


class pogs_params(C.Structure):
    _fields_ = [("abs_tol", C.c_double), ("rel_tol", C.c_double), ("max_iter", C.c_int),
                ("rho0", C.c_double), ("alpha", C.c_double), ("delta", C.c_double), ("tau", C.c_double),
                ("sk_sweeps", C.c_int), ("gamma", C.c_double), ("gram_prec", C.c_int),
                ("refine_steps", C.c_int), ("gap_stop", C.c_int), ("adaptive_rho", C.c_int),
                ("equil", C.c_int), ("verbose", C.c_int), ("loop_mode", C.c_int), ("check_every", C.c_int),
                ("chol_prec", C.c_int), ("proj_mode", C.c_int), ("cg_max_iter", C.c_int), ("cg_tol", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pogs_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("rho", C.c_double), ("r_pri", C.c_double),
                ("r_dual", C.c_double), ("eps_pri", C.c_double), ("eps_dual", C.c_double),
                ("gap", C.c_double), ("obj", C.c_double), ("r_pri_unscaled", C.c_double),
                ("r_dual_unscaled", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pogs_setup_report(C.Structure):
    _fields_ = [("ingest_ms", C.c_double), ("equil_ms", C.c_double), ("gram_ms", C.c_double),
                ("factor_ms", C.c_double), ("inverse_ms", C.c_double), ("gram_prec_used", C.c_int),
                ("chol_prec_used", C.c_int), ("device_bytes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pogs_problem(C.Structure):
    _fields_ = [("A", C.c_void_p), ("m", C.c_int64), ("n", C.c_int64), ("lda", C.c_int64), ("f", pogs_fn),
                ("g", pogs_fn)]


class pogs_result(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("mu", C.c_void_p), ("nu", C.c_void_p), ("info", pogs_info)]


class pogs_server_done(C.Structure):
    _fields_ = [("tag", C.c_int64), ("info", pogs_info), ("submit_s", C.c_double), ("admit_s", C.c_double),
                ("done_s", C.c_double)]


_P = C.c_void_p
lib.pogs_default_params.argtypes = [C.POINTER(pogs_params)]
lib.pogs_default_params.restype = None
lib.pogs_setup.argtypes = [_P, C.c_int64, C.c_int64, C.c_int64, C.c_char, C.POINTER(pogs_params), _P, C.POINTER(_P)]
lib.pogs_setup.restype = C.c_int
lib.pogs_setup_csr.argtypes = [C.c_int64, C.c_int64, C.c_int64, _P, _P, _P, C.POINTER(pogs_params), _P, C.POINTER(_P)]
lib.pogs_setup_csr.restype = C.c_int
lib.pogs_check_bounded_wait.argtypes = [_P]
lib.pogs_check_bounded_wait.restype = C.c_int
lib.pogs_solve.argtypes = [_P, C.POINTER(pogs_fn), C.POINTER(pogs_fn), C.POINTER(pogs_params), _P, _P, _P, _P,
                           C.POINTER(pogs_info)]
lib.pogs_solve.restype = C.c_int
lib.pogs_solve_warm.argtypes = [_P, C.POINTER(pogs_fn), C.POINTER(pogs_fn), C.POINTER(pogs_params), _P, _P, _P, _P, _P,
                                _P, C.POINTER(pogs_info)]
lib.pogs_solve_warm.restype = C.c_int
lib.pogs_free.argtypes = [_P]
lib.pogs_free.restype = None
lib.pogs_prox_eval.argtypes = [C.POINTER(pogs_fn), C.c_int64, _P, _P, C.c_float, _P, _P]
lib.pogs_prox_eval.restype = C.c_int
lib.pogs_get_equil.argtypes = [_P, _P, _P]
lib.pogs_get_equil.restype = C.c_int
lib.pogs_get_ahat.argtypes = [_P, _P]
lib.pogs_get_ahat.restype = C.c_int
lib.pogs_project.argtypes = [_P, _P, _P, _P, _P, C.POINTER(pogs_params)]
lib.pogs_project.restype = C.c_int
lib.pogs_get_setup_report.argtypes = [_P, C.POINTER(pogs_setup_report)]
lib.pogs_get_setup_report.restype = C.c_int
lib.pogs_time_kernels.argtypes = [_P, C.c_int, _P, _P]
lib.pogs_time_kernels.restype = C.c_int
lib.pogs_gram.argtypes = [_P, C.c_int64, C.c_int64, C.c_int64, C.c_int, _P, _P]
lib.pogs_gram.restype = C.c_int
lib.pogs_gram_noalloc.argtypes = [_P, C.c_int64, C.c_int64, C.c_int64, C.c_int, _P, _P]
lib.pogs_gram_noalloc.restype = C.c_int
lib.pogs_solve_batch.argtypes = [C.c_int, C.POINTER(pogs_problem), C.POINTER(pogs_params), C.POINTER(pogs_result), _P]
lib.pogs_solve_batch.restype = C.c_int
lib.pogs_server_create.argtypes = [C.c_size_t, C.c_int, C.c_int, C.POINTER(pogs_params), _P, C.POINTER(_P)]
lib.pogs_server_create.restype = C.c_int
lib.pogs_server_submit.argtypes = [_P, C.POINTER(pogs_problem), _P, _P, _P, _P, C.c_int64]
lib.pogs_server_submit.restype = C.c_int
lib.pogs_server_step.argtypes = [_P, C.c_int]
lib.pogs_server_step.restype = C.c_int
lib.pogs_server_poll.argtypes = [_P, C.POINTER(pogs_server_done), C.c_int]
lib.pogs_server_poll.restype = C.c_int
lib.pogs_server_pending.argtypes = [_P]
lib.pogs_server_pending.restype = C.c_int
lib.pogs_server_destroy.argtypes = [_P]
lib.pogs_server_destroy.restype = None
lib.pogs_kernel_launches.argtypes = []
lib.pogs_kernel_launches.restype = C.c_longlong
lib.pogs_device_allocations.argtypes = []
lib.pogs_device_allocations.restype = C.c_longlong
lib.pogs_ldl_analyze.argtypes = [C.c_int64, C.c_int64, _P, _P, _P, _P, _P]
lib.pogs_ldl_analyze.restype = C.c_int


class PogsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where} failed with status {code} ({ERR.get(code, '?')})")
        self.code = code


def _check(code: int, where: str) -> int:
    if code < 0:
        raise PogsError(code, where)
    return code


# ---- marshalling helpers ------------------------------------------------------------------
_TORCH_DTYPES: dict = {}
_NP_DTYPES = {np.float32: np.dtype(np.float32), np.uint8: np.dtype(np.uint8)}


def _torch_dtype(dtype):
    if not _TORCH_DTYPES:
        import torch
        _TORCH_DTYPES.update({np.float32: torch.float32, np.uint8: torch.uint8})
    return _TORCH_DTYPES[dtype]


def _ptr(a, dtype, keep: list):
    """Raw pointer of a contiguous numpy array or torch tensor (host or device); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype is not _NP_DTYPES[dtype] or not a.flags.c_contiguous:
            a = np.ascontiguousarray(a, dtype=dtype)
        keep.append(a)
        return a.ctypes.data
    if hasattr(a, "data_ptr"):   # torch tensor
        want = _torch_dtype(dtype)
        if a.dtype != want or not a.is_contiguous():
            a = a.to(want).contiguous()
        keep.append(a)
        return a.data_ptr()
    arr = np.ascontiguousarray(a, dtype=dtype)
    keep.append(arr)
    return arr.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def make_fn(p, keep: list) -> pogs_fn:
    """pogs_fn from an object with attributes h, a, b, c, d, e (arrays or tensors; a..e may be None)."""
    return pogs_fn(_ptr(p.h, np.uint8, keep), _ptr(getattr(p, "a", None), np.float32, keep),
                   _ptr(getattr(p, "b", None), np.float32, keep), _ptr(getattr(p, "c", None), np.float32, keep),
                   _ptr(getattr(p, "d", None), np.float32, keep), _ptr(getattr(p, "e", None), np.float32, keep))


# ---- C entry points, same names ---------------------------------------------------------------
def pogs_default_params(**overrides) -> pogs_params:
    p = pogs_params()
    lib.pogs_default_params(C.byref(p))
    for k, v in overrides.items():
        if isinstance(v, str) and k == "gram_prec":
            v = GRAM[v.upper()]
        if isinstance(v, str) and k == "chol_prec":
            v = CHOL[v.upper()]
        if isinstance(v, str) and k == "proj_mode":
            v = PROJ[v.upper()]
        setattr(p, k, v)
    return p


def pogs_setup(A, params: pogs_params | None = None, stream=None, order: str = "R"):
    """A: 2-D float32 numpy array (host) or torch tensor (host or CUDA), logical shape (m, n).
    order 'R' passes A's row-major storage, 'C' its column-major storage. Returns a handle."""
    keep: list = []
    m, n = A.shape
    o = order.upper()
    if hasattr(A, "data_ptr"):
        import torch
        src = A.to(torch.float32)
        src = src.contiguous() if o == "R" else src.t().contiguous()
        ptr = src.data_ptr()
        keep.append(src)
    else:
        src = np.ascontiguousarray(A, np.float32) if o == "R" else np.asfortranarray(A, np.float32)
        ptr = src.ctypes.data
        keep.append(src)
    lda = n if o == "R" else m
    h = _P()
    rc = lib.pogs_setup(ptr, m, n, lda, o.encode(), C.byref(params) if params is not None else None,
                        _stream_ptr(stream), C.byref(h))
    _check(rc, "pogs_setup")
    return h.value


def pogs_setup_csr(indptr, indices, data, shape, params: pogs_params | None = None, stream=None):
    """Sparse A in CSR form: indptr (m + 1), indices (nnz, sorted and unique in each row), data
    (nnz); numpy arrays or torch tensors (host or CUDA), converted to int32 / float32.  Also
    accepts a scipy.sparse matrix as `indptr` (shape and the other arrays then come from it)."""
    if hasattr(indptr, "tocsr"):
        Asp = indptr.tocsr()
        Asp.sort_indices()
        Asp.sum_duplicates()
        indptr, indices, data, shape = Asp.indptr, Asp.indices, Asp.data, Asp.shape
    m, n = shape
    keep: list = []

    def arr(a, dt):
        if hasattr(a, "data_ptr"):
            import torch
            t = a.to(torch.int32 if dt == np.int32 else torch.float32).contiguous()
            keep.append(t)
            return t.data_ptr()
        v = np.ascontiguousarray(a, dt)
        keep.append(v)
        return v.ctypes.data

    rp, ci, va = arr(indptr, np.int32), arr(indices, np.int32), arr(data, np.float32)
    nnz = int(indices.numel() if hasattr(indices, "numel") else len(indices))
    h = _P()
    rc = lib.pogs_setup_csr(m, n, nnz, rp, ci, va, C.byref(params) if params is not None else None,
                            _stream_ptr(stream), C.byref(h))
    _check(rc, "pogs_setup_csr")
    return h.value


def pogs_solve(handle, f, g, params: pogs_params | None = None, x=None, y=None, mu=None, nu=None) -> pogs_info:
    """Outputs x, y, mu, nu: preallocated float32 arrays/tensors (host or device) or None."""
    keep: list = []
    fs, gs = make_fn(f, keep), make_fn(g, keep)
    info = pogs_info()
    rc = lib.pogs_solve(handle, C.byref(fs), C.byref(gs), C.byref(params) if params is not None else None,
                        _outptr(x), _outptr(y), _outptr(mu), _outptr(nu), C.byref(info))
    _check(rc, "pogs_solve")
    return info


def pogs_solve_warm(handle, f, g, params: pogs_params | None = None, x0=None, nu0=None, x=None, y=None, mu=None,
                    nu=None) -> pogs_info:
    """pogs_solve from an initial x0 (length n) and/or nu0 (length m), host or device, either None."""
    keep: list = []
    fs, gs = make_fn(f, keep), make_fn(g, keep)
    info = pogs_info()
    rc = lib.pogs_solve_warm(handle, C.byref(fs), C.byref(gs), C.byref(params) if params is not None else None,
                             _ptr(x0, np.float32, keep), _ptr(nu0, np.float32, keep), _outptr(x), _outptr(y),
                             _outptr(mu), _outptr(nu), C.byref(info))
    _check(rc, "pogs_solve_warm")
    return info


def _outptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous() and str(a.dtype) == "torch.float32"
        return a.data_ptr()
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def pogs_free(handle) -> None:
    lib.pogs_free(handle)


def pogs_prox_eval(fn, v, rho: float = 1.0, rho_vec=None, out=None, stream=None):
    """All arrays must be CUDA tensors of length k (the parametric prox of Section 5)."""
    keep: list = []
    fs = make_fn(fn, keep)
    import torch
    k = v.numel()
    if out is None:
        out = torch.empty_like(v)
    rc = lib.pogs_prox_eval(C.byref(fs), k, _ptr(v, np.float32, keep), _ptr(rho_vec, np.float32, keep),
                            C.c_float(rho), out.data_ptr(), _stream_ptr(stream))
    _check(rc, "pogs_prox_eval")
    return out


def pogs_get_equil(handle, m: int, n: int):
    D = np.empty(m, np.float32)
    E = np.empty(n, np.float32)
    _check(lib.pogs_get_equil(handle, D.ctypes.data, E.ctypes.data), "pogs_get_equil")
    return D, E


def pogs_get_ahat(handle, m: int, n: int):
    Ah = np.empty((m, n), np.float32)
    _check(lib.pogs_get_ahat(handle, Ah.ctypes.data), "pogs_get_ahat")
    return Ah


def pogs_project(handle, c, d, params: pogs_params | None = None):
    keep: list = []
    n, m = len(c), len(d)
    x = np.empty(n, np.float32)
    y = np.empty(m, np.float32)
    rc = lib.pogs_project(handle, _ptr(c, np.float32, keep), _ptr(d, np.float32, keep), x.ctypes.data,
                          y.ctypes.data, C.byref(params) if params is not None else None)
    _check(rc, "pogs_project")
    return x, y


def pogs_get_setup_report(handle) -> pogs_setup_report:
    r = pogs_setup_report()
    _check(lib.pogs_get_setup_report(handle, C.byref(r)), "pogs_get_setup_report")
    return r


KERNEL_NAMES = ("prox", "A_pass1", "Linv", "LinvT", "A_pass2", "check", "iteration")


def pogs_time_kernels(handle, reps: int = 20):
    """Per-kernel device times (ms) and algorithmic bytes of one iteration of the last solve."""
    ms = (C.c_double * 7)()
    by = (C.c_double * 7)()
    _check(lib.pogs_time_kernels(handle, reps, ms, by), "pogs_time_kernels")
    return {k: (ms[i], by[i]) for i, k in enumerate(KERNEL_NAMES)}


def pogs_kernel_launches() -> int:
    return int(lib.pogs_kernel_launches())


def pogs_device_allocations() -> int:
    return int(lib.pogs_device_allocations())


LDL_STATS = ("N", "nnz_l", "supernodes", "levels", "max_front", "panel_entries", "update_entries", "front_entries")


def pogs_ldl_analyze(indptr, indices, shape):
    """Symbolic analysis of the sparse LDL^T of K = [I A^T; A -I] for a CSR pattern (host arrays):
    returns (stats dict, perm, colcount)."""
    m, n = shape
    rp = np.ascontiguousarray(indptr, dtype=np.int32)
    ci = np.ascontiguousarray(indices, dtype=np.int32)
    stats = (C.c_int64 * 8)()
    perm = np.empty(m + n, np.int32)
    cc = np.empty(m + n, np.int32)
    _check(lib.pogs_ldl_analyze(m, n, rp.ctypes.data, ci.ctypes.data, stats, perm.ctypes.data, cc.ctypes.data),
           "pogs_ldl_analyze")
    return {k: int(stats[i]) for i, k in enumerate(LDL_STATS)}, perm, cc


def pogs_gram(A, gram_prec="BF16X3", stream=None):
    """G = A^T A (m >= n) or A A^T (m < n) for a CUDA float32 tensor A; lower triangle valid."""
    import torch
    m, n = A.shape
    A = A.contiguous()
    q = min(m, n)
    G = torch.zeros(q, q, dtype=torch.float32, device=A.device)
    prec = GRAM[gram_prec.upper()] if isinstance(gram_prec, str) else gram_prec
    _check(lib.pogs_gram(A.data_ptr(), m, n, n, prec, G.data_ptr(), _stream_ptr(stream)), "pogs_gram")
    return G


def pogs_gram_noalloc(A, G, gram_prec="BF16X3", stream=None):
    """pogs_gram into a caller-provided CUDA tensor G (q x q), using the library's fixed scratch."""
    m, n = A.shape
    prec = GRAM[gram_prec.upper()] if isinstance(gram_prec, str) else gram_prec
    assert A.is_contiguous() and G.is_contiguous() and G.shape == (min(m, n), min(m, n))
    return _check(lib.pogs_gram_noalloc(A.data_ptr(), m, n, n, prec, G.data_ptr(), _stream_ptr(stream)),
                  "pogs_gram_noalloc")


def _ptrs(arrs, dtype, keep: list, block: bool) -> np.ndarray:
    """Raw pointers (0 for None) of a sequence of arrays or tensors, by the rules of _ptr, as
    uint64.  Torch tensors keep their own storage (a converted copy when the dtype or layout
    differs).  With block, host arrays are copied end to end into one array of `dtype` (one
    allocation and one pass; a pointer lookup per numpy array costs microseconds, thousands of
    times per batch); without it each points at its own storage, as in _ptr."""
    out = np.zeros(len(arrs), np.uint64)
    if block and arrs and all(type(a) is np.ndarray and a.ndim == 1 for a in arrs):   # the common case
        blk = np.concatenate(arrs, dtype=dtype, casting="unsafe")
        keep.append(blk)
        sizes = np.fromiter((a.size for a in arrs), np.int64, len(arrs))
        starts = (np.cumsum(sizes) - sizes).astype(np.uint64)
        out[:] = np.uint64(blk.ctypes.data) + starts * np.uint64(blk.itemsize)
        return out
    if arrs and hasattr(arrs[0], "data_ptr"):
        want_t, tt = _torch_dtype(dtype), type(arrs[0])
        if all(type(a) is tt and a.dtype is want_t and a.is_contiguous() for a in arrs):   # tensors as given
            out[:] = np.fromiter((a.data_ptr() for a in arrs), np.uint64, len(arrs))
            return out
    host_i, host_a = [], []
    want_t = None
    for i, a in enumerate(arrs):
        if a is None:
            continue
        if hasattr(a, "data_ptr"):   # torch tensor
            if want_t is None:
                want_t = _torch_dtype(dtype)
            if a.dtype != want_t or not a.is_contiguous():
                a = a.to(want_t).contiguous()
                keep.append(a)
            out[i] = a.data_ptr()
        elif block:
            host_i.append(i)
            host_a.append(np.ravel(a))
        else:
            out[i] = _ptr(a, dtype, keep)
    if host_a:
        blk = np.concatenate(host_a, dtype=dtype, casting="unsafe")
        keep.append(blk)
        sizes = np.fromiter((x.size for x in host_a), np.int64, len(host_a))
        starts = (np.cumsum(sizes) - sizes).astype(np.uint64)
        out[host_i] = np.uint64(blk.ctypes.data) + starts * np.uint64(blk.itemsize)
    return out


# pogs_problem and pogs_result as rows of 8-byte words (filled column by column below)
_PROBLEM_WORDS = C.sizeof(pogs_problem) // 8
_RESULT_WORDS = C.sizeof(pogs_result) // 8
assert C.sizeof(pogs_problem) == 16 * 8 and pogs_problem.f.offset == 32 and pogs_problem.g.offset == 80
assert pogs_result.info.offset == 32 and C.sizeof(pogs_result) % 8 == 0


def pogs_solve_batch(problems, params: pogs_params | None = None, stream=None):
    """problems: objects with A (m x n float32, host array or CUDA tensor), f and g (h, a..e).
    Returns a list of (info, x, y, mu, nu) with host float32 outputs."""
    keep: list = []
    n_p = len(problems)
    cnt = max(1, n_p)
    probs = (pogs_problem * cnt)()
    res = (pogs_result * cnt)()
    mn = np.array([pb.A.shape for pb in problems], np.int64).reshape(n_p, 2)
    m, n = mn[:, 0], mn[:, 1]
    # words of each pogs_problem: A, m, n, lda, f.h .. f.e, g.h .. g.e
    w = np.frombuffer(probs, np.uint64).reshape(cnt, _PROBLEM_WORDS)[:n_p]
    w[:, 0] = _ptrs([pb.A for pb in problems], np.float32, keep, block=False)
    w[:, 1] = m
    w[:, 2] = n
    w[:, 3] = n
    fs = [pb.f for pb in problems]
    gs = [pb.g for pb in problems]
    w[:, 4] = _ptrs([f.h for f in fs], np.uint8, keep, block=True)
    w[:, 10] = _ptrs([g.h for g in gs], np.uint8, keep, block=True)
    for j, k in enumerate("abcde"):
        w[:, 5 + j] = _ptrs([getattr(f, k, None) for f in fs], np.float32, keep, block=True)
        w[:, 11 + j] = _ptrs([getattr(g, k, None) for g in gs], np.float32, keep, block=True)
    # all outputs in one host block: instance i's x, y, mu, nu are consecutive views
    tot = 2 * (m + n)
    off = np.cumsum(tot) - tot
    block = np.empty(int(tot.sum()), np.float32)
    base = np.uint64(block.ctypes.data)
    r = np.frombuffer(res, np.uint64).reshape(cnt, _RESULT_WORDS)[:n_p]
    r[:, 0] = base + 4 * off.astype(np.uint64)
    r[:, 1] = base + 4 * (off + n).astype(np.uint64)
    r[:, 2] = base + 4 * (off + n + m).astype(np.uint64)
    r[:, 3] = base + 4 * (off + 2 * n + m).astype(np.uint64)
    outs = [(block[o:o + ni], block[o + ni:o + ni + mi], block[o + ni + mi:o + 2 * ni + mi],
             block[o + 2 * ni + mi:o + 2 * (ni + mi)]) for o, mi, ni in zip(off.tolist(), m.tolist(), n.tolist())]
    rc = lib.pogs_solve_batch(n_p, probs, C.byref(params) if params is not None else None, res,
                              _stream_ptr(stream))
    _check(rc, "pogs_solve_batch")
    return [(res[i].info, *outs[i]) for i in range(n_p)]


class Server:
    """Continuous-batching server (pogs_server_*): submit, step, poll.  Keeps each request's
    input arrays and host output arrays alive until the request is polled."""

    def __init__(self, budget_bytes: int, large_workers: int = 8, max_resident: int = 4096,
                 params: pogs_params | None = None, stream=None):
        self.params = params if params is not None else pogs_default_params()
        h = _P()
        _check(lib.pogs_server_create(int(budget_bytes), large_workers, max_resident, C.byref(self.params),
                                      _stream_ptr(stream), C.byref(h)), "pogs_server_create")
        self.h = h.value
        self._live = {}

    def submit(self, prob, tag: int):
        keep: list = []
        m, n = prob.A.shape
        pr = pogs_problem()
        pr.A = _ptr(prob.A, np.float32, keep)
        pr.m, pr.n, pr.lda = m, n, n
        pr.f = make_fn(prob.f, keep)
        pr.g = make_fn(prob.g, keep)
        outs = [np.empty(n, np.float32), np.empty(m, np.float32), np.empty(n, np.float32), np.empty(m, np.float32)]
        _check(lib.pogs_server_submit(self.h, C.byref(pr), *(o.ctypes.data for o in outs), tag), "pogs_server_submit")
        self._live[tag] = (keep, pr, outs)

    def step(self, iters: int = 25):
        _check(lib.pogs_server_step(self.h, iters), "pogs_server_step")

    def poll(self, max_items: int = 4096):
        buf = (pogs_server_done * max_items)()
        k = lib.pogs_server_poll(self.h, buf, max_items)
        _check(k, "pogs_server_poll")
        res = []
        for i in range(k):
            d = buf[i]
            _, _, outs = self._live.pop(d.tag)
            res.append((d.tag, d.info, d.submit_s, d.admit_s, d.done_s, *outs))
        return res

    def pending(self) -> int:
        return lib.pogs_server_pending(self.h)

    def close(self):
        if self.h:
            lib.pogs_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
