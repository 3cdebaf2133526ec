"""B300-native (sm_103a) graph-form ADMM: the per-iteration hot path of POGS
(separable proxes + graph projection with a cached Cholesky factor) behind a C ABI.

The Python layer only marshals arguments to libpogs_b300.so (include/pogs.h); there is
no CPU fallback -- importing fails if the CUDA library has not been built.
"""
from ._lib import (  # noqa: F401
    CHOL, ERR, GRAM, H, PROJ, KERNEL_NAMES, LIB_PATH, MAX_ITER, OK, PogsError, lib, pogs_default_params, pogs_fn,
    pogs_free, pogs_get_ahat, pogs_gram, pogs_gram_noalloc, pogs_get_equil, pogs_get_setup_report, pogs_info, pogs_kernel_launches, pogs_device_allocations, pogs_ldl_analyze,
    Server, pogs_params, pogs_problem, pogs_project, pogs_prox_eval, pogs_result, pogs_setup, pogs_setup_csr, pogs_solve_batch, pogs_setup_report, pogs_solve, pogs_solve_warm, pogs_time_kernels)
from .solver import Solver  # noqa: F401
