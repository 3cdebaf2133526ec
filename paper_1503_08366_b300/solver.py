"""Convenience wrapper around the C handle (setup once, solve many)."""
from __future__ import annotations

import numpy as np

from . import _lib as L


class Solver:
    """Owns one pogs_handle: factorization caching for a fixed matrix A (Section 3.5)."""

    def __init__(self, A, params: L.pogs_params | None = None, stream=None, order: str = "R"):
        """A: dense (numpy / torch) or a scipy.sparse matrix (set up through the CSR entry point)."""
        self.m, self.n = A.shape
        self.params = params if params is not None else L.pogs_default_params()
        if hasattr(A, "tocsr"):
            self.handle = L.pogs_setup_csr(A, None, None, A.shape, self.params, stream=stream)
        else:
            self.handle = L.pogs_setup(A, self.params, stream=stream, order=order)

    def solve(self, f, g, params: L.pogs_params | None = None, device_out: bool = False, x0=None, nu0=None):
        """Returns (info, x, y, mu, nu) -- the unscaled half-step tuple.  x0 / nu0: optional warm
        start (Section 5), host or device float32 arrays of length n / m."""
        if device_out:
            import torch
            x = torch.empty(self.n, dtype=torch.float32, device="cuda")
            mu = torch.empty_like(x)
            y = torch.empty(self.m, dtype=torch.float32, device="cuda")
            nu = torch.empty_like(y)
        else:
            x, mu = np.empty(self.n, np.float32), np.empty(self.n, np.float32)
            y, nu = np.empty(self.m, np.float32), np.empty(self.m, np.float32)
        prm = params if params is not None else self.params
        if x0 is None and nu0 is None:
            info = L.pogs_solve(self.handle, f, g, prm, x, y, mu, nu)
        else:
            info = L.pogs_solve_warm(self.handle, f, g, prm, x0, nu0, x, y, mu, nu)
        return info, x, y, mu, nu

    def equil(self):
        return L.pogs_get_equil(self.handle, self.m, self.n)

    def ahat(self):
        return L.pogs_get_ahat(self.handle, self.m, self.n)

    def project(self, c, d, params: L.pogs_params | None = None):
        return L.pogs_project(self.handle, c, d, params)

    def close(self):
        if self.handle:
            L.pogs_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
