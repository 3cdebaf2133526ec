"""Graph-form ADMM, FP64 (Algorithm 1 + over-relaxation + the adaptive penalty of
Section 4.3), on the pre-conditioned problem of Eq. 12, returning the unscaled half-step tuple.

Readings of places where the paper is silent or ambiguous (each one is also listed in
the design notes):
  * rho^0 = params.rho0 (default 1); x^0 = y^0 = x~^0 = y~^0 = 0 (Algorithm 1).
  * Over-relaxation (Section 3.2) replaces x^{k+1/2} by alpha x^{k+1/2} + (1-alpha) x^k in
    the projection input and the dual update only; mu^{k+1/2}, nu^{k+1/2} and the
    residuals use the unrelaxed half step (Section 3.3, Eq. 11).
  * Residuals, their tolerances and the gap are measured on the pre-conditioned
    (iterated) problem: eps_pri = eps_abs + eps_rel ||y^{k+1/2}||,
    eps_dual = eps_abs + eps_rel ||mu^{k+1/2}|| (Section 3.4), literal norms.
  * Gap test: the half-step tuple is Fenchel feasible (Section 3.3), so its gap is
    eta = y^T nu + x^T mu (Eq. 7); with gap_stop it must also satisfy
    |eta| <= eps_abs + eps_rel |f(y) + g(x)| (Section 3.4's eps_gap).  gap_stop = False
    stops on the two residual tests alone, as Section 4.3 does.
  * Adaptive penalty (Section 4.3): the convergence test comes first; when it fails, the
    penalty controller below may change rho, with both bookkeeping steps starting at 0 and
    the iteration counter k = 0, 1, ...; on a change x~, y~ are rescaled by
    rho^k / rho^{k+1} (Section 3.2, 'Varying penalty').
  * Returned tuple (Section 5): x = E x^, y = D^{-1} y^, mu = E^{-1} mu^, nu = D nu^
    (the dual scalings follow from nu^T y = nu^^T y^ and mu^T x = mu^^T x^).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .equil import Equilibration, equilibrate, fold_f, fold_g, default_gamma
from .project import Projector, cgls
from .prox import prox_f, f_value


@dataclasses.dataclass
class Params:
    abs_tol: float = 1e-4
    rel_tol: float = 1e-3
    max_iter: int = 10000          # Section 6.1
    rho0: float = 1.0
    alpha: float = 1.7             # Section 5
    delta: float = 1.05            # Section 5
    tau: float = 0.8               # Section 5
    sk_sweeps: int = 10
    gamma: float | None = None     # None -> (m+n) sqrt(2^-23)
    adaptive_rho: bool = True
    gap_stop: bool = True
    equil: bool = True
    proj: str = "direct"           # "direct" (cached Cholesky) or "cgls" (indirect, Section 3.5)
    cg_iters: int = 50             # CGLS step cap per projection
    cg_tol: float = 1e-6           # CGLS stop: ||B^T r|| <= cg_tol ||r||


@dataclasses.dataclass
class Result:
    status: int          # 0 converged, 1 max_iter reached
    iters: int
    rho: float
    x: np.ndarray        # unscaled half-step tuple
    y: np.ndarray
    mu: np.ndarray
    nu: np.ndarray
    xh: np.ndarray       # pre-conditioned half-step tuple
    yh: np.ndarray
    muh: np.ndarray
    nuh: np.ndarray
    r_pri: float
    r_dual: float
    eps_pri: float
    eps_dual: float
    gap: float
    obj: float
    D: np.ndarray
    E: np.ndarray
    history: list


def _identity_equil(A):
    m, n = A.shape
    return Equilibration(np.ones(m), np.ones(n), A.copy())


@dataclasses.dataclass
class PenaltyController:
    """Adaptive penalty of Section 4.3.

    The controller waits until one residual has (approximately) converged and then nudges rho
    by the factor delta so that the other one follows: a small dual residual calls for a
    larger rho (a larger penalty favours primal feasibility, Section 3.2), a small primal
    residual for a smaller one.  To keep rho from flip-flopping, a change of direction is
    allowed only once tau * k has passed the iteration of the last change in the other
    direction.  When both residuals are small, the dual case is served first.  The state is
    just those two iteration numbers, both 0 at the start (k itself starts at 0, so nothing
    changes before k = 1).
    """
    delta: float
    tau: float
    k_last_increase: int = 0
    k_last_decrease: int = 0

    def next_rho(self, k: int, rho: float, dual_small: bool, primal_small: bool) -> float:
        """rho^{k+1} after the (not converged) iteration k run with rho^k = rho."""
        if dual_small and self.tau * k > self.k_last_decrease:
            self.k_last_increase = k
            return self.delta * rho
        if primal_small and self.tau * k > self.k_last_increase:
            self.k_last_decrease = k
            return rho / self.delta
        return rho


def rescale_scaled_duals(xt, yt, rho_old: float, rho_new: float):
    """Section 3.2, 'Varying penalty': x~ and y~ are duals scaled by 1/rho (Section 3.3 has
    mu^k = -rho x~^k, nu^k = -rho y~^k), so a change of rho multiplies them by
    rho^k / rho^{k+1}, which leaves the unscaled duals mu^k and nu^k as they were."""
    s = rho_old / rho_new
    return xt * s, yt * s


@dataclasses.dataclass
class StopTest:
    """The Section 3.4 quantities of one half-step tuple (pre-conditioned variables)."""
    r_pri: float       # ||A x^{k+1/2} - y^{k+1/2}||         (Eq. 11)
    r_dual: float      # ||A^T nu^{k+1/2} + mu^{k+1/2}||     (Eq. 11)
    eps_pri: float     # eps_abs + eps_rel ||y^{k+1/2}||
    eps_dual: float    # eps_abs + eps_rel ||mu^{k+1/2}||
    gap: float         # y^T nu + x^T mu of the Fenchel-feasible half tuple (Eq. 7)
    obj: float         # f(y^{k+1/2}) + g(x^{k+1/2})
    eps_gap: float     # eps_abs + eps_rel |obj|

    def converged(self, gap_stop: bool) -> bool:
        residuals_ok = self.r_pri < self.eps_pri and self.r_dual < self.eps_dual
        return residuals_ok and (not gap_stop or abs(self.gap) < self.eps_gap)


def section34_test(p: "Params", Ah, fh, gh, xh, yh, mu, nu) -> StopTest:
    """Residuals of Eq. 11 and the tolerances of Section 3.4 at the half-step tuple."""
    obj = float(np.sum(f_value(fh, yh, 1e-9)) + np.sum(f_value(gh, xh, 1e-9)))
    return StopTest(r_pri=float(np.linalg.norm(Ah @ xh - yh)),
                    r_dual=float(np.linalg.norm(Ah.T @ nu + mu)),
                    eps_pri=p.abs_tol + p.rel_tol * float(np.linalg.norm(yh)),
                    eps_dual=p.abs_tol + p.rel_tol * float(np.linalg.norm(mu)),
                    gap=float(yh @ nu + xh @ mu), obj=obj,
                    eps_gap=p.abs_tol + p.rel_tol * abs(obj))


def solve(A, f, g, params: Params | None = None, eq: Equilibration | None = None,
          record: bool = False, x0=None, nu0=None, factor: Projector | None = None) -> Result:
    """Solve Eq. 1 for the given f, g.  eq: a precomputed equilibration of A (else Algorithm 2
    runs here); factor: a Projector of eq.Ahat built earlier, reused instead of factoring again
    (Section 3.5, factorization caching)."""
    p = params or Params()
    A = np.asarray(A, np.float64)
    m, n = A.shape
    if eq is None:
        if p.equil:
            eq = equilibrate(A, p.sk_sweeps, p.gamma if p.gamma is not None else default_gamma(m, n))
        else:
            eq = _identity_equil(A)
    Ah, D, E = eq.Ahat, eq.D, eq.E
    fh, gh = fold_f(f, D), fold_g(g, E)
    proj = (factor if factor is not None else Projector(Ah)) if p.proj == "direct" else None
    u_cg = None   # CGLS warm start: the previous projection's least-squares variable

    x, xt = np.zeros(n), np.zeros(n)
    y, yt = np.zeros(m), np.zeros(m)
    rho = float(p.rho0)
    # Warm start (Section 5): an initial x^0 and/or nu^0 in the original variables.  In the
    # pre-conditioned problem x^ = E^-1 x and nu^ = D^-1 nu (the inverse of the unscaling of the
    # returned tuple).  The graph point starts at (x^0, A^ x^0); the scaled duals at
    # y~ = -nu^0 / rho and x~ = -A^T y~, which keeps the Section 3.3 invariant.  A part that is
    # not given starts at zero, and the first prox step estimates it: it returns nu^{1/2} in the
    # subdifferential of f at y^{1/2} (mu^{1/2} likewise for g).
    if x0 is not None:
        x = np.asarray(x0, np.float64) / E
        y = Ah @ x
    if nu0 is not None:
        yt = -(np.asarray(nu0, np.float64) / D) / rho
        xt = -(Ah.T @ yt)
    ctrl = PenaltyController(delta=p.delta, tau=p.tau)
    hist = []
    status, iters = 1, p.max_iter
    xh = yh = mu = nu = None
    st = None
    for k in range(p.max_iter):
        # Algorithm 1, prox step
        vx, vy = x - xt, y - yt
        xh = prox_f(gh, vx, rho)
        yh = prox_f(fh, vy, rho)
        # Section 3.3: feasible half-step duals
        mu = -rho * (xh - x + xt)
        nu = -rho * (yh - y + yt)
        # Section 3.2: over-relaxation
        xr = p.alpha * xh + (1.0 - p.alpha) * x
        yr = p.alpha * yh + (1.0 - p.alpha) * y
        # Algorithm 1, projection and dual update
        if proj is not None:
            xn, yn = proj(xr + xt, yr + yt)
        else:
            xn, yn, u_cg, _ = cgls(Ah, xr + xt, yr + yt, u0=u_cg, iters=p.cg_iters, tol=p.cg_tol)
        xt = xt + xr - xn
        yt = yt + yr - yn
        x, y = xn, yn
        # Section 3.4
        st = section34_test(p, Ah, fh, gh, xh, yh, mu, nu)
        if record:
            hist.append(dict(k=k, rho=rho, r_pri=st.r_pri, r_dual=st.r_dual, eps_pri=st.eps_pri,
                             eps_dual=st.eps_dual, gap=st.gap, obj=st.obj,
                             dual_inv=float(np.linalg.norm(xt + Ah.T @ yt))))
        if st.converged(p.gap_stop):
            status, iters = 0, k + 1
            break
        # Section 4.3 adaptive penalty, then the Section 3.2 rescale of the scaled duals
        if p.adaptive_rho:
            rho_new = ctrl.next_rho(k, rho, st.r_dual < st.eps_dual, st.r_pri < st.eps_pri)
            if rho_new != rho:
                xt, yt = rescale_scaled_duals(xt, yt, rho, rho_new)
                rho = rho_new

    if st is None:
        r_pri = r_dual = eps_pri = eps_dual = gap = obj = np.nan
    else:
        r_pri, r_dual, eps_pri, eps_dual, gap, obj = (st.r_pri, st.r_dual, st.eps_pri, st.eps_dual,
                                                      st.gap, st.obj)
    return Result(status=status, iters=iters, rho=rho,
                  x=E * xh, y=yh / D, mu=mu / E, nu=D * nu,
                  xh=xh, yh=yh, muh=mu, nuh=nu,
                  r_pri=r_pri, r_dual=r_dual, eps_pri=eps_pri, eps_dual=eps_dual,
                  gap=gap, obj=obj, D=D, E=E, history=hist)


def objective(A, f, g, x, y, tol=1e-7) -> float:
    """f(y) + g(x) of the original problem (Eq. 1)."""
    return float(np.sum(f_value(f, y, tol)) + np.sum(f_value(g, x, tol)))


def unscaled_residuals(A, x, y, mu, nu):
    """||A x - y|| and ||A^T nu + mu|| of the original problem (Eqs. 4, 5)."""
    A = np.asarray(A, np.float64)
    return float(np.linalg.norm(A @ x - y)), float(np.linalg.norm(A.T @ nu + mu))
