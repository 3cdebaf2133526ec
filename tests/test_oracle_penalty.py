"""Pins for the oracle's adaptive penalty (Section 4.3), the rescale of the scaled duals on a
change of rho (Section 3.2, 'Varying penalty') and the stopping test (Section 3.4).

None of these checks the oracle against a copy of itself:
  * the controller is driven with a hand-made sequence of residual outcomes and compared with
    rho values worked out by hand from the Section 4.3 description;
  * the rescale is checked by replaying the oracle's own rho schedule through ADMM written in
    the unscaled dual variables mu^k = -rho x~^k, nu^k = -rho y~^k (Section 3.3), which carry
    no scaling and so need no rescale at all: the two forms must give the same iterates;
  * the stopping test is checked from the outside: the half-step tuple the oracle returns at
    its stop iteration K must meet the Section 3.4 test evaluated here on that tuple, and the
    tuple it returns when capped at K - 1 iterations must not.
"""
import numpy as np
import pytest

import workloads as W
from oracle import admm as OA
from oracle import equil as OE
from oracle import project as OPJ
from oracle import prox as OP

# Residual outcomes (dual residual small, primal residual small) for k = 0..24 and rho^{k+1}
# after each, with delta = 2, tau = 0.8, rho^0 = 1.  Worked by hand from Section 4.3: a small
# dual residual raises rho if 0.8 k exceeds the iteration of the last decrease, else a small
# primal residual lowers it if 0.8 k exceeds the iteration of the last increase; both
# bookkeeping iterations start at 0 and the comparisons are strict.
HAND_SEQUENCE = [
    # k  dual   primal  rho^{k+1}   (why)
    (0, True, False, 1.0),     # 0.8*0 = 0 is not > 0
    (1, True, False, 2.0),     # 0.8 > 0: raise; last increase = 1
    (2, False, True, 1.0),     # 1.6 > 1: lower; last decrease = 2
    (3, True, False, 2.0),     # 2.4 > 2: raise; last increase = 3
    (4, False, True, 1.0),     # 3.2 > 3: lower; last decrease = 4
    (5, True, False, 1.0),     # 4.0 is not > 4 (strict)
    (6, True, False, 2.0),     # 4.8 > 4: raise; last increase = 6
    (7, False, True, 2.0),     # 5.6 is not > 6
    (8, False, True, 1.0),     # 6.4 > 6: lower; last decrease = 8
    (9, True, True, 0.5),      # raise blocked (7.2 <= 8), lower allowed (7.2 > 6); last decrease = 9
    (10, True, True, 0.25),    # raise blocked (8.0 <= 9), lower allowed; last decrease = 10
    (11, True, False, 0.25),   # 8.8 <= 10
    (12, True, False, 0.25),   # 9.6 <= 10
    (13, True, False, 0.5),    # 10.4 > 10: raise; last increase = 13
    (14, True, True, 1.0),     # both allowed? raise: 11.2 > 10 yes -> the dual case comes first
    (15, False, True, 1.0),    # 12.0 <= 14
    (16, False, True, 1.0),    # 12.8 <= 14
    (17, False, True, 1.0),    # 13.6 <= 14
    (18, False, True, 0.5),    # 14.4 > 14: lower; last decrease = 18
    (19, False, False, 0.5),
    (20, False, False, 0.5),
    (21, False, False, 0.5),
    (22, False, False, 0.5),
    (23, False, False, 0.5),
    (24, True, True, 1.0),     # both allowed (19.2 > 18 and > 14): the dual case wins, raise
]


def test_penalty_controller_hand_worked_sequence():
    ctrl = OA.PenaltyController(delta=2.0, tau=0.8)
    rho = 1.0
    got = []
    for k, dual_small, primal_small, _ in HAND_SEQUENCE:
        rho = ctrl.next_rho(k, rho, dual_small, primal_small)
        got.append(rho)
    assert got == [r for *_, r in HAND_SEQUENCE]


def test_delta_one_leaves_the_iteration_unchanged():
    """delta = 1 makes every penalty change a no-op: the iterates equal those of a fixed rho."""
    P = W.lasso(80, 30, seed=4)
    a = OA.solve(P.A, P.f, P.g, OA.Params(delta=1.0, max_iter=60), record=True)
    b = OA.solve(P.A, P.f, P.g, OA.Params(adaptive_rho=False, max_iter=60), record=True)
    assert [h["obj"] for h in a.history] == [h["obj"] for h in b.history]
    assert np.array_equal(a.xh, b.xh) and np.array_equal(a.nuh, b.nuh)


def _replay_unscaled(A, f, g, p: OA.Params, rhos):
    """ADMM (Algorithm 1 with over-relaxation) carried in the unscaled duals mu^k, nu^k of
    Section 3.3 and run with a given rho^k per iteration.  The scaled duals are only formed
    inside an iteration (x~ = -mu / rho^k with that iteration's rho), so a change of rho needs
    no rescale.  Returns the Section 3.4 quantities of every iteration."""
    eq = OE.equilibrate(np.asarray(A, float), p.sk_sweeps, OE.default_gamma(*A.shape))
    Ah = eq.Ahat
    fh, gh = OE.fold_f(f, eq.D), OE.fold_g(g, eq.E)
    proj = OPJ.Projector(Ah)
    m, n = Ah.shape
    x, y = np.zeros(n), np.zeros(m)
    mu, nu = np.zeros(n), np.zeros(m)           # mu^0 = nu^0 = 0
    out = []
    for rho in rhos:
        xs, ys = -mu / rho, -nu / rho            # x~^k, y~^k in this iteration's scaling
        xh = OP.prox_f(gh, x - xs, rho)
        yh = OP.prox_f(fh, y - ys, rho)
        muh = -rho * (xh - x + xs)
        nuh = -rho * (yh - y + ys)
        xr = p.alpha * xh + (1 - p.alpha) * x
        yr = p.alpha * yh + (1 - p.alpha) * y
        xn, yn = proj(xr + xs, yr + ys)
        mu = mu - rho * (xr - xn)                # -rho^k (x~^k + xr - x^{k+1})
        nu = nu - rho * (yr - yn)
        x, y = xn, yn
        out.append((np.linalg.norm(Ah @ xh - yh), np.linalg.norm(Ah.T @ nuh + muh), yh @ nuh + xh @ muh))
    return out


@pytest.mark.parametrize("cls,shape,seed", [("lasso", (80, 30), 4), ("logistic", (40, 60), 3),
                                            ("huber", (60, 25), 2)])
def test_rescale_on_rho_change_matches_unscaled_duals(cls, shape, seed):
    P = W.CLASSES[cls](*shape, seed=seed)
    p = OA.Params(max_iter=120)
    r = OA.solve(P.A, P.f, P.g, p, record=True)
    rhos = [h["rho"] for h in r.history]
    assert len(set(rhos)) >= 4, "the run must change rho several times"
    ref = _replay_unscaled(P.A.astype(float), P.f, P.g, p, rhos)
    for h, (rp, rd, gap) in zip(r.history, ref):
        assert h["r_pri"] == pytest.approx(rp, rel=1e-8, abs=1e-12)
        assert h["r_dual"] == pytest.approx(rd, rel=1e-8, abs=1e-12)
        assert h["gap"] == pytest.approx(gap, rel=1e-8, abs=1e-12)


def _section34_outside(A, res, p: OA.Params):
    """The Section 3.4 test on a returned tuple, in the pre-conditioned variables
    (x^ = x / E, y^ = D y, mu^ = E mu, nu^ = nu / D)."""
    Ah = res.D[:, None] * np.asarray(A, float) * res.E[None, :]
    xh, yh, muh, nuh = res.x / res.E, res.y * res.D, res.mu * res.E, res.nu / res.D
    r_pri = np.linalg.norm(Ah @ xh - yh)
    r_dual = np.linalg.norm(Ah.T @ nuh + muh)
    ok = (r_pri < p.abs_tol + p.rel_tol * np.linalg.norm(yh)
          and r_dual < p.abs_tol + p.rel_tol * np.linalg.norm(muh))
    if p.gap_stop:
        fh, gh = OE.fold_f(res.f_params, res.D), OE.fold_g(res.g_params, res.E)
        obj = float(np.sum(OP.f_value(fh, yh, 1e-9)) + np.sum(OP.f_value(gh, xh, 1e-9)))
        ok = ok and abs(yh @ nuh + xh @ muh) < p.abs_tol + p.rel_tol * abs(obj)
    return ok


# huber: g = 0, so mu^ = 0 and eps_dual = eps_abs while ||nu^|| is about 2 (a dual tolerance
# built on nu would stop far earlier); nnls 25x60: the primal test decides, ||x^|| >> ||y^||;
# lasso_small with the gap test: the gap decides the last iteration.
STOP_CASES = [("huber", (60, 25), 2, False), ("nnls", (25, 60), 0, False), ("lasso", (200, 100), 0, True),
              ("logistic", (40, 60), 3, False)]


@pytest.mark.parametrize("cls,shape,seed,gap_stop", STOP_CASES)
def test_stop_iteration_is_the_first_meeting_section34(cls, shape, seed, gap_stop):
    P = W.CLASSES[cls](*shape, seed=seed)
    p = OA.Params(gap_stop=gap_stop, max_iter=5000)
    A = P.A.astype(float)
    r = OA.solve(A, P.f, P.g, p)
    assert r.status == 0
    r.f_params, r.g_params = P.f, P.g
    assert _section34_outside(A, r, p), "the returned tuple must meet the Section 3.4 test"
    q = OA.Params(gap_stop=gap_stop, max_iter=r.iters - 1)
    prev = OA.solve(A, P.f, P.g, q)
    assert prev.status == 1
    prev.f_params, prev.g_params = P.f, P.g
    assert not _section34_outside(A, prev, q), "the iteration before the stop must fail the test"
