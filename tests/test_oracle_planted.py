"""The pins must catch plausible mistakes: each case plants one in the oracle (on the CPU,
via monkeypatch) and checks that the corresponding pin then fails."""
import numpy as np
import pytest

from oracle import equil as OE
from oracle import project as OPJ
from oracle import prox as OP
from tests import test_oracle_admm as TA
from tests import test_oracle_equil_project as TE
from tests import test_oracle_prox as TP


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_dropped_shift_in_parametric_prox(monkeypatch):
    orig = OP.prox_f

    def bad(params, v, rho):   # forgets to add b back: y = z / a
        return orig(params, v, rho) - np.asarray(params.b, float) / np.asarray(params.a, float)
    monkeypatch.setattr(OP, "prox_f", bad)
    _fails(TP.test_parametric_prox_vs_bruteforce, OP.SQUARE)


def test_wrong_huber_threshold(monkeypatch):
    orig = OP.prox_h

    def bad(h, v, rho):
        if h == OP.HUBER:
            v = np.asarray(v, float)
            rho = np.broadcast_to(np.asarray(rho, float), v.shape)
            return np.where(np.abs(v) <= 1.0, rho * v / (1 + rho), v - np.sign(v) / rho)
        return orig(h, v, rho)
    monkeypatch.setattr(OP, "prox_h", bad)
    _fails(TP.test_parametric_prox_vs_bruteforce, OP.HUBER)


def test_wrong_hinge_side(monkeypatch):
    orig = OP.prox_h

    def bad(h, v, rho):
        if h == OP.HINGE:
            return orig(OP.MAXPOS, v, rho)
        return orig(h, v, rho)
    monkeypatch.setattr(OP, "prox_h", bad)
    _fails(TP.test_prox_output_is_fenchel_feasible, OP.HINGE)


def test_swapped_sk_regularizer(monkeypatch):
    def bad(A, sweeps, gamma):
        A = np.asarray(A, float)
        m, n = A.shape
        A2, e = A * A, np.ones(n)
        for _ in range(sweeps):
            d = n / (A2 @ e + gamma / n)
            e = m / (A2.T @ d + gamma / m)
        return d, e
    monkeypatch.setattr(OE, "sinkhorn_knopp", bad)
    _fails(TE.test_sk_optimality_conditions_at_convergence, (30, 12))


def test_paper_sign_of_fat_update(monkeypatch):
    orig_call = OPJ.Projector.__call__

    def bad(self, c, d):
        x, y = orig_call(self, c, d)
        if not self.tall:
            x = np.asarray(c, float) - self.A.T @ (np.asarray(d, float) - y)
        return x, y
    monkeypatch.setattr(OPJ.Projector, "__call__", bad)
    _fails(TE.test_reduced_updates_match_kkt, (5, 12))


def test_transposed_projection_operand(monkeypatch):
    def bad_init(self, A):
        self.A = np.asarray(A, float)
        m, n = self.A.shape
        self.tall = m >= n
        G = self.A @ self.A.T if self.tall else self.A.T @ self.A   # wrong Gram
        G = G[: min(m, n), : min(m, n)] + np.eye(min(m, n))
        self.L = np.linalg.cholesky(G)
    monkeypatch.setattr(OPJ.Projector, "__init__", bad_init)
    _fails(TE.test_reduced_updates_match_kkt, (12, 5))


def test_skewed_projection_breaks_dual_invariant(monkeypatch):
    """A projection that is slightly off the graph breaks x~ + A^T y~ = 0 (Section 3.3)."""
    orig_proj = OPJ.Projector.__call__

    def skewed(self, c, d):
        x, y = orig_proj(self, c, d)
        return x * (1 + 1e-3), y
    monkeypatch.setattr(OPJ.Projector, "__call__", skewed)
    _fails(TA.test_dual_feasibility_invariant_every_iteration)


def test_relaxed_half_step_in_duals_breaks_fenchel_pin(monkeypatch):
    """Using the relaxed point in the prox output (a plausible slip) breaks Fenchel feasibility."""
    orig = OP.prox_f

    def bad(params, v, rho):
        return 1.7 * orig(params, v, rho) - 0.7 * np.asarray(v, float)
    monkeypatch.setattr(OP, "prox_f", bad)
    _fails(TP.test_prox_output_is_fenchel_feasible, OP.ABS)


# ---- adaptive penalty (Section 4.3), rescale (Section 3.2) and stopping test (Section 3.4) ----

from oracle import admm as OA  # noqa: E402
from tests import test_oracle_penalty as TR  # noqa: E402


def test_dropped_rescale_on_rho_change(monkeypatch):
    monkeypatch.setattr(OA, "rescale_scaled_duals", lambda xt, yt, r0, r1: (xt, yt))
    _fails(TR.test_rescale_on_rho_change_matches_unscaled_duals, "lasso", (80, 30), 4)


def test_inverted_rescale_on_rho_change(monkeypatch):
    monkeypatch.setattr(OA, "rescale_scaled_duals", lambda xt, yt, r0, r1: (xt * (r1 / r0), yt * (r1 / r0)))
    _fails(TR.test_rescale_on_rho_change_matches_unscaled_duals, "lasso", (80, 30), 4)


def _planted_controller(monkeypatch, rule):
    def next_rho(self, k, rho, dual_small, primal_small):
        return rule(self, k, rho, dual_small, primal_small)
    monkeypatch.setattr(OA.PenaltyController, "next_rho", next_rho)


def test_delta_applied_in_the_wrong_direction(monkeypatch):
    def rule(self, k, rho, dual_small, primal_small):   # small dual residual lowers rho
        if dual_small and self.tau * k > self.k_last_decrease:
            self.k_last_increase = k
            return rho / self.delta
        if primal_small and self.tau * k > self.k_last_increase:
            self.k_last_decrease = k
            return rho * self.delta
        return rho
    _planted_controller(monkeypatch, rule)
    _fails(TR.test_penalty_controller_hand_worked_sequence)


def test_primal_case_tested_first(monkeypatch):
    def rule(self, k, rho, dual_small, primal_small):
        if primal_small and self.tau * k > self.k_last_increase:
            self.k_last_decrease = k
            return rho / self.delta
        if dual_small and self.tau * k > self.k_last_decrease:
            self.k_last_increase = k
            return rho * self.delta
        return rho
    _planted_controller(monkeypatch, rule)
    _fails(TR.test_penalty_controller_hand_worked_sequence)


def test_non_strict_hysteresis(monkeypatch):
    def rule(self, k, rho, dual_small, primal_small):
        if dual_small and self.tau * k >= self.k_last_decrease:
            self.k_last_increase = k
            return rho * self.delta
        if primal_small and self.tau * k >= self.k_last_increase:
            self.k_last_decrease = k
            return rho / self.delta
        return rho
    _planted_controller(monkeypatch, rule)
    _fails(TR.test_penalty_controller_hand_worked_sequence)


def test_hysteresis_against_the_same_direction(monkeypatch):
    def rule(self, k, rho, dual_small, primal_small):   # waits on its own last change instead
        if dual_small and self.tau * k > self.k_last_increase:
            self.k_last_increase = k
            return rho * self.delta
        if primal_small and self.tau * k > self.k_last_decrease:
            self.k_last_decrease = k
            return rho / self.delta
        return rho
    _planted_controller(monkeypatch, rule)
    _fails(TR.test_penalty_controller_hand_worked_sequence)


def _planted_tolerances(monkeypatch, eps_pri_of, eps_dual_of):
    orig = OA.section34_test

    def bad(p, Ah, fh, gh, xh, yh, mu, nu):
        st = orig(p, Ah, fh, gh, xh, yh, mu, nu)
        v = dict(x=xh, y=yh, mu=mu, nu=nu)
        st.eps_pri = p.abs_tol + p.rel_tol * float(np.linalg.norm(v[eps_pri_of]))
        st.eps_dual = p.abs_tol + p.rel_tol * float(np.linalg.norm(v[eps_dual_of]))
        return st
    monkeypatch.setattr(OA, "section34_test", bad)


def test_dual_tolerance_on_nu(monkeypatch):
    _planted_tolerances(monkeypatch, "y", "nu")
    _fails(TR.test_stop_iteration_is_the_first_meeting_section34, "huber", (60, 25), 2, False)


def test_primal_tolerance_on_x(monkeypatch):
    _planted_tolerances(monkeypatch, "x", "mu")
    _fails(TR.test_stop_iteration_is_the_first_meeting_section34, "nnls", (25, 60), 0, False)


def test_gap_test_dropped(monkeypatch):
    monkeypatch.setattr(OA.StopTest, "converged",
                        lambda self, gap_stop: self.r_pri < self.eps_pri and self.r_dual < self.eps_dual)
    _fails(TR.test_stop_iteration_is_the_first_meeting_section34, "lasso", (200, 100), 0, True)
