"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin
fails for each: evidence that the pins constrain the oracle and not just
restate it."""
import numpy as np
import pytest
import torch

import oracle.model as om
from paper_1501_04741_gb300 import inputs
from tests import test_oracle_lattice as TL
from tests import test_oracle_physics as TP


def _mutate(monkeypatch, name, fn):
    monkeypatch.setattr(om.Model, name, fn)


def test_dropped_exact_difference_term_is_caught(monkeypatch):
    orig = om.Model.collide

    def bad(self, F, theta, flags, y):
        saved = self.g.clone()
        self.g = torch.zeros_like(saved)     # force dropped from u_post
        try:
            return orig(self, F, theta, flags, y)
        finally:
            self.g = saved
    _mutate(monkeypatch, "collide", bad)
    with pytest.raises(AssertionError):
        TP.test_body_force_momentum_growth_is_exact()


def test_wrong_porosity_switch_is_caught(monkeypatch):
    _mutate(monkeypatch, "G", lambda self, theta: theta)   # G(theta) = theta, inverted roles
    with pytest.raises(AssertionError):
        TP.test_porosity_limits()


def test_wrong_zou_he_transverse_sign_is_caught(monkeypatch):
    orig = om.Model.zou_he

    def bad(self, f, inward, u_n=None, rho=None):
        fr, r, u = orig(self, f, inward, u_n=u_n, rho=rho)
        # flip the transverse correction of the diagonal unknowns
        E = self.fl.E
        zero = np.nonzero(E[:, 0] * inward == 0)[0]
        rows = [fr[i] for i in range(self.Q)]
        for i in np.nonzero(E[:, 0] * inward > 0)[0]:
            for t in (1, 2):
                if E[i, t] != 0:
                    et = torch.tensor(E[zero, t], dtype=torch.float64)
                    Nt = 0.5 * (et[:, None] * f[zero]).sum(0)
                    rows[i] = rows[i] + 2 * float(E[i, t]) * Nt
        return torch.stack(rows), r, u
    _mutate(monkeypatch, "zou_he", bad)
    with pytest.raises(AssertionError):
        TP.test_zou_he_prescribed_values_after_collision()


def test_wrong_equilibrium_coefficient_is_caught(monkeypatch):
    def bad(self, rho, u):
        cs2 = self.fl.cs2
        eu = self.E @ u
        uu = (u * u).sum(0)
        return self.w[:, None] * rho * (1 + eu / cs2 + eu * eu / (2 * cs2) - uu / (2 * cs2))
    _mutate(monkeypatch, "feq", bad)
    # MRT and BGK share the equilibrium, so their agreement cannot see this;
    # the equilibrium no longer carries the node's mass, which the
    # conservation pin of the collision does
    TL.test_mrt_with_T_equal_omega_is_bgk("D2Q9")
    with pytest.raises(AssertionError):
        TL.test_collision_conserves_mass_and_forced_momentum("BGK", "D2Q9")


def test_missing_dissipation_factor_is_caught(monkeypatch):
    orig = om.Model.objective

    def bad(self, F, theta, flags, y, n_inlet=1, n_outlet=1):
        return 0.5 * orig(self, F, theta, flags, y, n_inlet, n_outlet)
    _mutate(monkeypatch, "objective", bad)
    with pytest.raises(AssertionError):
        TP.test_dissipation_objective_closed_form()


def test_scalar_using_pre_collision_velocity_is_caught(monkeypatch):
    orig = om.Model.macroscopic

    def bad(self, F, theta, flags):
        m = orig(self, F, theta, flags)
        m["v"] = m["u"]          # scalar and outlet terms see u_pre, not u_post
        return m
    _mutate(monkeypatch, "macroscopic", bad)
    with pytest.raises(AssertionError):
        TL.test_collision_conserves_mass_and_forced_momentum("BGK", "D2Q9")


# ---- one-shot optimisation (Sec. 3.3) -----------------------------------------
def _oneshot_pins():
    from tests import test_oracle_oneshot as TO
    return TO


def _converged_case(TO):
    from oracle.solver import Oracle
    P = TO._channel()
    th0 = TO._theta_band(P, 0)
    mask = inputs.design_mask(P)
    o = Oracle(P, th0)
    K = 400
    th, F, v, g = o.oneshot(K, 0.0, design=mask)
    return P, th0, mask, o, K, th, F, v, g


def test_penalty_pushing_away_from_binary_is_caught(monkeypatch):
    from oracle.solver import Oracle
    TO = _oneshot_pins()

    def bad(th, g, zeta, penalty, s, mask):
        d = s * g + penalty * (1.0 - 2.0 * th)          # sign of dP/dtheta flipped
        return torch.where(mask, torch.clamp(th + zeta * d, 0.0, 1.0), th)
    monkeypatch.setattr(Oracle, "design_update", staticmethod(bad))
    with pytest.raises(AssertionError):
        TO.test_penalty_alone_follows_closed_form()


def test_update_outside_the_design_mask_is_caught(monkeypatch):
    from oracle.solver import Oracle
    TO = _oneshot_pins()

    def bad(th, g, zeta, penalty, s, mask):
        d = s * g - penalty * (1.0 - 2.0 * th)
        return torch.clamp(th + zeta * d, 0.0, 1.0)     # mask ignored
    monkeypatch.setattr(Oracle, "design_update", staticmethod(bad))
    with pytest.raises(AssertionError):
        TO.test_penalty_alone_follows_closed_form()


def test_descending_when_maximising_is_caught(monkeypatch):
    from oracle.solver import Oracle
    TO = _oneshot_pins()
    case = _converged_case(TO)

    def bad(th, g, zeta, penalty, s, mask):
        d = -s * g - penalty * (1.0 - 2.0 * th)         # step against the objective
        return torch.where(mask, torch.clamp(th + zeta * d, 0.0, 1.0), th)
    monkeypatch.setattr(Oracle, "design_update", staticmethod(bad))
    with pytest.raises(AssertionError):
        TO.test_one_update_moves_the_objective_by_zeta_g_squared(case, True)


def test_gradient_without_the_adjoint_is_caught(monkeypatch):
    """A gradient estimate that leaves out the adjoint weights (only the
    direct dF/dtheta, zero for these objectives) fails the FD pin."""
    from oracle.solver import Oracle
    TO = _oneshot_pins()
    orig = Oracle.adjoint_step

    def bad(self, lam_next, F):
        gF, gth = orig(self, lam_next, F)
        return gF, torch.zeros_like(gth)
    monkeypatch.setattr(Oracle, "adjoint_step", bad)
    case = _converged_case(TO)
    with pytest.raises(AssertionError):
        TO.test_zero_step_estimate_is_the_steady_gradient(case)


def test_threshold_tie_to_solid_is_caught(monkeypatch):
    from oracle.solver import Oracle
    TO = _oneshot_pins()

    def bad(theta, eta, design=None):
        th = np.asarray(theta, dtype=np.float32).reshape(-1)
        mask = np.ones(th.shape, bool) if design is None else np.asarray(design).reshape(-1).astype(bool)
        w = np.float32(1.0) - th
        out = th.copy()
        out[mask] = np.where(w[mask] <= np.float32(eta), 1.0, 0.0)   # tie goes solid
        return out.reshape(np.shape(theta))
    monkeypatch.setattr(Oracle, "threshold", staticmethod(bad))
    with pytest.raises(AssertionError):
        TO.test_threshold_rule()


# ---- MMA (Sec. 3.3, oracle.mma) --------------------------------------------
def test_mma_swapped_approximation_terms_are_caught(monkeypatch):
    from oracle import mma as M
    from tests import test_oracle_mma as TM
    orig = M.subproblem

    def bad(x, g, L, U, prm=M.MMAParams()):
        return orig(x, -np.asarray(g), L, U, prm)       # p and q exchanged
    monkeypatch.setattr(M, "subproblem", bad)
    with pytest.raises(AssertionError):
        TM.test_approximation_is_first_order_exact_and_convex()


def test_mma_inverted_oscillation_rule_is_caught(monkeypatch):
    import dataclasses

    from oracle import mma as M
    from tests import test_oracle_mma as TM
    orig = M.MMAParams
    # asymptotes farther when a variable oscillates, closer when it does not
    monkeypatch.setattr(M, "MMAParams", lambda: dataclasses.replace(orig(), s_dec=1.2, s_inc=0.7))
    with pytest.raises(AssertionError):
        TM.test_converges_on_a_separable_quadratic()


def test_mma_closed_form_with_swapped_asymptotes_is_caught(monkeypatch):
    from oracle import mma as M
    from tests import test_oracle_mma as TM
    orig = M.subproblem

    def bad(x, g, L, U, prm=M.MMAParams()):
        y, aux = orig(x, g, L, U, prm)
        alpha, beta, p, q = aux
        sp, sq = np.sqrt(p), np.sqrt(q)
        y = np.clip((sp * U + sq * L) / (sp + sq), alpha, beta)
        return y, aux
    monkeypatch.setattr(M, "subproblem", bad)
    with pytest.raises(AssertionError):
        TM.test_subproblem_minimiser_matches_grid_search()


def test_wrong_power_law_exponent_is_caught(monkeypatch):
    orig = om.Model.G

    def bad(self, theta):
        if self.P.porosity == "power":
            return 1 - theta ** (self.P.porosity_q - 1)
        return orig(self, theta)
    _mutate(monkeypatch, "G", bad)
    with pytest.raises(AssertionError):
        TP.test_porosity_law_at_intermediate_theta("power", 3.0, 0.6)


def test_swapped_diffusivity_interpolation_is_caught(monkeypatch):
    _mutate(monkeypatch, "alpha",
            lambda self, theta: theta * self.P.alpha_fluid + (1 - theta) * self.P.alpha_solid)
    with pytest.raises(AssertionError):
        TP.test_scalar_diffusivity_interpolates_in_theta(0.3)


def test_inverted_signed_inlet_is_caught(monkeypatch):
    orig = om.Model.inlet_scalar

    def bad(self, s, y):
        c = orig(self, s, y)
        return -c if self.P.scalar_inlet == "signed" else c     # -1 above, +1 below
    _mutate(monkeypatch, "inlet_scalar", bad)
    with pytest.raises(AssertionError):
        TP.test_signed_inlet_values_after_collision()


def test_heat_flux_with_the_pressure_term_is_caught(monkeypatch):
    orig = om.Model.objective

    def bad(self, F, theta, flags, y, n_inlet=1, n_outlet=1):
        if self.P.objective == "heatflux":                     # pressure term kept
            saved = self.P
            self.P = saved.replace(objective="heatflux_dp")
            try:
                return orig(self, F, theta, flags, y, n_inlet, n_outlet)
            finally:
                self.P = saved
        return orig(self, F, theta, flags, y, n_inlet, n_outlet)
    _mutate(monkeypatch, "objective", bad)
    with pytest.raises(AssertionError):
        TP.test_heat_flux_pressure_drop_term()


def _window_weights(extra: int, scale_extra: int):
    """Window weights with `extra` more terms and weight 1/(K + scale_extra)."""
    def weights_for(N, K):
        c = np.zeros(N + 1)
        if K <= 0:
            c[N] = 1.0
        else:
            c[max(N - K + 1 - extra, 0):] = 1.0 / (K + scale_extra)
        return c
    return weights_for


@pytest.mark.parametrize("extra,scale_extra", [(1, 0), (0, 1), (1, 1)])
def test_window_off_by_one_is_caught(monkeypatch, extra, scale_extra):
    import oracle.solver as osv
    wf = _window_weights(extra, scale_extra)
    monkeypatch.setattr(om.Model, "weights",
                        lambda self: wf(int(self.P.nsteps), int(self.P.obj_window)))
    with pytest.raises(AssertionError):
        TP.test_window_objective_is_the_mean_of_the_last_K_steps("D2Q9", (6, 5, 1), 7, 3)
    monkeypatch.undo()
    monkeypatch.setattr(osv, "_weights", lambda P, N: wf(N, int(P.obj_window)))
    with pytest.raises(AssertionError):
        TP.test_window_objective_is_the_mean_of_the_last_K_steps("D3Q19", (4, 3, 5), 7, 3)


def test_outlet_scalar_taken_as_plain_sum_is_caught(monkeypatch):
    def naive(self, g, v):
        return g, g.sum(0)             # T* = sum g, unknowns left as they came in
    _mutate(monkeypatch, "scalar_outlet", naive)
    for lat in ("D2Q9", "D3Q19"):
        with pytest.raises(AssertionError):
            TP.test_outlet_scalar_reconstruction_worked_example(lat)


def test_outlet_scalar_with_pre_collision_sign_is_caught(monkeypatch):
    # unknowns at equilibrium with the velocity reversed (e.v taken with the
    # outward instead of the streaming direction)
    orig = om.Model.scalar_outlet

    def bad(self, g, v):
        return orig(self, g, -v)
    _mutate(monkeypatch, "scalar_outlet", bad)
    for lat in ("D2Q9", "D3Q19"):
        with pytest.raises(AssertionError):
            TP.test_outlet_scalar_reconstruction_worked_example(lat)


def test_pressure_inlet_without_the_cap_is_caught(monkeypatch):
    def uncapped(self, f):
        return self.zou_he(f, +1, rho=self.P.rho_out + self.P.dp / self.fl.cs2)[0]
    _mutate(monkeypatch, "inlet", uncapped)
    with pytest.raises(AssertionError):
        TP.test_pressure_inlet_prescribed_values("D3Q19")


def test_pressure_inlet_density_without_cs2_is_caught(monkeypatch):
    orig = om.Model.inlet

    def bad(self, f):
        saved = self.P
        self.P = saved.replace(dp=saved.dp / 3.0)       # rho_in = rho_out + dp
        try:
            return orig(self, f)
        finally:
            self.P = saved
    _mutate(monkeypatch, "inlet", bad)
    with pytest.raises(AssertionError):
        TP.test_pressure_inlet_prescribed_values("D2Q9")
