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
