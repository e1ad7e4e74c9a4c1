"""Pins of the oracle's one-shot optimisation (Sec. 3.3) and threshold (Sec. 3.2).

* penalty alone (no objective, so the adjoint and its gradient vanish): the
  update of Eq. gradient:update with P of Eq. P, theta <- theta - zeta p (1 - 2
  theta), maps u = theta - 1/2 to u (1 + 2 zeta p): a closed form per node;
  nodes outside the design mask never move;
* with zeta = 0 the one-shot iteration is the primal LLBS and the ALBS run side
  by side; once converged, the gradient estimate of Eq. adjoint:derivative is
  the gradient of the steady objective, checked against central finite
  differences of the converged primal (no adjoint code involved);
* one update from a converged state moves the steady objective by
  s zeta |g|^2 to first order (s = +1 maximising, -1 minimising), which fixes
  the sign of the step and the mask it acts on;
* the threshold rule: w = 1 - theta below eta -> solid (theta = 1), else fluid.
"""
import numpy as np
import pytest

from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs


def _channel(**kw):
    base = dict(dims=(16, 8, 1), tau=1.0, force=(1e-4, 0.0, 0.0), design=(4, 12, 2, 6, 0, 1),
                nsteps=10)
    base.update(kw)
    return inputs.channel2d(**base)


def _theta_band(P, seed, lo=0.3, hi=0.7):
    th = inputs.theta_uniform(P, seed)
    return np.where(inputs.design_mask(P), lo + (hi - lo) * th, 0.0).astype(np.float32)


def test_penalty_alone_follows_closed_form():
    P = _channel(dims=(24, 12, 1), design=(6, 18, 2, 10, 0, 1), objective="none")
    mask = inputs.design_mask(P)
    # a porous background outside the design box, which must not move
    th0 = np.where(mask, _theta_band(P, 3), np.float32(0.2)).astype(np.float32)
    o = Oracle(P, th0)
    zeta, p, K = 0.01, 2.0, 8
    th, _, v, g = o.oneshot(K, zeta, penalty=p, design=mask)
    th = th.numpy()
    u0 = th0.astype(np.float64) - 0.5
    want = 0.5 + u0 * (1.0 + 2.0 * zeta * p) ** K
    assert np.abs(th[mask] - want[mask]).max() <= 1e-12
    assert np.array_equal(th[~mask], th0[~mask].astype(np.float64))
    assert float(np.abs(g.numpy()).max()) == 0.0 and float(v.abs().max()) == 0.0
    # P = sum(1/4 - u^2) shrinks by the same factor squared on the u^2 part
    P0, PK = o.penalty(th0, mask), o.penalty(th, mask)
    q = float((u0[mask] ** 2).sum())
    assert abs(PK - (mask.sum() / 4 - q * (1 + 2 * zeta * p) ** (2 * K))) <= 1e-12
    assert PK < P0


def test_penalty_clips_to_binary_values():
    P = _channel(dims=(24, 12, 1), design=(6, 18, 2, 10, 0, 1), objective="none")
    th0 = _theta_band(P, 4, 0.05, 0.95)
    mask = inputs.design_mask(P)
    th, *_ = Oracle(P, th0).oneshot(40, 0.5, penalty=1.0, design=mask)
    th = th.numpy()
    want = np.where(th0 > 0.5, 1.0, 0.0)
    assert np.array_equal(th[mask], want[mask])


@pytest.fixture(scope="module")
def converged():
    P = _channel()
    th0 = _theta_band(P, 0)
    mask = inputs.design_mask(P)
    o = Oracle(P, th0)
    K = 400
    th, F, v, g = o.oneshot(K, 0.0, design=mask)
    return P, th0, mask, o, K, th, F, v, g


def test_zero_step_estimate_is_the_steady_gradient(converged):
    P, th0, mask, o, K, th, F, v, g = converged
    assert np.array_equal(th.numpy(), th0.astype(np.float64))     # zeta = 0: no update
    g = g.numpy().reshape(-1)
    idx = [int(i) for i in np.flatnonzero(mask.reshape(-1))[::7]]
    h = 1e-6
    for i in idx:
        tp = th0.reshape(-1).astype(np.float64).copy()
        tm = tp.copy()
        tp[i] += h
        tm[i] -= h
        fd = (o.steady_objective(K, tp) - o.steady_objective(K, tm)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-5 * np.abs(g).max(), (i, g[i], fd)


@pytest.mark.parametrize("maximize", [True, False])
def test_one_update_moves_the_objective_by_zeta_g_squared(converged, maximize):
    P, th0, mask, o, K, _, F, v, _ = converged
    zeta = 2e2   # theta moves by ~2e-5 (|g| ~ 1e-7)
    th1, _, _, g = o.oneshot(1, zeta, maximize=maximize, design=mask, F0=F, v0=v)
    g = g.numpy()
    s = 1.0 if maximize else -1.0
    assert np.allclose(th1.numpy()[mask] - th0[mask], s * zeta * g[mask], rtol=1e-6, atol=0)
    J0 = o.steady_objective(2 * K, th0)
    J1 = o.steady_objective(2 * K, th1.numpy())
    pred = s * zeta * float((g[mask] ** 2).sum())
    assert abs((J1 - J0) - pred) <= 1e-3 * abs(pred)


def test_threshold_rule():
    th = np.array([0.0, 0.25, 0.5, 0.75, 1.0, 0.6], dtype=np.float32)
    design = np.array([1, 1, 1, 1, 1, 0], dtype=bool)
    # eta = 0.5: w = (1, .75, .5, .25, 0); w < eta -> solid; w == eta -> fluid
    out = Oracle.threshold(th, 0.5, design)
    assert np.array_equal(out, np.array([0, 0, 0, 1, 1, 0.6], dtype=np.float32))
    # eta = 0: nothing below it, all design nodes fluid
    assert np.array_equal(Oracle.threshold(th, 0.0, design)[design], np.zeros(5, np.float32))
    # eta above 1: every design node solid
    assert np.array_equal(Oracle.threshold(th, 1.01, design)[design], np.ones(5, np.float32))
    # the decision is taken on FP32 values: theta = 0.3f gives w = 0.7f - rounding
    th3 = np.array([0.3], dtype=np.float32)
    w3 = np.float32(1.0) - th3[0]
    assert Oracle.threshold(th3, float(w3))[0] == 0.0            # tie -> fluid
    assert Oracle.threshold(th3, float(np.nextafter(w3, np.float32(2))))[0] == 1.0


def test_threshold_scan_matches_binary_runs():
    P = _channel()
    th0 = _theta_band(P, 1, 0.0, 1.0)
    mask = inputs.design_mask(P)
    o = Oracle(P, th0)
    etas = [0.0, 0.5, 1.01]
    Js = o.threshold_scan(th0, etas, 60, mask)
    open_design = np.where(mask, 0.0, th0)
    closed = np.where(mask, 1.0, th0)
    assert Js[0] == o.steady_objective(60, open_design)
    assert Js[2] == o.steady_objective(60, closed)
    # a solid block dissipates less than the open channel under the same force
    assert Js[2] < Js[1] < Js[0]
