"""One-shot optimisation (Sec. 3.3) and threshold scan (Sec. 3.2) on the GPU
against the FP64 oracle.

Cases: the 2D channel (dissipation, minimised), a short 3D exchanger (BGK +
D3Q7, heat flux maximised) and a short 3D mixer (MRT + 2 x D3Q7, outlet
variance minimised, whose adjoint source needs the outlet mean of every
iterate).  theta starts in [0.3, 0.7] on the design box and zeta keeps it
away from the clamps, so both sides take the same path.

Tolerances.  Each iteration's gradient estimate carries the FP32 error of one
primal and one adjoint step (about 1e-5 relative per step, accumulated over
the iterations the flow and the adjoint remember); the design change
theta^K - theta^0 is the sum of those estimates, so it is compared at 1e-3
of its largest entry, and the last estimate g and the adjoint iterate at
1e-3 of their largest entries; J at 1e-4 relative (the gate of the unsteady
objective).  Design decisions (clamps, thresholds) are bit-exact.
"""
import numpy as np
import pytest
import torch

from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs
from paper_1501_04741_gb300.albm import AlbmError, Solver
from paper_1501_04741_gb300.optimize import one_shot

pytestmark = pytest.mark.gpu


def _band(P, seed, lo=0.3, hi=0.7):
    th = inputs.theta_uniform(P, seed)
    return np.where(inputs.design_mask(P), lo + (hi - lo) * th, 0.0).astype(np.float32)


# name: (problem, iterations, zeta, penalty, maximise)
CASES = {
    "channel2d_dissipation": (inputs.channel2d(dims=(40, 21, 1), design=(10, 30, 4, 17, 0, 1),
                                               force=(1e-4, 0, 0), nsteps=40), 60, 250.0, 4e-6, False),
    "exchanger3d_heatflux": (inputs.scaled(inputs.exchanger3d(), (24, 10, 9), nsteps=40), 60, 5.0,
                             2e-4, True),
    "mixer3d_variance": (inputs.scaled(inputs.mixer3d(), (10, 11, 10), nsteps=40, obj_window=1),
                         300, 0.3, 3e-3, False),
}


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    P, K, zeta, pen, mx = CASES[request.param]
    th0 = _band(P, 0)
    mask = inputs.design_mask(P)
    o = Oracle(P, th0)
    thK, FK, vK, gK = o.oneshot(K, zeta, penalty=pen, maximize=mx, design=mask)
    with Solver(P, torch.from_numpy(th0.reshape(-1)).cuda()) as s:
        s.set_design(mask)
        s.oneshot_reset()
        s.oneshot_step(K, zeta, pen, mx)
        J, Pv = s.oneshot_eval()
        gpu = dict(theta=_np(s.theta()), f=_np(s.populations(0)), v=_np(s.adjoint()),
                   g=_np(s.gradient()), J=J, P=Pv)
    ora = dict(theta=thK.numpy().reshape(-1), f=FK.reshape(o.model.M, -1).numpy(),
               v=vK.reshape(o.model.M, -1).numpy(), g=gK.numpy().reshape(-1),
               J=float(o.F_obj(FK)), P=o.penalty(thK.numpy(), mask))
    return request.param, P, th0.reshape(-1), mask.reshape(-1), gpu, ora


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_design_trajectory(case):
    name, P, th0, mask, gpu, ora = case
    d_gpu, d_ora = gpu["theta"] - th0, ora["theta"] - th0
    assert np.abs(d_ora).max() > 1e-3, "the case must move the design"
    assert _rel(d_gpu, d_ora) <= 1e-3, (name, _rel(d_gpu, d_ora))
    assert np.array_equal(gpu["theta"][~mask], th0[~mask].astype(np.float64))
    assert gpu["theta"].min() >= 0.0 and gpu["theta"].max() <= 1.0


def test_state_adjoint_and_gradient_estimate(case):
    name, P, th0, mask, gpu, ora = case
    assert _rel(gpu["f"], ora["f"]) <= 1e-5, (name, _rel(gpu["f"], ora["f"]))
    assert _rel(gpu["v"], ora["v"]) <= 1e-3, (name, _rel(gpu["v"], ora["v"]))
    assert _rel(gpu["g"], ora["g"]) <= 1e-3, (name, _rel(gpu["g"], ora["g"]))


def test_objective_and_penalty(case):
    name, P, th0, mask, gpu, ora = case
    assert abs(gpu["J"] - ora["J"]) <= 1e-4 * abs(ora["J"]), (name, gpu["J"], ora["J"])
    assert abs(gpu["P"] - ora["P"]) <= 1e-4 * abs(ora["P"]), (name, gpu["P"], ora["P"])


def test_penalty_alone_closed_form():
    P = inputs.channel2d(dims=(64, 21, 1), design=(10, 50, 4, 17, 0, 1), objective="none")
    mask = inputs.design_mask(P).reshape(-1)
    th0 = np.where(mask, _band(P, 5).reshape(-1), np.float32(0.2)).astype(np.float32)
    zeta, pen, K = 0.01, 2.0, 8
    with Solver(P, torch.from_numpy(th0).cuda()) as s:
        s.set_design(mask)
        s.oneshot_reset()
        s.oneshot_step(K, zeta, pen, True)
        th = _np(s.theta())
        _, Pv = s.oneshot_eval()
    want = 0.5 + (th0.astype(np.float64) - 0.5) * (1 + 2 * zeta * pen) ** K
    # FP32 storage of theta after each of the K updates
    assert np.abs(th[mask] - want[mask]).max() <= 1e-6
    assert np.array_equal(th[~mask], th0[~mask].astype(np.float64))
    assert abs(Pv - float((want[mask] * (1 - want[mask])).sum())) <= 1e-5 * Pv


def test_clamps_are_exact():
    """A large step drives every design node to a clamp after one update;
    which clamp is decided by the sign of the step, far from zero."""
    P, K, zeta, pen, mx = CASES["exchanger3d_heatflux"]
    th0 = _band(P, 2, 0.05, 0.95)
    mask = inputs.design_mask(P)
    with Solver(P, torch.from_numpy(th0.reshape(-1)).cuda()) as s:
        s.set_design(mask)
        s.oneshot_reset()
        s.oneshot_step(3, 10.0, 10.0, mx)      # penalty dominates: 10*10*(1-2 theta)
        th = _np(s.theta()).reshape(mask.shape)
    want, *_ = Oracle(P, th0).oneshot(3, 10.0, penalty=10.0, maximize=mx, design=mask)
    assert np.array_equal(th[mask], want.numpy()[mask])
    assert set(np.unique(th[mask])) <= {0.0, 1.0}


@pytest.mark.parametrize("name", ["channel2d_dissipation", "exchanger3d_heatflux"])
def test_threshold_scan(name):
    P = CASES[name][0]
    th0 = _band(P, 1, 0.0, 1.0)
    mask = inputs.design_mask(P)
    etas = [0.0, 0.3, 0.5, 0.7, 1.01]
    nsteps = 40
    o = Oracle(P, th0)
    want = o.threshold_scan(th0, etas, nsteps, mask)
    with Solver(P, torch.from_numpy(th0.reshape(-1)).cuda()) as s:
        s.set_design(mask)
        got = s.threshold_scan(etas, nsteps)
        assert np.array_equal(_np(s.theta()), th0.reshape(-1).astype(np.float64))  # restored
        s.threshold_apply(0.5)
        th_bin = _np(s.theta())
    for e, a, b in zip(etas, got, want):
        assert abs(a - b) <= 1e-4 * max(abs(b), 1e-12), (name, e, a, b)
    assert np.array_equal(th_bin, Oracle.threshold(th0, 0.5, mask).reshape(-1).astype(np.float64))


def test_modes_are_exclusive():
    P = CASES["channel2d_dissipation"][0]
    th0 = _band(P, 0)
    with Solver(P, torch.from_numpy(th0.reshape(-1)).cuda()) as s:
        with pytest.raises(AlbmError, match="LBM_ERR_STATE"):
            s.oneshot_step(1, 1.0)                     # not started
        s.oneshot_reset()
        s.oneshot_step(2, 1.0)
        with pytest.raises(AlbmError, match="LBM_ERR_STATE"):
            s.primal_step(1)
        with pytest.raises(AlbmError, match="LBM_ERR_ARG"):
            s.oneshot_step(1, -1.0)
        s.reset()                                      # back to the unsteady mode
        s.primal_step(1)


def test_driver_runs_schedule_and_scan():
    P, K, zeta, pen, mx = CASES["exchanger3d_heatflux"]
    th0 = _band(P, 0)
    mask = inputs.design_mask(P)
    r = one_shot(P, th0, 120, zeta, maximize=mx, penalty0=pen, penalty_growth=2.0, chunk=40,
                 design=mask, etas=[0.2, 0.5, 0.8], eval_steps=40)
    assert [h[0] for h in r.history] == [40, 80, 120]
    assert [h[3] for h in r.history] == [pen, 2 * pen, 4 * pen]
    assert r.best_J == max(r.scan)
    # the applied design follows the threshold rule on the library's own theta
    m = mask.reshape(-1)
    solid = (np.float32(1.0) - r.theta) < np.float32(r.best_eta)
    want = np.where(m, np.where(solid, np.float32(1.0), np.float32(0.0)), r.theta)
    assert np.array_equal(r.theta_binary, want)


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_oneshot_with_16bit_storage(precision):
    """The one-shot iteration with 16-bit states (even nx: the paired primal
    kernel, and for the variance objective its per-step outlet mean) follows
    the FP32 run: design change within the reduced-precision bounds of the
    unsteady solve (gradients 0.6 BF16 / 0.1 FP16 relative), J within 1e-1 /
    1e-2."""
    P, K, zeta, pen, mx = CASES["mixer3d_variance"]
    P = P.replace(dims=(10, 11, 10))
    th0 = _band(P, 0)
    mask = inputs.design_mask(P)
    out = {}
    for prec in ("fp32", precision):
        with Solver(P.replace(precision=prec), torch.from_numpy(th0.reshape(-1)).cuda()) as s:
            s.set_design(mask)
            s.oneshot_reset()
            s.oneshot_step(K, zeta, pen, mx)
            J, Pv = s.oneshot_eval()
            out[prec] = (_np(s.theta()) - th0.reshape(-1), J)
    d32, J32 = out["fp32"]
    d16, J16 = out[precision]
    gb, jb = (0.6, 1e-1) if precision == "bf16" else (0.1, 1e-2)
    assert np.isfinite(d16).all() and np.isfinite(J16)
    assert _rel(d16, d32) <= gb, _rel(d16, d32)
    assert abs(J16 - J32) <= jb * abs(J32), (J16, J32)
