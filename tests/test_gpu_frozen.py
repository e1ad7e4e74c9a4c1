"""The paper's fixed-point adjoint (ALBS at a held state, Sec. 2.2) on the GPU
against the FP64 oracle's ``frozen_adjoint``.

Convention of the library (adjoint_mode 1): iteration k consumes v^{k-1},
writes v^k = (d(SW)/df(f-hat))^T v^{k-1} + dF/df(f-hat) and the gradient
estimate of Eq. adjoint:derivative from v^{k-1}.  The oracle's
frozen_adjoint(F, k) returns v^k and the gradient from v^k, so after k GPU
iterations lambda is compared with frozen_adjoint(F, k) and dJ/dtheta with
frozen_adjoint(F, k - 1).  Bars: 1e-4 relative (inf-norm), the gradient bar
of the unsteady parity tests; the oracle's ALBS is pinned against finite
differences of the steady objective (tests/test_oracle_adjoint.py).
"""
import numpy as np
import pytest
import torch

from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs

pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _solver(P, theta, **kw):
    from paper_1501_04741_gb300.albm import Solver
    return Solver(P, torch.from_numpy(np.asarray(theta, np.float32).reshape(-1)).cuda(), **kw)


def _frozen_on_state(P, th, F, iters):
    """GPU: set the state, run `iters` ALBS iterations at it."""
    M = F.shape[0]
    with _solver(P.replace(adjoint_mode="frozen", obj_window=0, nsteps=0), th) as s:
        s.set_populations(torch.tensor(F.reshape(M, -1).numpy(), dtype=torch.float32,
                                       device="cuda"))
        s.adjoint_step(iters)
        return _np(s.adjoint()), _np(s.gradient())


def _check(lam_gpu, g_gpu, o, F, iters):
    _, v = o.frozen_adjoint(F, iters)
    g_prev, _ = o.frozen_adjoint(F, iters - 1)
    v = v.reshape(o.model.M, -1).numpy()
    g_prev = g_prev.reshape(-1).numpy()
    assert np.abs(lam_gpu - v).max() <= 1e-4 * np.abs(v).max(), np.abs(lam_gpu - v).max()
    assert np.abs(g_gpu - g_prev).max() <= 1e-4 * np.abs(g_prev).max(), \
        np.abs(g_gpu - g_prev).max() / np.abs(g_prev).max()


def test_frozen_albs_at_a_converged_channel():
    # D2Q9 BGK channel converged to its steady state (the oracle's pinned
    # case): 3000 ALBS iterations at the FP32-rounded fixed point
    P = inputs.channel2d(dims=(12, 8, 1), design=(3, 9, 2, 6, 0, 1), force=(1e-4, 0, 0),
                         tau=0.8)
    th = inputs.theta_uniform(P, 5) * np.float32(0.5)
    o = Oracle(P, th)
    _, traj = o.primal(nsteps=3000, keep=False)
    F = traj[-1].to(torch.float32).to(torch.float64)
    lam, g = _frozen_on_state(P, th, F, 3000)
    _check(lam, g, o, F, 3000)


@pytest.mark.parametrize("name", ["mixer_mrt_variance", "exchanger_bgk_heatflux_dp",
                                  "paper_mixer_mixflux"])
def test_frozen_albs_on_3d_states(name):
    # a transient state (the primal after a few steps) of the 3D physics:
    # MRT fluid with two scalars and the outlet variance, BGK with the heat
    # flux and the pressure drop, the paper's signed mixer with its flux
    base = {"mixer_mrt_variance": inputs.scaled(inputs.mixer3d(), (21, 11, 10), nsteps=30,
                                                obj_window=0),
            "exchanger_bgk_heatflux_dp": inputs.scaled(inputs.exchanger3d(), (23, 10, 9),
                                                       nsteps=30),
            "paper_mixer_mixflux": inputs.scaled(inputs.paper_mixer_empty(), (23, 10, 10),
                                                 nsteps=30)}[name]
    th = inputs.theta_uniform(base, 3)
    o = Oracle(base, th)
    _, traj = o.primal(keep=False)
    F = traj[-1].to(torch.float32).to(torch.float64)
    lam, g = _frozen_on_state(base, th, F, 25)
    _check(lam, g, o, F, 25)


def test_frozen_run_follows_the_primal_then_the_same_number_of_iterations():
    # lbm_run in adjoint_mode 1: N primal steps from rest, then N ALBS
    # iterations at f^N (the schedule of Sec. 3.3)
    P = inputs.channel2d(dims=(12, 8, 1), design=(3, 9, 2, 6, 0, 1), force=(1e-4, 0, 0),
                         tau=0.8, nsteps=1500)
    th = inputs.theta_uniform(P, 7) * np.float32(0.5)
    o = Oracle(P, th)
    J, traj = o.primal(keep=False)
    g_ref, _ = o.frozen_adjoint(traj[-1], P.nsteps - 1)
    g_ref = g_ref.reshape(-1).numpy()
    with _solver(P.replace(adjoint_mode="frozen"), th) as s:
        s.run()
        J_gpu = s.objective()
        g = _np(s.gradient())
        assert s.time == P.nsteps
    assert abs(J_gpu - J) <= 5e-5 * abs(J)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()


def test_frozen_mode_guards():
    from paper_1501_04741_gb300.albm import AlbmError, Solver, batch_adjoint_step
    P = inputs.channel2d(dims=(12, 8, 1), nsteps=10)
    th = torch.zeros(P.n_nodes, device="cuda")
    with pytest.raises(AlbmError, match="obj_window"):
        Solver(P.replace(adjoint_mode="frozen", obj_window=3), th)
    with Solver(P.replace(adjoint_mode="frozen"), th) as s:
        s.primal_step(10)
        with pytest.raises(AlbmError, match="unsteady"):
            batch_adjoint_step([s], 1)
        s.adjoint_step(4)
        s.adjoint_step(4)                 # iterations continue past the horizon
        assert np.isfinite(_np(s.gradient())).all()
