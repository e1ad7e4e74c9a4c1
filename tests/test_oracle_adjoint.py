"""Pins of the oracle's adjoint: the one-step duality identity (forward-mode
tangent against reverse-mode adjoint), central finite differences of J on tiny
lattices for every objective and node type, and the paper's fixed-point ALBS
against finite differences of the steady objective (no GPU)."""
import numpy as np
import pytest
import torch

from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs


def _cases():
    ch = inputs.channel2d(dims=(10, 8, 1), design=(3, 8, 2, 6, 0, 1), nsteps=40,
                          force=(1e-4, 0, 0))
    mix = inputs.scaled(inputs.mixer3d(), (10, 6, 6), nsteps=16, obj_window=4)
    exch = inputs.scaled(inputs.exchanger3d(), (12, 6, 6), nsteps=16)
    return {
        "channel2d_bgk": ch,
        "channel2d_mrt": ch.replace(collision="MRT"),
        "channel2d_scalar": ch.replace(nscalars=1, alpha_fluid=0.02, alpha_solid=0.3,
                                       porosity="ramp", porosity_q=2.0),
        "mixer3d_mrt": mix,
        "mixer3d_bgk_mixflux": mix.replace(collision="BGK", objective="mixflux"),
        "exchanger3d_bgk": exch,
        "exchanger3d_mrt_power": exch.replace(collision="MRT", porosity="power",
                                              porosity_q=3.0),
        # the paper's channels: signed inlet with the mixing flux, heat flux alone
        "paper_mixer_signed": inputs.scaled(inputs.paper_mixer_empty(), (10, 6, 6), nsteps=16),
        "paper_exchanger_heatflux": inputs.scaled(inputs.paper_exchanger_empty(), (12, 6, 6),
                                                  nsteps=16),
        # the paper's pressure inlet: above the velocity cap (dp = 0.03 drives
        # the short channel faster than 0.05) and below it
        "exchanger_pressure_capped": inputs.scaled(inputs.paper_exchanger_empty(), (12, 6, 6),
                                                   nsteps=16).replace(inlet="pressure", dp=0.03),
        "exchanger_pressure_open": inputs.scaled(inputs.paper_exchanger_empty(), (12, 6, 6),
                                                 nsteps=16).replace(inlet="pressure", dp=0.004),
    }


CASES = _cases()


def _theta(P, seed):
    th = inputs.theta_uniform(P, seed)
    # put porosity on the boundary nodes too so every node type has a theta path
    rng = np.random.default_rng(seed + 100)
    th = th + (0.3 * rng.random(th.shape)).astype(np.float32) * (th == 0)
    return th.astype(np.float32)


def _state(o, seed):
    rng = np.random.default_rng(seed)
    m = o.model
    F = o.initial().clone()
    F[:m.Q] *= torch.tensor(1 + 0.02 * rng.standard_normal(F[:m.Q].shape))
    if m.NS:
        F[m.Q:] = torch.tensor(0.1 * rng.random(F[m.Q:].shape))
    return F


@pytest.mark.parametrize("name", list(CASES))
def test_one_step_duality(name):
    # <lambda, A df> = <A^T lambda, df> for one step A = d(S W)/df, with A df
    # from forward-mode differentiation and A^T lambda from the adjoint step.
    P = CASES[name]
    o = Oracle(P, _theta(P, 1))
    F = _state(o, 2)
    rng = np.random.default_rng(3)
    lam = torch.tensor(rng.standard_normal(F.shape))
    df = torch.tensor(rng.standard_normal(F.shape))
    dth = torch.tensor(rng.standard_normal(o.n))
    _, tangent = torch.func.jvp(lambda Fv, th: o.step(Fv, th), (F, o.theta), (df, dth))
    lamF, lamth = o.adjoint_step(lam, F)
    lhs = float((lam * tangent).sum())
    rhs = float((lamF * df).sum() + (lamth * dth).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("name", list(CASES))
def test_one_step_adjoint_against_forward_differences(name):
    # The adjoint step against the forward map alone, without any automatic
    # differentiation on the other side: <lambda, (SW(f + h df, theta + h
    # dtheta) - SW(f - h df, theta - h dtheta)) / 2h> is the directional
    # derivative <lambda, A df + B dtheta> up to O(h^2), and must equal
    # <A^T lambda, df> + <B^T lambda, dtheta> from the adjoint step.  A
    # dropped term, a wrong sign or a transposed index in the reverse
    # product fails it.
    P = CASES[name]
    o = Oracle(P, _theta(P, 1))
    F = _state(o, 2)
    rng = np.random.default_rng(13)
    lam = torch.tensor(rng.standard_normal(F.shape))
    df = torch.tensor(rng.standard_normal(F.shape)) * 0.01
    dth = torch.tensor(rng.standard_normal(o.n)) * 0.1
    h = 1e-5
    lamF, lamth = o.adjoint_step(lam, F)
    # the population and the theta directions separately, so that a small
    # theta term cannot hide behind the population term
    for a, b, rhs in ((df, 0 * dth, float((lamF * df).sum())),
                      (0 * df, dth, float((lamth * dth).sum()))):
        with torch.no_grad():
            up = o.step(F + h * a, o.theta + h * b)
            dn = o.step(F - h * a, o.theta - h * b)
        lhs = float((lam * (up - dn)).sum()) / (2 * h)
        assert abs(lhs - rhs) <= 1e-6 * max(abs(rhs), 1e-4), (lhs, rhs)


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_matches_central_differences(name):
    P = CASES[name]
    o = Oracle(P, _theta(P, 4))
    J, g, _ = o.gradient()
    flat = g.reshape(-1).numpy()
    idx = list(np.argsort(-np.abs(flat))[:2])
    # one node of every type present
    fl = o.flags.numpy()
    for t in np.unique(fl):
        idx.append(int(np.nonzero(fl == t)[0][len(np.nonzero(fl == t)[0]) // 2]))
    scale = np.abs(flat).max()
    for i in idx:
        h = 1e-5
        fd = o.fd(int(i), h=h)
        assert abs(fd - flat[i]) <= 1e-6 * scale + 1e-6 * abs(flat[i]), (i, fd, flat[i])


def test_frozen_albs_matches_steady_finite_differences():
    # The paper's ALBS (Eq. adjoint:iteration at the converged f-hat) gives
    # the gradient of the steady objective (Eq. adjoint:derivative).
    P = inputs.channel2d(dims=(12, 8, 1), design=(3, 9, 2, 6, 0, 1), force=(1e-4, 0, 0),
                         tau=0.8)
    th = inputs.theta_uniform(P, 5) * np.float32(0.5)
    nconv = 3000
    o = Oracle(P, th)
    _, traj = o.primal(nsteps=nconv, keep=False)
    F_hat = traj[-1]
    # converged: one more step changes nothing at this precision
    assert float((o.step(F_hat) - F_hat).abs().max()) < 1e-13
    g, _ = o.frozen_adjoint(F_hat, iters=3000)
    flat = g.reshape(-1).numpy()
    scale = np.abs(flat).max()
    for i in list(np.argsort(-np.abs(flat))[:3]):
        fd = o.fd(int(i), h=1e-5, nsteps=nconv)
        assert abs(fd - flat[i]) <= 1e-6 * scale, (i, fd, flat[i])
