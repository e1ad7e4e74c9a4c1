"""Tile-staged kernels (TMA bulk copies of x-row segments into shared memory)
on lattices whose nx is a multiple of the 128-node tile: one step against the
FP64 oracle at the one-step tolerances, whole trajectories against the
one-thread-per-node kernels, and the wrap-around halos at both ends of a row
(nx = 128: one tile spans the row; nx = 384: first, middle and last tiles)."""
import numpy as np
import pytest
import torch

from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "d3q19_mrt_mixer_128": inputs.scaled(inputs.mixer3d(), (128, 12, 10), nsteps=30,
                                             obj_window=6),
        "d3q19_bgk_exchanger_384": inputs.scaled(inputs.exchanger3d(), (384, 10, 9), nsteps=30),
        "d2q9_bgk_scalar_256": inputs.channel2d(dims=(256, 21, 1), design=(60, 200, 4, 17, 0, 1),
                                                nsteps=40, force=(1e-4, 0, 0), nscalars=1,
                                                alpha_fluid=0.02, alpha_solid=0.2),
        "d3q19_mrt_mixer_128_bf16": inputs.scaled(inputs.mixer3d(), (128, 12, 10), nsteps=30,
                                                  obj_window=6, precision="bf16"),
    }


CASES = _cases()


def _theta(P, seed):
    th = inputs.theta_uniform(P, seed)
    rng = np.random.default_rng(seed + 100)
    th = th + (0.3 * rng.random(th.shape)).astype(np.float32) * (th == 0)
    return th.astype(np.float32)


def _solver(P, theta):
    from paper_1501_04741_gb300.albm import Solver
    return Solver(P, torch.from_numpy(theta.reshape(-1)).cuda())


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _random_state(o, seed):
    rng = np.random.default_rng(seed)
    m = o.model
    F = o.initial().clone()
    F[:m.Q] *= torch.tensor(1 + 0.02 * rng.standard_normal(F[:m.Q].shape))
    if m.NS:
        F[m.Q:] = torch.tensor(0.1 * rng.random(F[m.Q:].shape))
    return F.to(torch.float32).to(torch.float64)


@pytest.mark.parametrize("kernel", ["tiles", "async"])
@pytest.mark.parametrize("name", [n for n in CASES if not n.endswith("bf16")])
def test_tiles_one_step_against_oracle(name, kernel):
    P = CASES[name].replace(objective="none", obj_window=0, kernel=kernel)
    th = _theta(P, 1)
    o = Oracle(P, th)
    F = _random_state(o, 2)
    M = o.model.M
    post = o.collide(F).reshape(M, -1).numpy()
    nxt = o.step(F).reshape(M, -1).numpy()
    rng = np.random.default_rng(5)
    lam = rng.standard_normal(F.shape).astype(np.float32)
    gF, gth = o.adjoint_step(torch.tensor(lam, dtype=torch.float64), F)
    gF, gth = gF.reshape(M, -1).numpy(), gth.numpy()
    with _solver(P, th) as s:
        s.set_populations(torch.tensor(F.reshape(M, -1).numpy(), dtype=torch.float32, device="cuda"))
        s.primal_step(1)
        g_post = _np(s.populations(1))
        g_next = _np(s.populations(0))
        s.adjoint_seed(torch.tensor(lam.reshape(M, -1), device="cuda"))
        s.adjoint_step(1)
        lam0 = _np(s.adjoint())
        grad = _np(s.gradient())
    scale = np.abs(post).max()
    assert np.abs(g_post - post).max() <= 2e-6 * scale
    assert np.abs(g_next - nxt).max() <= 2e-6 * scale
    assert np.abs(lam0 - gF).max() <= 2e-5 * np.abs(gF).max()
    assert np.abs(grad - gth).max() <= 2e-5 * np.abs(gth).max()


@pytest.mark.parametrize("name", list(CASES))
def test_tiles_match_per_node_kernels(name):
    P = CASES[name]
    th = _theta(P, 3)
    out = {}
    for kern in ("plain", "tiles", "async"):
        with _solver(P.replace(kernel=kern), th) as s:
            s.primal_step(P.nsteps)
            f = _np(s.populations(0))
            J = s.objective()
            s.adjoint_step(P.nsteps)
            out[kern] = (f, J, _np(s.gradient()))
    f0, J0, g0 = out["plain"]
    for kern in ("tiles", "async"):
        f1, J1, g1 = out[kern]
        assert np.abs(f1 - f0).max() <= 1e-6 * np.abs(f0).max()
        assert abs(J1 - J0) <= 1e-6 * abs(J0)
        assert np.abs(g1 - g0).max() <= 1e-5 * np.abs(g0).max()


def test_tiles_refused_when_nx_is_not_a_tile_multiple():
    from paper_1501_04741_gb300.albm import AlbmError
    P = inputs.channel2d(dims=(100, 20, 1), kernel="tiles")
    with pytest.raises(AlbmError, match="multiple of 128"):
        _solver(P, inputs.theta_uniform(P, 0))
