"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 kernels against FP64):
* flags and node indexing: bit-exact;
* one primal step from the same state: max |f_gpu - f_oracle| <= 2e-6 max|f|;
* one adjoint step from the same state and lambda: <= 2e-5 of max|lambda|
  (and of max|dJ/dtheta| for the theta terms);
* whole trajectories, the two bars the problem statement fixes:
  - fluid populations within 1e-5 relative error element by element,
    max_i |f_gpu,i - f_i| / |f_i| <= 1e-5 (every fluid population is
    positive and near its weight w_i at these flow speeds);
  - scalar populations, whose values cross zero (signed inlets) or start at
    zero, within 1e-5 absolute; the scalar fields are bounded by their
    boundary values (magnitude 1), so this is the same bar relative to the
    field's range;
  - dJ/dtheta within 1e-4 (inf-norm relative);
  - J within 5e-5 relative.  J has no stated bar: the dissipation objective
    is quadratic in f - f_eq, about 1e-3 of |f| at these flow speeds, so a
    population error of 1e-5 |f| would allow a relative J error of order
    2e-5 |f| / |f - f_eq|; measured errors are below 2.5e-5.
Lattice sizes are odd so that the node count leaves a ragged last block.
"""
import numpy as np
import pytest
import torch

from oracle.model import build_flags
from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs

pytestmark = pytest.mark.gpu


def _cases():
    ch = inputs.channel2d(dims=(37, 21, 1), design=(8, 30, 4, 17, 0, 1), nsteps=60,
                          force=(1e-4, 0.0, 0.0))
    mix = inputs.scaled(inputs.mixer3d(), (21, 11, 10), nsteps=40, obj_window=6)
    exch = inputs.scaled(inputs.exchanger3d(), (23, 10, 9), nsteps=40)
    return {
        "d2q9_bgk": ch,
        "d2q9_mrt": ch.replace(collision="MRT"),
        "d2q9_bgk_scalar_ramp": ch.replace(nscalars=1, alpha_fluid=0.02, alpha_solid=0.3,
                                           porosity="ramp", porosity_q=2.0),
        "d3q19_mrt_mixer": mix,
        "d3q19_bgk_mixer_mixflux": mix.replace(collision="BGK", objective="mixflux",
                                               nscalars=1),
        "d3q19_bgk_exchanger": exch,
        "d3q19_mrt_exchanger_power": exch.replace(collision="MRT", porosity="power",
                                                  porosity_q=3.0),
        # the paper's own channels (Tab. tab:cases): signed inlet + mixing
        # flux, and the heat flux without the pressure term
        "d3q19_mrt_paper_mixer": inputs.scaled(inputs.paper_mixer_empty(), (23, 10, 10),
                                               nsteps=40),
        "d3q19_mrt_paper_exchanger": inputs.scaled(inputs.paper_exchanger_empty(), (14, 10, 9),
                                                   nsteps=120),
        # the pressure inlet below its velocity cap throughout
        "d3q19_bgk_exchanger_pressure_open": exch.replace(inlet="pressure", dp=0.003,
                                                          objective="heatflux_dp"),
    }


CASES = _cases()


def _theta(P, seed):
    th = inputs.theta_uniform(P, seed)
    rng = np.random.default_rng(seed + 100)
    th = th + (0.3 * rng.random(th.shape)).astype(np.float32) * (th == 0)
    return th.astype(np.float32)


def _random_state(o, seed):
    rng = np.random.default_rng(seed)
    m = o.model
    F = o.initial().clone()
    F[:m.Q] *= torch.tensor(1 + 0.02 * rng.standard_normal(F[:m.Q].shape))
    if m.NS:
        F[m.Q:] = torch.tensor(0.1 * rng.random(F[m.Q:].shape))
    return F.to(torch.float32).to(torch.float64)   # representable in FP32


def _solver(P, theta, **kw):
    from paper_1501_04741_gb300.albm import Solver
    return Solver(P, torch.from_numpy(theta.reshape(-1)).cuda(), **kw)


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def assert_populations_close(f_gpu, f_ref, Q, label=""):
    """The trajectory bar: fluid rows element by element within 1e-5
    relative, scalar rows within 1e-5 absolute."""
    rel = np.abs(f_gpu[:Q] - f_ref[:Q]) / np.abs(f_ref[:Q])
    print(f"[parity] {label} fluid max rel {rel.max():.2e}", end="")
    assert rel.max() <= 1e-5, rel.max()
    if f_ref.shape[0] > Q:
        ab = np.abs(f_gpu[Q:] - f_ref[Q:]).max()
        print(f"  scalar max abs {ab:.2e}", end="")
        assert ab <= 1e-5, ab
    print()


@pytest.mark.parametrize("name", list(CASES))
def test_flags_bit_exact(name):
    P = CASES[name]
    th = _theta(P, 0)
    with _solver(P, th) as s:
        assert np.array_equal(s.flags(), build_flags(P).reshape(-1))


@pytest.mark.parametrize("name", list(CASES))
def test_one_primal_step(name):
    P = CASES[name].replace(objective="none")
    th = _theta(P, 1)
    o = Oracle(P, th)
    F = _random_state(o, 2)
    post = o.collide(F).reshape(o.model.M, -1).numpy()
    nxt = o.step(F).reshape(o.model.M, -1).numpy()
    with _solver(P, th) as s:
        s.set_populations(torch.tensor(F.reshape(o.model.M, -1).numpy(), dtype=torch.float32,
                                       device="cuda"))
        back = _np(s.populations(0))
        assert np.abs(back - F.reshape(o.model.M, -1).numpy()).max() <= 1e-7
        s.primal_step(1)
        g_post = _np(s.populations(1))
        g_next = _np(s.populations(0))
    scale = np.abs(post).max()
    assert np.abs(g_post - post).max() <= 2e-6 * scale
    assert np.abs(g_next - nxt).max() <= 2e-6 * scale


@pytest.mark.parametrize("name", list(CASES))
def test_one_adjoint_step(name):
    P = CASES[name].replace(objective="none")
    th = _theta(P, 3)
    o = Oracle(P, th)
    F = _random_state(o, 4)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal(F.shape).astype(np.float32)
    gF, gth = o.adjoint_step(torch.tensor(lam, dtype=torch.float64), F)
    gF = gF.reshape(o.model.M, -1).numpy()
    gth = gth.numpy()
    with _solver(P, th) as s:
        s.set_populations(torch.tensor(F.reshape(o.model.M, -1).numpy(), dtype=torch.float32,
                                       device="cuda"))
        s.primal_step(1)
        s.adjoint_seed(torch.tensor(lam.reshape(o.model.M, -1), device="cuda"))
        s.adjoint_step(1)
        lam0 = _np(s.adjoint())
        grad = _np(s.gradient())
    assert np.abs(lam0 - gF).max() <= 2e-5 * np.abs(gF).max()
    assert np.abs(grad - gth).max() <= 2e-5 * max(np.abs(gth).max(), 1e-30)


@pytest.mark.parametrize("name", list(CASES))
def test_trajectory_objective_and_gradient(name):
    P = CASES[name]
    th = _theta(P, 6)
    o = Oracle(P, th)
    J, g, _ = o.gradient()
    _, traj = o.primal(keep=False)
    fN = traj[-1].reshape(o.model.M, -1).numpy()
    g = g.reshape(-1).numpy()
    with _solver(P, th) as s:
        s.primal_step(P.nsteps)
        f_gpu = _np(s.populations(0))
        J_gpu = s.objective()
        s.adjoint_step(P.nsteps)
        grad = _np(s.gradient())
    assert_populations_close(f_gpu, fN, o.model.Q, name)
    assert abs(J_gpu - J) <= 5e-5 * abs(J) + 1e-12, (J_gpu, J)
    assert np.abs(grad - g).max() <= 1e-4 * np.abs(g).max()


def test_checkpoint_recompute_is_exact():
    # Every state kept (level-1 stride 1) against a pool of 8 states with
    # level-1 checkpoints every 30 steps, which forces the recompute
    # schedule: the recomputed states are bit-identical, so J and the
    # gradient are too.
    P = CASES["d3q19_mrt_mixer"].replace(nsteps=90, ckpt_every=30)
    th = _theta(P, 7)
    with _solver(P.replace(ckpt_every=1), th) as s:
        s.run()
        g_all = _np(s.gradient())
        assert s.recompute_steps() == 0
        J_all = s.objective()
    state_bytes = 4 * P.n_nodes * (19 + 2 * 7)
    with _solver(P, th, mem_budget=8 * state_bytes) as s:
        s.run()
        g_small = _np(s.gradient())
        assert s.recompute_steps() > 0
        J_small = s.objective()
    assert J_all == J_small
    assert np.array_equal(g_all, g_small)


def test_channel2d_full_config_parity():
    # D2Q9 BGK 128x64, tau = 0.8, 2000 primal then 2000 adjoint steps,
    # viscous dissipation; theta ~ U[0,1] on the central 32x32 block.
    P = inputs.channel2d()
    th = inputs.theta_uniform(P, 0)
    o = Oracle(P, th)
    J, g, _ = o.gradient()
    _, traj = o.primal(keep=False)
    fN = traj[-1].reshape(9, -1).numpy()
    g = g.reshape(-1).numpy()
    with _solver(P, th) as s:
        s.primal_step(P.nsteps)
        f_gpu = _np(s.populations(0))
        J_gpu = s.objective()
        s.adjoint_step(P.nsteps)
        grad = _np(s.gradient())
    assert_populations_close(f_gpu, fN, 9, "channel2d full")
    assert abs(J_gpu - J) <= 5e-5 * abs(J), (J_gpu, J)
    assert np.abs(grad - g).max() <= 1e-4 * np.abs(g).max()
    # and within 1e-3 of central differences of the FP64 objective
    for i in list(np.argsort(-np.abs(g))[:3]):
        fd = o.fd(int(i), h=1e-5)
        assert abs(grad[i] - fd) <= 1e-3 * np.abs(g).max()
