"""Parity at the full workload sizes, on sampled nodes.

The kernels run on the full 256x128x128 mixer (D3Q19 MRT + two D3Q7 scalars)
and the 512x256x256 heat exchanger (D3Q19 BGK + D3Q7), in the launch
configuration the benchmark times.  The oracle cannot run those lattices for
thousands of steps, but W^x and its transpose are node-local (Sec. 2.1), so
at sampled nodes it evaluates, from the GPU's own f^n and lambda^{n+1}:
  * one primal step: W^x(f^n(x)) against the GPU's post-collision state;
  * one adjoint step: sum_j lambda^{n+1}_j(x + e_j) dW^x_j/df_k(f^n(x)) and
    the theta terms against the GPU's lambda^n(x) and gradient increment.
Samples cover every node type.  Tolerances are those of the small-lattice
one-step tests (2e-6 of max|f|, 2e-5 of max|lambda| / max|dtheta|).
"""
import numpy as np
import pytest
import torch

from oracle.model import Model, build_flags
from paper_1501_04741_gb300 import inputs

pytestmark = pytest.mark.gpu


def _samples(flags_flat, n_random, seed):
    rng = np.random.default_rng(seed)
    idx = set(rng.choice(flags_flat.size, n_random, replace=False).tolist())
    for t in np.unique(flags_flat):
        where = np.nonzero(flags_flat == t)[0]
        idx.update(rng.choice(where, min(64, where.size), replace=False).tolist())
    return np.array(sorted(idx), dtype=np.int64)


def _coords(P, idx):
    Lx, Ly, Lz = P.dims
    return idx % Lx, (idx // Lx) % Ly, idx // (Lx * Ly)


def _shifted(P, idx, e):
    x, y, z = _coords(P, idx)
    Lx, Ly, Lz = P.dims
    return ((x + e[0]) % Lx) + Lx * (((y + e[1]) % Ly) + Ly * ((z + e[2]) % Lz))


def _workloads():
    mix = inputs.mixer3d(nsteps=400, obj_window=50)
    exch = inputs.exchanger3d(nsteps=240)
    return {"mixer3d_full": (mix, inputs.theta_uniform(mix, 0)),
            "exchanger3d_full": (exch, inputs.theta_grf(exch, 0))}


WORK = _workloads()


@pytest.mark.parametrize("name", list(WORK))
def test_fullsize_sampled_primal_and_adjoint(name):
    from paper_1501_04741_gb300.albm import Solver
    P, theta = WORK[name]
    model = Model(P)
    flags = build_flags(P).reshape(-1)
    th = theta.reshape(-1)
    idx = _samples(flags, 4000, 1)
    Lx, Ly, Lz = P.dims
    y = torch.from_numpy(((idx // Lx) % Ly).astype(np.int64))
    fl_t = torch.from_numpy(flags[idx].astype(np.int64))
    th_t = torch.from_numpy(th[idx].astype(np.float64))
    n0 = P.nsteps - 100                          # outside the objective window
    with Solver(P, torch.from_numpy(th).cuda()) as s:
        assert np.array_equal(s.flags(), flags)
        s.primal_step(n0)
        f_n = s.populations(0)[:, idx].double().cpu()
        s.primal_step(1)
        post = s.populations(1)[:, idx].double().cpu().numpy()
        # primal: W^x(f^n(x)) at the sampled nodes
        ref = model.collide(f_n, th_t, fl_t, y).numpy()
        assert np.abs(post - ref).max() <= 2e-6 * np.abs(ref).max()
        s.primal_step(P.nsteps - n0 - 1)
        assert s.check_finite() == 0
        # adjoint: run back to n0 + 1, then one step to n0
        s.adjoint_step(P.nsteps - (n0 + 1))
        lam_next = s.adjoint().cpu()
        g_before = s.gradient().cpu().numpy()
        s.adjoint_step(1)
        lam = s.adjoint()[:, idx].double().cpu().numpy()
        dth = s.gradient().cpu().numpy()[idx] - g_before[idx]
        f_n2 = s.populations_at(n0, 0)[:, idx].double().cpu()
    assert torch.equal(f_n2, f_n)                  # recomputed state is bit-identical
    a = torch.stack([lam_next[m, torch.from_numpy(_shifted(P, idx, e))]
                     for m, e in enumerate(model.E_all)]).double()
    Fv = f_n.clone().requires_grad_(True)
    tv = th_t.clone().requires_grad_(True)
    out = model.collide(Fv, tv, fl_t, y)
    gF, gth = torch.autograd.grad(out, (Fv, tv), grad_outputs=a)
    gF, gth = gF.numpy(), gth.numpy()
    assert np.abs(lam - gF).max() <= 2e-5 * np.abs(gF).max()
    assert np.abs(dth - gth).max() <= 2e-5 * np.abs(gth).max()
