"""torch.autograd.Function over the library: theta -> J with the adjoint as
backward, single and batched (mixed D2Q9 / D3Q19 instances in batched
launches), checked against the FP64 oracle's gradient (1e-4, inf-norm
relative) and its central finite differences (1e-3)."""
import numpy as np
import pytest
import torch

from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs

pytestmark = pytest.mark.gpu


def _small_cases():
    ch = inputs.channel2d(dims=(40, 22, 1), design=(10, 30, 5, 17, 0, 1), nsteps=120,
                          force=(1e-4, 0, 0))
    ex = inputs.scaled(inputs.exchanger3d(), (22, 10, 10), nsteps=80)
    return [ch, ex]


def test_autograd_single_matches_oracle_and_fd():
    from paper_1501_04741_gb300.albm import Solver
    from paper_1501_04741_gb300.autograd import albm_objective
    for P in _small_cases():
        th_np = inputs.theta_uniform(P, 3)
        o = Oracle(P, th_np)
        J_ref, g_ref, _ = o.gradient()
        g_ref = g_ref.reshape(-1).numpy()
        theta = torch.from_numpy(th_np.reshape(-1)).cuda().requires_grad_(True)
        with Solver(P, theta.detach()) as s:
            J = albm_objective(theta, s)
            (2.5 * J).backward()
        assert J.dtype == torch.float64
        assert abs(J.item() - J_ref) <= 5e-5 * abs(J_ref)
        g = theta.grad.double().cpu().numpy() / 2.5
        assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max() + 1e-6 * np.abs(g).max()
        for i in np.argsort(-np.abs(g_ref))[:2]:
            fd = o.fd(int(i), h=1e-5)
            assert abs(g[i] - fd) <= 1e-3 * np.abs(g_ref).max()


def test_autograd_batch_mixed_families():
    from paper_1501_04741_gb300.albm import Solver
    from paper_1501_04741_gb300.autograd import albm_objective, albm_objectives
    batch = inputs.batch_instances(8, seed=5, size_scale=0.12, steps=(30, 90))
    solvers, thetas = [], []
    for P, th in batch:
        t = torch.from_numpy(th.reshape(-1)).cuda().requires_grad_(True)
        thetas.append(t)
        solvers.append(Solver(P, t.detach()))
    try:
        Js = albm_objectives(thetas, solvers)
        w = torch.linspace(1.0, 2.0, len(batch), dtype=torch.float64, device="cuda")
        (w * Js).sum().backward()
        for k, ((P, th), s) in enumerate(zip(batch, solvers)):
            o = Oracle(P, th)
            J_ref, g_ref, _ = o.gradient()
            g_ref = g_ref.reshape(-1).numpy()
            assert abs(Js[k].item() - J_ref) <= 5e-5 * abs(J_ref)
            g = thetas[k].grad.double().cpu().numpy() / float(w[k])
            assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
        # batched and single autograd agree bit for bit
        P0, th0 = batch[0]
        t0 = torch.from_numpy(th0.reshape(-1)).cuda().requires_grad_(True)
        with Solver(P0, t0.detach()) as s0:
            J0 = albm_objective(t0, s0)
            J0.backward()
        assert J0.item() == Js[0].item()
        assert torch.equal(t0.grad, thetas[0].grad / w[0].float())
    finally:
        for s in solvers:
            s.close()


def test_stale_graph_is_refused():
    from paper_1501_04741_gb300.albm import Solver
    from paper_1501_04741_gb300.autograd import albm_objective
    P = _small_cases()[0]
    th = torch.from_numpy(inputs.theta_uniform(P, 1).reshape(-1)).cuda().requires_grad_(True)
    with Solver(P, th.detach()) as s:
        J1 = albm_objective(th, s)
        J2 = albm_objective(th, s)
        with pytest.raises(RuntimeError, match="another forward"):
            J1.backward()
        J2.backward()
        assert th.grad is not None
