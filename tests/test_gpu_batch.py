"""Batched launches (one kernel per step for many instances) give results
bit-identical to driving each instance alone, for uneven sizes and horizons,
for batches split above the 64-instance table, and for the checkpoint
schedule running under them."""
import numpy as np
import pytest
import torch

from paper_1501_04741_gb300 import inputs

pytestmark = pytest.mark.gpu


def _family_2d(k):
    rng = np.random.default_rng(k)
    out = []
    for i in range(k):
        Lx = int(rng.integers(12, 70))
        Ly = int(rng.integers(8, 40))
        n = int(rng.integers(20, 90))
        P = inputs.channel2d(dims=(Lx, Ly, 1), design=(Lx // 4, 3 * Lx // 4, Ly // 4, 3 * Ly // 4, 0, 1),
                             nsteps=n, force=(1e-4, 0, 0))
        out.append(P)
    return out


def _family_3d(k):
    rng = np.random.default_rng(100 + k)
    out = []
    for i in range(k):
        d = (int(rng.integers(12, 30)), int(rng.integers(8, 16)), int(rng.integers(8, 14)))
        out.append(inputs.scaled(inputs.exchanger3d(), d, nsteps=int(rng.integers(15, 60))))
    return out


def _alone(P, th, **kw):
    from paper_1501_04741_gb300.albm import Solver
    with Solver(P, torch.from_numpy(th.reshape(-1)).cuda(), **kw) as s:
        s.run()
        return s.objective(), s.gradient().cpu().numpy()


def _batched(Ps, ths, **kw):
    from paper_1501_04741_gb300.albm import Solver, batch_adjoint_step, batch_primal_step
    ss = [Solver(P, torch.from_numpy(th.reshape(-1)).cuda(), **kw) for P, th in zip(Ps, ths)]
    try:
        horizon = max(P.nsteps for P in Ps)
        batch_primal_step(ss, horizon)
        for s, P in zip(ss, Ps):
            assert s.time == P.nsteps
        Js = [s.objective() for s in ss]
        batch_adjoint_step(ss, horizon)
        for s in ss:
            assert s.adjoint_time == 0
        gs = [s.gradient().cpu().numpy() for s in ss]
        return Js, gs
    finally:
        for s in ss:
            s.close()


def test_mixed_sizes_and_window_objective_equal_alone():
    """One instance above 2^20 nodes (its own launch inside the batched step)
    beside small ones (the shared launch), with an objective recorded over a
    window of steps (per-step sums folded from block partials): J and
    dJ/dtheta bit-identical to each instance driven alone."""
    big = inputs.channel2d(dims=(1040, 1024, 1), design=(260, 780, 256, 768, 0, 1), nsteps=12,
                           force=(1e-4, 0, 0), obj_window=5)
    assert big.n_nodes >= 1 << 20
    Ps = [big,
          inputs.channel2d(dims=(42, 18, 1), design=(10, 30, 4, 14, 0, 1), nsteps=12,
                           force=(1e-4, 0, 0), obj_window=4),
          inputs.channel2d(dims=(60, 20, 1), design=(15, 45, 5, 15, 0, 1), nsteps=9,
                           force=(1e-4, 0, 0), obj_window=4)]
    ths = [inputs.theta_uniform(P, i + 7) for i, P in enumerate(Ps)]
    Js, gs = _batched(Ps, ths)
    for P, th, J, g in zip(Ps, ths, Js, gs):
        J1, g1 = _alone(P, th)
        assert J == J1, (P.dims, J, J1)
        assert np.array_equal(g, g1), P.dims


@pytest.mark.parametrize("family", ["2d", "3d"])
def test_batched_equals_alone(family):
    Ps = _family_2d(7) if family == "2d" else _family_3d(5)
    ths = [inputs.theta_uniform(P, i) for i, P in enumerate(Ps)]
    Js, gs = _batched(Ps, ths)
    for P, th, J, g in zip(Ps, ths, Js, gs):
        J1, g1 = _alone(P, th)
        assert J == J1
        assert np.array_equal(g, g1)


def test_batch_split_beyond_table_and_small_pools():
    Ps = _family_2d(70)
    ths = [inputs.theta_uniform(P, i) for i, P in enumerate(Ps)]
    Js, gs = _batched(Ps[:70], ths[:70])
    for i in (0, 33, 64, 69):
        J1, g1 = _alone(Ps[i], ths[i])
        assert Js[i] == J1 and np.array_equal(gs[i], g1)
    Pc = [P.replace(ckpt_every=7) for P in Ps[:6]]
    # room for the level-1 checkpoints (nsteps/7 + 1) plus a few recompute slots
    budgets = [(P.nsteps // 7 + 6) * 4 * 9 * P.n_nodes for P in Pc]
    from paper_1501_04741_gb300.albm import Solver, batch_adjoint_step, batch_primal_step
    ss = [Solver(P, torch.from_numpy(th.reshape(-1)).cuda(), mem_budget=b)
          for P, th, b in zip(Pc, ths[:6], budgets)]
    try:
        batch_primal_step(ss, 100)
        batch_adjoint_step(ss, 100)
        for s, P, th in zip(ss, Pc, ths[:6]):
            assert s.recompute_steps() > 0
            J1, g1 = _alone(P, th)
            assert s.objective() == J1 and np.array_equal(s.gradient().cpu().numpy(), g1)
    finally:
        for s in ss:
            s.close()


def test_solves_are_bit_reproducible():
    # the objective reduction has a fixed order, so J (and the variance
    # source that depends on its outlet mean) repeat bit for bit
    P = inputs.scaled(inputs.mixer3d(), (64, 32, 32), nsteps=120, obj_window=40)
    th = inputs.theta_uniform(P, 9)
    a = _alone(P, th)
    b = _alone(P, th)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_per_handle_step_counts_match_single_steps():
    # lbm_batch_primal_steps / lbm_batch_adjoint_steps with a different count
    # per handle reach the same states as stepping each handle alone
    from paper_1501_04741_gb300.albm import Solver, batch_adjoint_step, batch_primal_step
    Ps = [inputs.channel2d(dims=(40 + 8 * i, 21, 1), design=(8, 30, 4, 17, 0, 1), nsteps=50,
                           force=(1e-4, 0.0, 0.0)) for i in range(3)]
    ths = [torch.from_numpy(inputs.theta_uniform(P, 20 + i).reshape(-1)).cuda()
           for i, P in enumerate(Ps)]
    batch = [Solver(P, th) for P, th in zip(Ps, ths)]
    try:
        batch_primal_step(batch, [7, 0, 13])
        assert [s.time for s in batch] == [7, 0, 13]
        batch_primal_step(batch, [100, 50, 100])       # capped at the horizon
        assert [s.time for s in batch] == [50, 50, 50]
        batch_adjoint_step(batch, [5, 50, 20])
        assert [s.adjoint_time for s in batch] == [45, 0, 30]
        batch_adjoint_step(batch, 50)
        got = [(s.objective(), s.gradient().cpu().numpy()) for s in batch]
    finally:
        for s in batch:
            s.close()
    for (J, g), P, th in zip(got, Ps, ths):
        with Solver(P, th) as s:
            s.run()
            assert s.objective() == J
            assert np.array_equal(s.gradient().cpu().numpy(), g)
