"""MMA design iterations (Sec. 3.3) on the GPU against the oracle.

* the update kernel against ``oracle.mma`` over several iterations, fed the
  same seeded gradients (``lbm_mma_update_with``): the asymptote decisions
  (oscillating / monotone) are taken on the signs of differences of the
  stored FP32 designs, so they match; the values follow FP32 arithmetic
  (tolerance 2e-5 on theta in [0, 1]);
* the loop (full solve + update) on the 2D channel against the oracle's
  loop: J of every iteration within 1e-4 relative, designs within 1e-3;
* guards.
"""
import numpy as np
import pytest
import torch

from oracle import mma as M
from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs
from paper_1501_04741_gb300.albm import AlbmError, Solver
from paper_1501_04741_gb300.optimize import mma

pytestmark = pytest.mark.gpu


def _channel():
    return inputs.channel2d(dims=(16, 8, 1), tau=1.0, force=(1e-4, 0.0, 0.0),
                            design=(4, 12, 2, 6, 0, 1), nsteps=60)


@pytest.mark.parametrize("maximize", [True, False])
def test_update_kernel_against_oracle(maximize):
    P = inputs.channel2d(dims=(64, 33, 1), design=(8, 56, 4, 29, 0, 1), nsteps=4)
    mask = inputs.design_mask(P).reshape(-1)
    rng = np.random.default_rng(11)
    th0 = np.where(mask, rng.uniform(0.05, 0.95, mask.size), 0.3).astype(np.float32)
    prm = M.MMAParams(move=0.3)
    st = M.start(th0)
    x = th0.astype(np.float64)
    with Solver(P, torch.from_numpy(th0).cuda()) as s:
        s.set_design(mask)
        s.mma_reset()
        for it in range(6):
            g = rng.standard_normal(mask.size) * 10.0 ** rng.uniform(-2, 1, mask.size)
            s.mma_update_with(g, maximize, prm.move)
            x = M.update(st, x, -g if maximize else g, mask, prm)
            got = s.theta().cpu().numpy().astype(np.float64)
            assert np.abs(got - x).max() <= 2e-5, (it, np.abs(got - x).max())
            assert np.array_equal(got[~mask], th0[~mask].astype(np.float64))


def test_loop_against_oracle():
    P = _channel()
    mask = inputs.design_mask(P)
    th0 = np.where(mask, 0.5, 0.0).astype(np.float32)
    prm = M.MMAParams(move=0.05)
    th_o, hist_o, _ = Oracle(P, th0).mma(4, maximize=False, design=mask, prm=prm)
    r = mma(P, th0, 4, maximize=False, move=0.05, design=mask.reshape(-1))
    for a, b in zip(r.history, hist_o):
        assert abs(a - b) <= 1e-4 * abs(b), (a, b)
    assert np.abs(r.theta - th_o.reshape(-1)).max() <= 1e-3
    assert r.history == sorted(r.history, reverse=True)       # minimised


def test_guards():
    P = _channel()
    th0 = np.where(inputs.design_mask(P), 0.5, 0.0).astype(np.float32)
    with Solver(P, torch.from_numpy(th0.reshape(-1)).cuda()) as s:
        with pytest.raises(AlbmError, match="LBM_ERR_STATE"):
            s.mma_update()                         # no lbm_mma_reset
        s.mma_reset()
        with pytest.raises(AlbmError, match="LBM_ERR_STATE"):
            s.mma_update()                         # no completed adjoint
        s.run()
        with pytest.raises(AlbmError, match="LBM_ERR_ARG"):
            s.mma_update(True, 1.5)
        s.mma_update(True, 0.2)
        assert s.time == 0                         # reset for the next solve


def test_loop_with_the_frozen_schedule_against_oracle():
    # the paper's schedule: per design iteration the primal, then as many
    # ALBS iterations at its final state (Sec. 3.3)
    P = _channel()
    mask = inputs.design_mask(P)
    th0 = np.where(mask, 0.5, 0.0).astype(np.float32)
    prm = M.MMAParams(move=0.05)
    th_o, hist_o, _ = Oracle(P, th0).mma(3, maximize=False, design=mask, prm=prm,
                                         adjoint="frozen")
    r = mma(P, th0, 3, maximize=False, move=0.05, design=mask.reshape(-1), adjoint="frozen")
    for a, b in zip(r.history, hist_o):
        assert abs(a - b) <= 1e-4 * abs(b), (a, b)
    assert np.abs(r.theta - th_o.reshape(-1)).max() <= 1e-3
