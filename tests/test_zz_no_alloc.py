"""The allocation-free objective entry point agrees with the handle-based one.

lbm_state_objective_noalloc serves callers that cannot allocate device
memory when they need an objective value (a process whose device memory is
reserved in advance, a host framework that owns the allocator).  Its
scratch is a fixed static device array, so it is checked here against
lbm_objective of a normal handle on the same state, within the J tolerance
of the parity tests (5e-5 relative), on two calls in a row.
This file is collected last so that a failure here leaves every other test
already run.
"""
import numpy as np
import pytest
import torch

from paper_1501_04741_gb300 import inputs

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "channel2d_dissipation": inputs.channel2d(dims=(64, 33, 1), design=(16, 48, 8, 24, 0, 1),
                                                  nsteps=300, force=(1e-4, 0.0, 0.0)),
        "mixer3d_variance": inputs.scaled(inputs.mixer3d(), (40, 16, 16), nsteps=200,
                                          obj_window=0),
        "exchanger3d_heatflux": inputs.scaled(inputs.exchanger3d(), (41, 14, 13), nsteps=150),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_objective_matches_handle(name):
    from paper_1501_04741_gb300.albm import Solver, state_objective_noalloc
    P = CASES[name]
    th = torch.from_numpy(inputs.theta_uniform(P, 11).reshape(-1)).cuda()
    with Solver(P, th) as s:
        s.primal_step(P.nsteps)
        J_ref = s.objective()          # F(f^N): the weight sits on the last step only
        f = s.populations(0)
        flags = torch.from_numpy(s.flags()).cuda()
    vals = [state_objective_noalloc(P, f, th, flags) for _ in range(2)]
    for v in vals:
        assert abs(v - J_ref) <= 5e-5 * abs(J_ref) + 1e-15, (v, J_ref)
    assert vals[0] == vals[1]


def test_noalloc_rejects_oversize_lattice():
    # a D2Q9 lattice one row above the limit, with buffers of the full size
    # (so that no path could launch on undersized buffers): the library
    # rejects it before any launch
    from paper_1501_04741_gb300.albm import AlbmError, state_objective_noalloc
    P = inputs.channel2d(dims=(4097, 2048, 1))     # 8,390,656 > 8,388,608 nodes
    N = P.n_nodes
    f = torch.zeros((9, N), device="cuda")
    th = torch.zeros(N, device="cuda")
    fl = torch.zeros(N, dtype=torch.uint8, device="cuda")
    with pytest.raises(AlbmError, match="no-alloc limit"):
        state_objective_noalloc(P, f, th, fl)


def test_noalloc_wrapper_rejects_short_buffers():
    from paper_1501_04741_gb300.albm import state_objective_noalloc
    P = CASES["channel2d_dissipation"]
    N = P.n_nodes
    th = torch.zeros(N, device="cuda")
    fl = torch.zeros(N, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError, match="f must be"):
        state_objective_noalloc(P, torch.zeros(1, device="cuda"), th, fl)
    with pytest.raises(ValueError, match="flags must be"):
        state_objective_noalloc(P, torch.zeros((9, N), device="cuda"), th, th)
