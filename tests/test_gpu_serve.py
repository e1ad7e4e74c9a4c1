"""Continuous batching on the GPU: requests that arrive while others run are
admitted and advanced together in batched launches, and every result (J and
dJ/dtheta) is bit-identical to the same request solved alone."""
import numpy as np
import pytest
import torch

from paper_1501_04741_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    from paper_1501_04741_gb300.albm import Solver
    from paper_1501_04741_gb300.serve import Request, Server, request_bytes, run_sequential
    spec = inputs.serving_requests(12, rate=200.0, seed=7, node_range=(2e3, 2e5), steps=(40, 160))
    reqs = [Request(i, t, P, th) for i, (t, P, th) in enumerate(spec)]
    cap = 6 * max(request_bytes(r.P) for r in reqs)       # forces queueing
    srv = Server(capacity_bytes=cap, steps_per_tick=16, work_per_tick=2e6)
    stats = srv.run(reqs)
    assert all(r.error is None for r in reqs)
    assert stats.max_resident >= 2
    for r in reqs:
        with Solver(r.P, r.theta) as s:
            s.run()
            assert s.objective() == r.J
            assert np.array_equal(s.gradient().cpu().numpy(), r.grad)
    seq = [Request(i, t, P, th) for i, (t, P, th) in enumerate(spec)]
    run_sequential(seq)
    for a, b in zip(reqs, seq):
        assert a.J == b.J and np.array_equal(a.grad, b.grad)
