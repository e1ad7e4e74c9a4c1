"""Failure detection on the GPU without a fault: a non-finite value written
into the state from the host is counted (LBM_ERR_NONFINITE) and the server's
watchdog retires only the request it spoils; a tile-staged kernel whose
bounded wait is armed to give up at once returns, the host reads
LBM_ERR_TIMEOUT, and the handle computes correct results again after
lbm_reset with the default bound."""
import numpy as np
import pytest
import torch

from paper_1501_04741_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_nonfinite_state_is_counted():
    from paper_1501_04741_gb300.albm import Solver
    P = inputs.channel2d(dims=(40, 21, 1), design=(10, 30, 4, 17, 0, 1), nsteps=20,
                         force=(1e-4, 0.0, 0.0))
    th = torch.from_numpy(inputs.theta_uniform(P, 1).reshape(-1)).cuda()
    with Solver(P, th) as s:
        s.primal_step(5)
        assert s.check_finite() == 0
        f = s.populations(0)
        f[3, 400] = float("nan")
        s.set_populations(f)
        assert s.check_finite() == 1
        s.primal_step(3)
        assert s.check_finite() > 1          # the NaN spreads with the stream


def test_watchdog_retires_only_the_spoiled_request():
    from paper_1501_04741_gb300.albm import Solver
    from paper_1501_04741_gb300.serve import Request, Server
    spec = inputs.serving_requests(6, rate=500.0, seed=5, node_range=(2e3, 4e4), steps=(30, 80))
    reqs = [Request(i, t, P, th) for i, (t, P, th) in enumerate(spec)]
    bad = reqs[3]
    th = np.array(bad.theta, dtype=np.float32, copy=True)
    x0, x1, y0, y1, z0, z1 = bad.P.design
    th[z0, y0 + 1, x0 + 1] = np.nan                   # one design node
    reqs[3] = Request(3, bad.arrival, bad.P, th)
    Server(steps_per_tick=16, work_per_tick=1e6).run(reqs)
    assert reqs[3].error == "non-finite objective or gradient"
    for i, r in enumerate(reqs):
        if i == 3:
            continue
        assert r.error is None
        with Solver(r.P, r.theta) as s:
            s.run()
            assert s.objective() == r.J


def test_staged_kernel_wait_gives_up_and_the_handle_recovers():
    from paper_1501_04741_gb300.albm import AlbmError, Solver
    P = inputs.scaled(inputs.mixer3d(), (128, 12, 10), nsteps=8, obj_window=2, kernel="tiles")
    th = torch.from_numpy(inputs.theta_uniform(P, 2).reshape(-1)).cuda()
    with Solver(P, th) as ref:
        ref.run()
        J_ref, g_ref = ref.objective(), ref.gradient().cpu().numpy()
    with Solver(P, th) as s:
        s.set_wait_polls(0)                          # every stage wait gives up at once
        s.primal_step(2)
        with pytest.raises(AlbmError, match="LBM_ERR_TIMEOUT"):
            s.objective()
        s.set_wait_polls(-1)
        s.reset()
        s.run()
        assert s.objective() == J_ref
        assert np.array_equal(s.gradient().cpu().numpy(), g_ref)
