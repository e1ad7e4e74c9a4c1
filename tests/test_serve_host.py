"""Host-side scheduling of the continuous-batching server against a fake
device (no GPU): admission by the byte model, FIFO order, waiting for
memory, oversize and malformed requests, cancellation, and that a failure
of one request leaves the others' results untouched."""
import numpy as np
import pytest

from paper_1501_04741_gb300 import inputs
from paper_1501_04741_gb300.serve import Request, Server, request_bytes


class FakeSolver:
    """Counts steps like a handle; J and the gradient depend only on theta."""

    live = 0

    def __init__(self, P, theta, stream=None, mem_budget=0.0):
        if P.tau <= 0.5:
            raise RuntimeError("LBM_ERR_ARG: tau must exceed 1/2")
        self.P = P
        self.theta = np.asarray(theta, dtype=np.float64).reshape(-1)
        self.time = 0
        self.adjoint_time = -1
        FakeSolver.live += 1

    def objective(self):
        return float(self.theta.sum())

    def gradient(self):
        return 2.0 * self.theta

    def close(self):
        FakeSolver.live -= 1


def _ks(ss, k):
    return list(k) if isinstance(k, (list, tuple)) else [k] * len(ss)


def fake_primal(ss, k):
    for s, ki in zip(ss, _ks(ss, k)):
        s.time = min(s.P.nsteps, s.time + ki)


def fake_adjoint(ss, k):
    for s, ki in zip(ss, _ks(ss, k)):
        if s.adjoint_time < 0:
            s.adjoint_time = s.time
        s.adjoint_time = max(0, s.adjoint_time - ki)


def _server(capacity, **kw):
    return Server(capacity_bytes=capacity, solver_factory=FakeSolver, primal_fn=fake_primal,
                  adjoint_fn=fake_adjoint, mem_get_info=lambda: (0, 0), **kw)


def _reqs(n, seed=0):
    out = []
    for i, (t, P, th) in enumerate(inputs.serving_requests(n, rate=1e4, seed=seed,
                                                            node_range=(1e3, 5e4),
                                                            steps=(40, 120))):
        out.append(Request(i, t, P, th))
    return out


def test_all_requests_finish_and_results_depend_only_on_the_request():
    reqs = _reqs(12)
    cap = 3.5 * max(request_bytes(r.P) for r in reqs)
    srv = _server(cap, steps_per_tick=10, work_per_tick=1e5)
    stats = srv.run(reqs)
    assert all(r.error is None and r.done is not None for r in reqs)
    for r in reqs:
        assert r.J == float(r.theta.astype(np.float64).sum())
    assert FakeSolver.live == 0
    assert stats.max_resident >= 2                 # requests overlapped
    assert stats.p99 >= stats.p50 >= 0


def test_admission_respects_capacity_and_fifo():
    reqs = _reqs(10, seed=1)
    cap = 2.2 * max(request_bytes(r.P) for r in reqs)
    seen = []

    def watch(srv):
        assert srv.committed <= cap
        seen.append([r.rid for r in srv.active])
    srv = _server(cap, steps_per_tick=15, work_per_tick=1e5)
    srv.run(reqs, on_tick=watch)
    order = sorted(reqs, key=lambda r: (r.admitted, r.rid))
    assert [r.rid for r in order] == sorted(r.rid for r in reqs)   # FIFO admission
    assert max(len(s) for s in seen) >= 2                           # batching happened
    assert any(r.admitted > r.arrival for r in reqs)                # someone waited for memory


def test_oversize_and_malformed_requests_fail_alone():
    reqs = _reqs(6, seed=2)
    cap = 4 * max(request_bytes(r.P) for r in reqs)
    big = inputs.exchanger3d(dims=(2048, 1024, 1024), nsteps=10)
    reqs.append(Request(100, reqs[-1].arrival, big, np.zeros(1, np.float32)))
    reqs.append(Request(101, reqs[-1].arrival, reqs[0].P.replace(tau=0.4), reqs[0].theta))
    srv = _server(cap, steps_per_tick=10, work_per_tick=1e5)
    srv.run(reqs)
    by = {r.rid: r for r in reqs}
    assert "capacity" in by[100].error
    assert "tau" in by[101].error
    for i in range(6):
        assert by[i].error is None and by[i].J == float(by[i].theta.astype(np.float64).sum())
    assert FakeSolver.live == 0


def test_cancellation_releases_memory():
    reqs = _reqs(8, seed=3)
    cap = 3 * max(request_bytes(r.P) for r in reqs)
    state = {"done": False}

    def cancel_one(srv):
        if not state["done"] and srv.active:
            victim = srv.active[0].rid
            assert srv.cancel(victim)
            state["done"] = True
            state["victim"] = victim
    srv = _server(cap, steps_per_tick=5, work_per_tick=1e5)
    srv.run(reqs, on_tick=cancel_one)
    v = state["victim"]
    for r in reqs:
        if r.rid == v:
            assert r.error == "cancelled"
        else:
            assert r.error is None
    assert srv.committed == 0 and FakeSolver.live == 0


def test_request_out_of_memory_in_a_batched_step_fails_alone():
    # A batched step that runs out of device memory is retried one request at
    # a time; the request whose pool cannot grow is retired with an error and
    # its memory released, the others finish with their own results.
    from paper_1501_04741_gb300.albm import AlbmError

    def primal_oom(ss, k):
        if any(s.P.nsteps == 77 for s in ss):
            raise AlbmError(2, "cudaMalloc failed: out of memory")
        fake_primal(ss, k)

    reqs = _reqs(6, seed=3)
    reqs[2] = Request(2, reqs[2].arrival, reqs[2].P.replace(nsteps=77), reqs[2].theta)
    srv = Server(capacity_bytes=1e15, solver_factory=FakeSolver, primal_fn=primal_oom,
                 adjoint_fn=fake_adjoint, mem_get_info=lambda: (0, 0))
    FakeSolver.live = 0
    srv.run(reqs)
    assert reqs[2].error == "out of device memory"
    assert srv.committed == 0 and FakeSolver.live == 0
    for i, r in enumerate(reqs):
        if i != 2:
            assert r.error is None and r.J == float(np.asarray(r.theta, np.float64).sum())
