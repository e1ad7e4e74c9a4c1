"""Host logic of the optimiser drivers (``optimize.one_shot``, ``optimize.mma``)
against a fake solver: the chunk schedule, the exponentially growing
penalty weight, the choice of the threshold level, the MMA loop and the
watchdog on a non-finite objective.  No GPU: the fake records the calls the
drivers make."""
import numpy as np
import pytest

from paper_1501_04741_gb300 import inputs, optimize


class FakeSolver:
    """Stands in for ``albm.Solver``: records calls, returns scripted values."""
    script_J = None          # objective values returned in order (one-shot eval / MMA solves)
    scan = None

    def __init__(self, P, theta, stream=None):
        self.P = P
        self._theta = np.asarray(theta, dtype=np.float32).reshape(-1).copy()
        self.calls = []
        self._k = 0
        FakeSolver.last = self

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.calls.append(("close",))

    def set_design(self, mask):
        self.calls.append(("set_design", mask is None))

    def oneshot_reset(self):
        self.calls.append(("oneshot_reset",))

    def oneshot_step(self, iters, zeta, penalty, maximize):
        self.calls.append(("oneshot_step", iters, zeta, penalty, maximize))

    def oneshot_eval(self):
        J = FakeSolver.script_J[self._k]
        self._k += 1
        return J, 10.0 - self._k

    def theta(self):
        class T:
            def __init__(self, a):
                self.a = a

            def cpu(self):
                return self

            def numpy(self):
                return self.a
        return T(self._theta.copy())

    def threshold_scan(self, etas, nsteps):
        self.calls.append(("threshold_scan", tuple(etas), nsteps))
        return list(FakeSolver.scan)

    def threshold_apply(self, eta):
        self.calls.append(("threshold_apply", eta))
        self._theta = np.where(self._theta > 1 - eta, 1.0, 0.0).astype(np.float32)

    def mma_reset(self):
        self.calls.append(("mma_reset",))

    def run(self):
        self.calls.append(("run",))

    def objective(self):
        J = FakeSolver.script_J[self._k]
        self._k += 1
        return J

    def mma_update(self, maximize, move):
        self.calls.append(("mma_update", maximize, move))


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(optimize, "Solver", FakeSolver)
    return FakeSolver


P = inputs.channel2d(dims=(16, 8, 1), design=(4, 12, 2, 6, 0, 1), nsteps=10)
TH = inputs.theta_uniform(P, 0)


def test_one_shot_schedule_and_penalty_growth(fake):
    fake.script_J = [1.0, 2.0, 3.0]
    fake.scan = []
    r = optimize.one_shot(P, TH, 250, 0.5, penalty0=1e-3, penalty_growth=10.0, chunk=100)
    steps = [c for c in fake.last.calls if c[0] == "oneshot_step"]
    assert [c[1] for c in steps] == [100, 100, 50]
    assert [c[3] for c in steps] == pytest.approx([1e-3, 1e-2, 1e-1])
    assert [h[0] for h in r.history] == [100, 200, 250]
    assert [h[1] for h in r.history] == [1.0, 2.0, 3.0]
    assert r.best_eta is None and r.theta_binary is None


@pytest.mark.parametrize("maximize,pick", [(True, 1), (False, 2)])
def test_one_shot_picks_the_best_threshold(fake, maximize, pick):
    fake.script_J = [1.0]
    fake.scan = [0.5, 0.9, 0.1]
    etas = [0.2, 0.5, 0.8]
    r = optimize.one_shot(P, TH, 10, 0.1, maximize=maximize, chunk=10, etas=etas, eval_steps=7)
    assert ("threshold_scan", tuple(etas), 7) in fake.last.calls
    assert r.best_eta == etas[pick] and r.best_J == fake.scan[pick]
    assert ("threshold_apply", etas[pick]) in fake.last.calls
    assert set(np.unique(r.theta_binary)) <= {0.0, 1.0}


def test_one_shot_stops_on_a_non_finite_objective(fake):
    fake.script_J = [1.0, float("nan")]
    fake.scan = []
    with pytest.raises(FloatingPointError):
        optimize.one_shot(P, TH, 300, 0.1, chunk=100)


def test_mma_loop(fake):
    fake.script_J = [3.0, 2.0, 1.5]
    r = optimize.mma(P, TH, 3, maximize=False, move=0.1)
    kinds = [c[0] for c in fake.last.calls]
    assert kinds[:2] == ["set_design", "mma_reset"]
    assert kinds.count("run") == 3 and kinds.count("mma_update") == 3
    assert all(c[1:] == (False, 0.1) for c in fake.last.calls if c[0] == "mma_update")
    assert r.history == [3.0, 2.0, 1.5]


def test_mma_stops_on_a_non_finite_objective(fake):
    fake.script_J = [3.0, float("inf")]
    with pytest.raises(FloatingPointError):
        optimize.mma(P, TH, 5)


def test_argument_checks(fake):
    with pytest.raises(ValueError):
        optimize.one_shot(P, TH, -1, 0.1)
    with pytest.raises(ValueError):
        optimize.one_shot(P, TH, 10, 0.1, chunk=0)
