"""Pins of the oracle's MMA (Sec. 3.3; Svanberg's method, ``oracle.mma``).

* the separable approximation reproduces the objective's gradient at the
  current iterate (first-order exactness, the defining property of MMA's
  approximations) and is convex there;
* the closed-form minimiser of the subproblem equals a brute-force grid
  search of the approximation over the move limits;
* on a separable quadratic the iteration converges to the minimiser, also
  when it lies outside the box (the bound is the answer);
* on the LBM channel a few MMA iterations lower the dissipation they
  minimise (and raise it when asked to maximise).
"""
import numpy as np
import pytest

from oracle import mma as M
from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs


def _approx(y, x, L, U, p, q):
    return p / (U - y) + q / (y - L)


def _random_case(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.05, 0.95, n)
    g = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 1, n)
    dl = rng.uniform(0.02, 0.8, n)
    du = rng.uniform(0.02, 0.8, n)
    return x, g, x - dl, x + du


def test_approximation_is_first_order_exact_and_convex():
    x, g, L, U = _random_case(200, 0)
    _, (_, _, p, q) = M.subproblem(x, g, L, U)
    h = 1e-7
    d1 = (_approx(x + h, x, L, U, p, q) - _approx(x - h, x, L, U, p, q)) / (2 * h)
    assert np.abs(d1 - g).max() <= 1e-6 * np.abs(g).max()
    d2 = 2 * p / (U - x) ** 3 + 2 * q / (x - L) ** 3
    assert (d2 > 0).all()


def test_subproblem_minimiser_matches_grid_search():
    x, g, L, U = _random_case(64, 1)
    y, (alpha, beta, p, q) = M.subproblem(x, g, L, U)
    assert ((alpha <= y) & (y <= beta)).all()
    for j in range(len(x)):
        grid = np.linspace(alpha[j], beta[j], 200001)
        f = _approx(grid, x[j], L[j], U[j], p[j], q[j])
        yj = grid[np.argmin(f)]
        assert abs(y[j] - yj) <= 2 * (beta[j] - alpha[j]) / 200000, (j, y[j], yj)


def test_converges_on_a_separable_quadratic():
    # f = |x - a|^2 / 2.  The approximation carries no curvature of f, so
    # near the minimiser each step spans most of the asymptote distance and
    # the iterate oscillates as the oscillation rule shrinks that distance to
    # its floor dmin (x_max - x_min): the iterate ends within the floor of an
    # interior minimiser, and exactly on the bound when the minimiser lies
    # outside the box.
    prm = M.MMAParams()
    a = np.array([0.2, 0.7, 0.45, -0.3, 1.4])
    x = np.full(5, 0.5)
    st = M.start(x)
    for _ in range(60):
        x = M.update(st, x, x - a, prm=prm)
    assert np.abs(x[:3] - a[:3]).max() <= prm.dmin * (prm.x_max - prm.x_min)
    assert x[3] == 0.0 and x[4] == 1.0
    # the last asymptotes (built around the previous iterate) of the
    # interior variables sit at the floor: they oscillated
    assert np.allclose(st.x1[:3] - st.L[:3], prm.dmin, rtol=1e-12)
    assert np.allclose(st.U[:3] - st.x1[:3], prm.dmin, rtol=1e-12)


def test_mask_and_bounds():
    x, g, L, U = _random_case(50, 2)
    st = M.start(x)
    mask = np.arange(50) % 3 == 0
    y = M.update(st, x, g * 1e3, mask)
    assert np.array_equal(y[~mask], x[~mask])
    assert ((y >= 0) & (y <= 1)).all()
    assert st.k == 1 and np.array_equal(st.x1, x)


@pytest.mark.parametrize("maximize", [False, True])
def test_mma_moves_the_channel_objective_the_right_way(maximize):
    P = inputs.channel2d(dims=(16, 8, 1), tau=1.0, force=(1e-4, 0.0, 0.0),
                         design=(4, 12, 2, 6, 0, 1), nsteps=60)
    mask = inputs.design_mask(P)
    th0 = np.where(mask, 0.5, 0.0).astype(np.float32)
    o = Oracle(P, th0)
    prm = M.MMAParams(move=0.05)
    th, hist, st = o.mma(4, maximize=maximize, design=mask, prm=prm)
    J_end = o.J(th)
    if maximize:
        assert hist[0] < hist[1] < hist[2] < hist[3] < J_end
    else:
        assert hist[0] > hist[1] > hist[2] > hist[3] > J_end
    assert np.array_equal(th[~mask], th0[~mask].astype(np.float64))
