"""Method of Moving Asymptotes for box-bounded design variables (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

Sec. 3.3 names MMA (Svanberg 1987, the paper's reference for it) as its
second optimiser and gives no formulas; the steps below follow Svanberg's
published method for min f(x) with x_min <= x <= x_max and no further
constraints, in the order of one design iteration k:

1. asymptotes L_j < x_j < U_j.  For k < 2: x_j -/+ s0 (x_max - x_min).  For
   k >= 2 the distances of the previous iteration are scaled by gamma_j:
   s_dec when x_j oscillates ((x^k - x^{k-1}) and (x^{k-1} - x^{k-2}) of
   opposite sign), s_inc when it moves monotonically, 1 when either
   difference is zero:
       L_j = x_j - gamma_j (x^{k-1}_j - L^{k-1}_j),
       U_j = x_j + gamma_j (U^{k-1}_j - x^{k-1}_j),
   then held between 0.01 and 10 times (x_max - x_min) from x_j.
2. move limits alpha_j = max(x_min, L_j + albefa (x_j - L_j), x_j - move (x_max - x_min)),
   beta_j = min(x_max, U_j - albefa (U_j - x_j), x_j + move (x_max - x_min)).
3. the convex separable approximation of f around x^k, in Svanberg's
   regularised form (both terms present, so the approximation is strictly
   convex): with g = df/dx at x^k, g+ = max(g, 0), g- = max(-g, 0),
       p_j = (U_j - x_j)^2 (1.001 g+ + 0.001 g- + raa0 / (x_max - x_min)),
       q_j = (x_j - L_j)^2 (0.001 g+ + 1.001 g- + raa0 / (x_max - x_min)),
       f~(y) = sum_j p_j / (U_j - y_j) + q_j / (y_j - L_j)  (+ const).
4. the next iterate minimises f~ over [alpha, beta]; the problem is
   separable and f~_j is strictly convex on (L_j, U_j) with its stationary
   point where p/(U - y)^2 = q/(y - L)^2:
       y_j = (sqrt(p_j) L_j + sqrt(q_j) U_j) / (sqrt(p_j) + sqrt(q_j)),
   clipped to [alpha_j, beta_j].
A maximised objective J is minimised as f = -J.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class MMAParams:
    s0: float = 0.5          # initial asymptote distance / (x_max - x_min)
    s_dec: float = 0.7       # oscillating variable: asymptotes closer
    s_inc: float = 1.2       # monotone variable: asymptotes farther
    albefa: float = 0.1      # move limit as a fraction of the distance to an asymptote
    move: float = 0.5        # move limit as a fraction of (x_max - x_min)
    raa0: float = 1e-5       # regularisation of the approximation
    dmin: float = 0.01       # asymptote distance bounds / (x_max - x_min)
    dmax: float = 10.0
    x_min: float = 0.0
    x_max: float = 1.0


def asymptotes(k, x, x1, x2, L1, U1, prm: MMAParams = MMAParams()):
    """Step 1: (L, U) of iteration k from x^k, x^{k-1}, x^{k-2} and the
    previous asymptotes (arrays; x1, x2, L1, U1 are unused for k < 2)."""
    x = np.asarray(x, np.float64)
    span = prm.x_max - prm.x_min
    if k < 2:
        return x - prm.s0 * span, x + prm.s0 * span
    d1 = np.sign(np.asarray(x, np.float64) - np.asarray(x1, np.float64))
    d2 = np.sign(np.asarray(x1, np.float64) - np.asarray(x2, np.float64))
    gamma = np.where(d1 * d2 < 0, prm.s_dec, np.where(d1 * d2 > 0, prm.s_inc, 1.0))
    dl = gamma * (np.asarray(x1, np.float64) - np.asarray(L1, np.float64))
    du = gamma * (np.asarray(U1, np.float64) - np.asarray(x1, np.float64))
    dl = np.clip(dl, prm.dmin * span, prm.dmax * span)
    du = np.clip(du, prm.dmin * span, prm.dmax * span)
    return x - dl, x + du


def subproblem(x, g, L, U, prm: MMAParams = MMAParams()):
    """Steps 2-4: the minimiser of the separable approximation on the move
    limits, and (alpha, beta, p, q) for inspection."""
    x, g, L, U = (np.asarray(v, np.float64) for v in (x, g, L, U))
    span = prm.x_max - prm.x_min
    alpha = np.maximum.reduce([np.full_like(x, prm.x_min), L + prm.albefa * (x - L),
                               x - prm.move * span])
    beta = np.minimum.reduce([np.full_like(x, prm.x_max), U - prm.albefa * (U - x),
                              x + prm.move * span])
    gp, gm = np.maximum(g, 0.0), np.maximum(-g, 0.0)
    reg = prm.raa0 / span
    p = (U - x) ** 2 * (1.001 * gp + 0.001 * gm + reg)
    q = (x - L) ** 2 * (0.001 * gp + 1.001 * gm + reg)
    sp, sq = np.sqrt(p), np.sqrt(q)
    y = (sp * L + sq * U) / (sp + sq)
    return np.clip(y, alpha, beta), (alpha, beta, p, q)


@dataclasses.dataclass
class MMAState:
    """Design history of the MMA iterations."""
    k: int
    x1: np.ndarray      # x^{k-1}
    x2: np.ndarray      # x^{k-2}
    L: np.ndarray       # asymptotes of the last iteration
    U: np.ndarray


def start(x) -> MMAState:
    x = np.asarray(x, np.float64)
    return MMAState(0, x.copy(), x.copy(), x.copy(), x.copy())


def update(state: MMAState, x, g, mask=None, prm: MMAParams = MMAParams()):
    """One MMA iteration on f with gradient g at x; variables outside mask
    stay.  Returns the new x and advances ``state``."""
    x = np.asarray(x, np.float64)
    L, U = asymptotes(state.k, x, state.x1, state.x2, state.L, state.U, prm)
    y, _ = subproblem(x, g, L, U, prm)
    if mask is not None:
        m = np.asarray(mask, bool)
        y = np.where(m, y, x)
    state.x2, state.x1 = state.x1, x.copy()
    state.L, state.U = L, U
    state.k += 1
    return y
