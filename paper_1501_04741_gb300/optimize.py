"""The optimisers of Sec. 3.3 driven through the C library: the one-shot
descent and MMA.

The loop of Sec. 3.3 -- one primal step, one adjoint (ALBS) step and one
design update per iteration, Eq. gradient:update -- runs entirely in
libalbm (``lbm_oneshot_step``).  This module only schedules it:

* iterations run in chunks; after each chunk the objective F of the current
  state and the penalty P of Eq. P are read back (``lbm_oneshot_eval``);
* the penalty weight starts at ``penalty0`` and is multiplied by
  ``penalty_growth`` after every chunk (the exponentially increasing weight
  of Sec. 4.2);
* at the end the threshold scan of Sec. 3.2 evaluates the binarised design
  for each level eta and the best level is applied (``lbm_threshold_scan``,
  ``lbm_threshold_apply``).

``mma`` runs the other optimiser of Sec. 3.3: a full solve per design
iteration (``lbm_run``) and one Method-of-Moving-Asymptotes update
(``lbm_mma_update``).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .albm import Solver
from .inputs import Problem


@dataclasses.dataclass
class OneShotResult:
    theta: np.ndarray                 # continuous design after the iterations (float32, N)
    history: list                     # (iterations done, J, P, penalty weight) per chunk
    etas: list                        # threshold levels scanned
    scan: list                        # J of the binarised design per level
    best_eta: float | None
    best_J: float | None
    theta_binary: np.ndarray | None   # design thresholded at best_eta


def one_shot(P: Problem, theta0, iters: int, zeta: float, *, maximize: bool = True,
             penalty0: float = 0.0, penalty_growth: float = 1.0, chunk: int = 100,
             design=None, etas=None, eval_steps: int | None = None,
             stream=None) -> OneShotResult:
    """Run ``iters`` one-shot iterations from ``theta0`` and (when ``etas`` is
    given) the threshold scan with ``eval_steps`` primal steps per level."""
    if iters < 0 or chunk < 1:
        raise ValueError("iters >= 0 and chunk >= 1 are required")
    with Solver(P, theta0, stream=stream) as s:
        s.set_design(design)
        s.oneshot_reset()
        history = []
        done, pen = 0, float(penalty0)
        while done < iters:
            k = min(chunk, iters - done)
            s.oneshot_step(k, zeta, pen, maximize)
            done += k
            J, Pv = s.oneshot_eval()
            history.append((done, J, Pv, pen))
            if not np.isfinite(J):
                raise FloatingPointError(f"one-shot objective became {J} after {done} iterations")
            pen *= penalty_growth
        theta = s.theta().cpu().numpy()
        if not etas:
            return OneShotResult(theta, history, [], [], None, None, None)
        etas = [float(e) for e in etas]
        scan = s.threshold_scan(etas, int(eval_steps or P.nsteps))
        pick = int(np.argmax(scan) if maximize else np.argmin(scan))
        s.threshold_apply(etas[pick])
        theta_bin = s.theta().cpu().numpy()
        return OneShotResult(theta, history, etas, scan, etas[pick], scan[pick], theta_bin)


@dataclasses.dataclass
class MMAResult:
    theta: np.ndarray        # design after the last update (float32, N)
    history: list            # J of each design iteration's solve


def mma(P: Problem, theta0, iters: int, *, maximize: bool = True, move: float = 0.5,
        design=None, stream=None, adjoint: str = "unsteady") -> MMAResult:
    """The MMA design loop of Sec. 3.3: per iteration a full solve and one MMA
    update of theta, all in the library (``lbm_run``, ``lbm_mma_update``).

    ``adjoint="unsteady"``: the solve is the N-step primal and its exact
    unsteady adjoint.  ``adjoint="frozen"``: the paper's schedule, the
    N-step primal (run until the flow has converged) followed by the same
    number of ALBS iterations at its final state (Sec. 3.3), whose gradient
    is that of the stationary objective F(f^N)."""
    if adjoint not in ("unsteady", "frozen"):
        raise ValueError(f"unknown adjoint schedule {adjoint!r}")
    if adjoint == "frozen":
        P = P.replace(adjoint_mode="frozen", obj_window=0)
    with Solver(P, theta0, stream=stream) as s:
        s.set_design(design)
        s.mma_reset()
        hist = []
        for _ in range(int(iters)):
            s.run()
            J = s.objective()
            if not np.isfinite(J):
                raise FloatingPointError(f"MMA objective became {J} at iteration {len(hist)}")
            hist.append(J)
            s.mma_update(maximize, move)
        return MMAResult(s.theta().cpu().numpy(), hist)
