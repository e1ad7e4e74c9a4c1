"""Primal LLBS iteration, unsteady discrete adjoint and finite differences (FP64).

Test infrastructure only (see ``oracle/__init__``).

State layout: ``F`` is a (M, Lz, Ly, Lx) float64 tensor, the pre-collision
densities f^n of every node (x fastest).  One step is the paper's push form
of Eq. "normal:iteration":

    f^{n+1}_j(x + e_j) = W^x_j(f^n(x), theta)      (shifts modulo Lx, Ly, Lz)

The objective is J = sum_n c_n F(f^n) (weights from ``Model.weights``).  The
exact gradient of J(theta) for the N-step map follows the chain rule used in
the proof of the Theorem (Sec. 2.2), applied to the time-dependent problem:

    lambda^N = c_N dF/df(f^N)
    lambda^n = (d(S W)/df)^T lambda^{n+1} + c_n dF/df(f^n),   n = N-1 .. 0
    dJ/dtheta = sum_n (d(S W)/dtheta)^T lambda^{n+1} + sum_n c_n dF/dtheta

where (d(S W)/df)^T lambda at (x, k) is sum_j lambda_j(x + e_j) dW^x_j/df_k,
i.e. the adjoint collision of Eq. "adjoint:operator" after streaming in the
opposite direction (Eq. "adjoint:iteration").  The vector-Jacobian products
are taken by torch.autograd on the step function.

``frozen_adjoint`` is the paper's ALBS itself: Eq. "adjoint:iteration"
iterated at a fixed state f-hat, with the gradient of Eq.
"adjoint:derivative" evaluated from the final iterate.

``oneshot`` is the one-shot optimisation of Sec. 3.3 (primal, adjoint and
design updated together, Eq. "gradient:update", with the penalty of Eq. P),
and ``threshold`` / ``threshold_scan`` the final binarisation of Sec. 3.2.
"""
from __future__ import annotations

import numpy as np
import torch

from .model import DT, INLET, OUTLET, Model, build_flags


class Oracle:
    """One problem on the full lattice."""

    def __init__(self, P, theta):
        self.P = P
        self.model = Model(P)
        Lx, Ly, Lz = P.dims
        self.shape = (Lz, Ly, Lx)
        self.n = Lx * Ly * Lz
        self.flags_np = build_flags(P)
        self.flags = torch.from_numpy(self.flags_np.reshape(-1).astype(np.int64))
        self.y = torch.arange(Ly).view(1, Ly, 1).expand(Lz, Ly, Lx).reshape(-1)
        self.theta = torch.as_tensor(np.asarray(theta, dtype=np.float32).reshape(-1)).to(DT)
        self.n_in = max(int((self.flags == INLET).sum()), 1)
        self.n_out = max(int((self.flags == OUTLET).sum()), 1)
        self.c = self.model.weights()

    # --- state --------------------------------------------------------------
    def initial(self):
        """f^0: fluid at rest equilibrium (rho = 1, u = 0), scalars zero."""
        m = self.model
        F = torch.zeros((m.M, self.n), dtype=DT)
        F[:m.Q] = m.w[:, None]
        return F.view(m.M, *self.shape)

    def stream(self, post):
        """Periodic streaming S of Sec. 2.1: (S p)_j(x + e_j) = p_j(x)."""
        out = []
        for j, e in enumerate(self.model.E_all):
            out.append(torch.roll(post[j], shifts=(int(e[2]), int(e[1]), int(e[0])),
                                  dims=(0, 1, 2)))
        return torch.stack(out)

    def unstream(self, a):
        """S^-1: gather a_j(x + e_j) to x (Lemma 1: S is unitary, S^T = S^-1)."""
        out = []
        for j, e in enumerate(self.model.E_all):
            out.append(torch.roll(a[j], shifts=(-int(e[2]), -int(e[1]), -int(e[0])),
                                  dims=(0, 1, 2)))
        return torch.stack(out)

    def collide(self, F, theta=None):
        th = self.theta if theta is None else theta
        M = self.model.M
        post = self.model.collide(F.reshape(M, -1), th, self.flags, self.y)
        return post.view(M, *self.shape)

    def step(self, F, theta=None):
        return self.stream(self.collide(F, theta))

    def F_obj(self, F, theta=None):
        th = self.theta if theta is None else theta
        return self.model.objective(F.reshape(self.model.M, -1), th, self.flags, self.y,
                                    self.n_in, self.n_out)

    # --- primal -------------------------------------------------------------
    def primal(self, nsteps=None, keep=True, F0=None):
        """Run N steps; returns (J, trajectory list f^0..f^N or [f^N])."""
        N = int(self.P.nsteps if nsteps is None else nsteps)
        c = self.model.weights() if nsteps is None else _weights(self.P, N)
        F = self.initial() if F0 is None else F0
        traj = [F] if keep else None
        J = 0.0
        with torch.no_grad():
            for n in range(N):
                if c[n] != 0.0:
                    J += c[n] * float(self.F_obj(F))
                F = self.step(F)
                if keep:
                    traj.append(F)
            if c[N] != 0.0:
                J += c[N] * float(self.F_obj(F))
        return J, (traj if keep else [F])

    def J(self, theta_np=None, nsteps=None):
        if theta_np is not None:
            saved = self.theta
            self.theta = torch.as_tensor(np.asarray(theta_np).reshape(-1)).to(DT)
            try:
                return self.primal(nsteps, keep=False)[0]
            finally:
                self.theta = saved
        return self.primal(nsteps, keep=False)[0]

    # --- adjoint ------------------------------------------------------------
    def source(self, F, weight):
        """weight * (dF/df, dF/dtheta) at state F."""
        Fv = F.detach().requires_grad_(True)
        th = self.theta.detach().requires_grad_(True)
        val = weight * self.F_obj(Fv, th)
        if not val.requires_grad:          # objective "none"
            return torch.zeros_like(Fv).detach(), torch.zeros_like(th).detach()
        gF, gth = torch.autograd.grad(val, (Fv, th), allow_unused=True)
        if gF is None:
            gF = torch.zeros_like(Fv)
        if gth is None:
            gth = torch.zeros_like(th)
        return gF.detach(), gth.detach()

    def adjoint_step(self, lam_next, F):
        """One backward step: ((d(SW)/df)^T lam, (d(SW)/dtheta)^T lam) at f^n = F."""
        Fv = F.detach().requires_grad_(True)
        th = self.theta.detach().requires_grad_(True)
        out = self.step(Fv, th)
        gF, gth = torch.autograd.grad(out, (Fv, th), grad_outputs=lam_next)
        return gF.detach(), gth.detach()

    def adjoint(self, traj, nsteps=None):
        """Unsteady adjoint over a stored trajectory f^0..f^N.

        Returns (dJ/dtheta as float64 (Lz, Ly, Lx), lambda^0).
        """
        N = len(traj) - 1
        c = _weights(self.P, N)
        grad = torch.zeros(self.n, dtype=DT)
        lam = torch.zeros_like(traj[N])
        if c[N] != 0.0:
            lam, gth = self.source(traj[N], c[N])
            grad += gth
        for n in range(N - 1, -1, -1):
            lam, gth = self.adjoint_step(lam, traj[n])
            grad += gth
            if c[n] != 0.0:
                s, gth2 = self.source(traj[n], c[n])
                lam = lam + s
                grad += gth2
        return grad.view(self.shape), lam

    def gradient(self, nsteps=None):
        """(J, dJ/dtheta, lambda^0) by primal + unsteady adjoint."""
        J, traj = self.primal(nsteps, keep=True)
        g, lam0 = self.adjoint(traj)
        return J, g, lam0

    # --- the paper's fixed-point ALBS ---------------------------------------
    def frozen_adjoint(self, F_hat, iters):
        """ALBS (Eq. adjoint:iteration) at the fixed state F_hat.

        v^{k+1} = (d(SW)/df(F_hat))^T v^k + dF/df(F_hat); the gradient is
        Eq. adjoint:derivative evaluated with the last iterate, plus the
        direct dependence of F on theta.
        """
        src, gth_direct = self.source(F_hat, 1.0)
        v = torch.zeros_like(F_hat)
        for _ in range(iters):
            v_next, _ = self.adjoint_step(v, F_hat)
            v = v_next + src
        _, gth = self.adjoint_step(v, F_hat)
        return (gth + gth_direct).view(self.shape), v

    # --- one-shot optimisation (Sec. 3.3) -----------------------------------
    def oneshot(self, iters, zeta, penalty=0.0, maximize=True, design=None, F0=None,
                v0=None):
        """The one-shot descent of Sec. 3.3 on theta (solid fraction).

        Iteration k, in the paper's order:
          1. one LLBS step (Eq. normal:iteration):     f^{k+1} = S W(f^k, theta^k)
          2. one ALBS step (Eq. adjoint:iteration) at the current primal state:
                                    v^{k+1} = (d(SW)/df(f^k))^T v^k + dF/df(f^k)
          3. the gradient estimate of Eq. adjoint:derivative from the adjoint
             iterate that step 2 consumes:
                                    g^k = (d(SW)/dtheta(f^k))^T v^k + dF/dtheta(f^k)
          4. the update of Eq. gradient:update with the penalty P of Eq. P,
             P = sum theta (1 - theta), on design nodes only:
                 theta^{k+1} = clip(theta^k + zeta (s g^k - penalty (1 - 2 theta^k)), 0, 1)
             with s = +1 when J is maximised, -1 when it is minimised (the
             penalty term always lowers P).

        Returns (theta^K as float64 (Lz, Ly, Lx), f^K, v^K, g^{K-1}).
        """
        th = self.theta.clone()
        mask = (torch.ones(self.n, dtype=torch.bool) if design is None else
                torch.as_tensor(np.asarray(design).reshape(-1).astype(bool)))
        s = 1.0 if maximize else -1.0
        F = self.initial() if F0 is None else F0
        v = torch.zeros_like(F) if v0 is None else v0
        g = torch.zeros(self.n, dtype=DT)
        saved = self.theta
        try:
            for _ in range(int(iters)):
                self.theta = th
                with torch.no_grad():
                    F_next = self.step(F)
                gF, gth = self.adjoint_step(v, F)
                src, gth_direct = self.source(F, 1.0)
                v_next = gF + src
                g = gth + gth_direct
                th = self.design_update(th, g, zeta, penalty, s, mask)
                F, v = F_next, v_next
        finally:
            self.theta = saved
        return th.view(self.shape), F, v, g.view(self.shape)

    @staticmethod
    def design_update(th, g, zeta, penalty, s, mask):
        """Eq. gradient:update on the penalised objective s J - penalty P,
        d(P)/d(theta) = 1 - 2 theta, kept in [0, 1], design nodes only."""
        d = s * g - penalty * (1.0 - 2.0 * th)
        return torch.where(mask, torch.clamp(th + zeta * d, 0.0, 1.0), th)

    def penalty(self, theta, design=None):
        """P of Eq. P over the design nodes."""
        th = torch.as_tensor(np.asarray(theta, dtype=np.float64).reshape(-1))
        if design is not None:
            th = th[torch.as_tensor(np.asarray(design).reshape(-1).astype(bool))]
        return float((th * (1.0 - th)).sum())

    def steady_objective(self, nsteps, theta=None):
        """F(f^N) of the primal run of N steps from rest (the objective of
        the converged flow when N is long enough)."""
        saved = self.theta
        try:
            if theta is not None:
                self.theta = torch.as_tensor(np.asarray(theta, dtype=np.float64).reshape(-1))
            F = self.initial()
            with torch.no_grad():
                for _ in range(int(nsteps)):
                    F = self.step(F)
                return float(self.F_obj(F))
        finally:
            self.theta = saved

    @staticmethod
    def threshold(theta, eta, design=None):
        """The threshold of Sec. 3.2 on design nodes: w = 1 - theta below eta
        becomes solid (theta = 1), otherwise fluid (theta = 0).  theta is
        held in FP32, and w and the comparison are taken in FP32.  A node
        with w equal to eta is fluid."""
        th = np.asarray(theta, dtype=np.float32).reshape(-1)
        mask = np.ones(th.shape, bool) if design is None else np.asarray(design).reshape(-1).astype(bool)
        w = np.float32(1.0) - th
        out = th.copy()
        out[mask] = np.where(w[mask] < np.float32(eta), np.float32(1.0), np.float32(0.0))
        return out.reshape(np.shape(theta))

    def threshold_scan(self, theta, etas, nsteps, design=None):
        """F(f^N) of the thresholded design for every level eta."""
        return [self.steady_objective(nsteps, self.threshold(theta, e, design)) for e in etas]

    # --- MMA design iterations (Sec. 3.3, oracle.mma) ------------------------
    def mma(self, iters, maximize=True, design=None, prm=None, adjoint="unsteady"):
        """MMA as Sec. 3.3 runs it: per design iteration a full solve, then one
        MMA update of theta on the design nodes (``oracle.mma.update``; a
        maximised J is minimised as -J).  Returns (theta, [J per iteration],
        MMA state).

        adjoint="unsteady": the N-step primal and the unsteady adjoint (exact
        dJ/dtheta of the horizon's J).  adjoint="frozen": the N-step primal,
        then N iterations of the ALBS at f^N (Sec. 3.3 iterates the adjoint
        as many times as the primal); the gradient of Eq. adjoint:derivative
        is taken with the iterate the N-th iteration consumes, v^{N-1}, i.e.
        ``frozen_adjoint(f^N, N - 1)``."""
        from . import mma as M
        prm = prm or M.MMAParams()
        th = self.theta.numpy().astype(np.float64).copy()
        state = M.start(th)
        mask = None if design is None else np.asarray(design).reshape(-1).astype(bool)
        hist = []
        saved = self.theta
        try:
            for _ in range(int(iters)):
                self.theta = torch.as_tensor(th)
                if adjoint == "frozen":
                    J, traj = self.primal(keep=False)
                    g, _ = self.frozen_adjoint(traj[-1], int(self.P.nsteps) - 1)
                else:
                    J, g, _ = self.gradient()
                hist.append(J)
                g = g.reshape(-1).numpy()
                th = M.update(state, th, -g if maximize else g, mask, prm)
        finally:
            self.theta = saved
        return th.reshape(self.shape), hist, state

    # --- finite differences -------------------------------------------------
    def fd(self, index, h=1e-6, nsteps=None):
        """Central difference of J w.r.t. theta at one flat node index."""
        base = self.theta.clone()
        try:
            self.theta = base.clone()
            self.theta[index] += h
            Jp = self.primal(nsteps, keep=False)[0]
            self.theta = base.clone()
            self.theta[index] -= h
            Jm = self.primal(nsteps, keep=False)[0]
        finally:
            self.theta = base
        return (Jp - Jm) / (2 * h)


def _weights(P, N):
    K = int(P.obj_window)
    c = np.zeros(N + 1)
    if K <= 0:
        c[N] = 1.0
    else:
        c[max(N - K + 1, 0):] = 1.0 / K
    return c
