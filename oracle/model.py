"""Node types, the local collision operator W^x and the objectives F^x (FP64).

Test infrastructure only (see ``oracle/__init__``).

Everything here acts on a flat list of nodes: ``F`` has shape (M, n) with the
M = Q + nscalars*Qs densities of one node stacked as in Sec. 2.1 (fluid
populations first, then each scalar lattice), together with that node's flag,
porosity ``theta`` and y coordinate (the inlet scalar profile depends on y).
W^x uses only the node's own densities (Sec. 2.1: the collision is local).

Node types (Sec. 3: interior, inlet/outlet, wall):

====  =========  ==========================================================
code  name       W^x
====  =========  ==========================================================
0     FLUID      FMRT (Sec. 3.1) or BGK (Eq. SRT) with Exact-Difference
                 forcing; Darcy porosity u_post = G(theta) u_pre + g (Sec. 3.2)
1     WALL       full-way bounce-back W_j = f_opp(j) for every lattice
2     INLET      Zou-He inlet on the x = 0 face, then the FLUID W; velocity
                 inlet (u = u_in) or pressure inlet (rho = rho_out + 3 dp)
                 whose velocity is capped at u_in (above the cap the node is
                 a velocity inlet at the cap, Sec. 4); scalars set to
                 equilibrium at the inlet value with the node's velocity
3     OUTLET     Zou-He pressure outlet on the x = Lx-1 face, then the FLUID
                 W; the unknown scalar populations are set to equilibrium at
                 the node's own scalar value, solved from the known ones
4     HOT        fluid bounce-back, scalars set to equilibrium at T_hot
====  =========  ==========================================================
"""
from __future__ import annotations

import numpy as np
import torch

from .lattice import Lattice, moment_basis

FLUID, WALL, INLET, OUTLET, HOT = 0, 1, 2, 3, 4

DT = torch.float64


def build_flags(P) -> np.ndarray:
    """uint8 (Lz, Ly, Lx) node-type array of the channel geometry.

    Order of precedence: inlet/outlet faces, then wall planes (edges and
    corners of the box are walls), then the hot patch on the y = 0 plane.
    """
    Lx, Ly, Lz = P.dims
    fl = np.zeros((Lz, Ly, Lx), dtype=np.uint8)
    if P.channel == "inlet_outlet":
        fl[:, :, 0] = INLET
        fl[:, :, Lx - 1] = OUTLET
    if "y" in P.walls:
        fl[:, 0, :] = WALL
        fl[:, Ly - 1, :] = WALL
    if "z" in P.walls:
        fl[0, :, :] = WALL
        fl[Lz - 1, :, :] = WALL
    if P.hot:
        x0, x1, z0, z1 = P.hot
        fl[max(z0, 0):min(z1, Lz), 0, max(x0, 0):min(x1, Lx)] = HOT
    return fl


class Model:
    """Fixed data of one problem: lattices, rates, MRT matrices."""

    def __init__(self, P):
        self.P = P
        self.fl = Lattice(P.lattice)
        self.sl = Lattice("D3Q7" if P.lattice == "D3Q19" else "D2Q9")
        self.Q, self.Qs, self.NS = self.fl.Q, self.sl.Q, int(P.nscalars)
        self.M = self.Q + self.NS * self.Qs
        self.E = torch.tensor(self.fl.E, dtype=DT)              # (Q, 3)
        self.w = torch.tensor(self.fl.w, dtype=DT)              # (Q,)
        self.Es = torch.tensor(self.sl.E, dtype=DT)
        self.ws = torch.tensor(self.sl.w, dtype=DT)
        # streaming vectors of all M densities of a node
        self.E_all = np.concatenate([self.fl.E] + [self.sl.E] * self.NS, axis=0)
        self.omega = 1.0 / P.tau
        self.nu = (P.tau - 0.5) / 3.0                             # 1/omega = 0.5 + 3 nu
        self.g = torch.tensor(P.force, dtype=DT)
        if P.collision == "MRT":
            U, conserved, stress = moment_basis(self.fl)
            s = np.full(self.Q, P.s_other, dtype=np.float64)
            s[stress] = self.omega
            s[conserved] = 0.0
            self.U = torch.tensor(U, dtype=DT)
            self.Uinv = torch.tensor(np.linalg.inv(U), dtype=DT)
            self.I_minus_T = torch.tensor(1.0 - s, dtype=DT)       # diagonal of (I - T)
        elif P.collision != "BGK":
            raise ValueError(P.collision)

    # --- equilibria ---------------------------------------------------------
    def feq(self, rho, u):
        """Second-order equilibrium w_i rho (1 + e.u/cs2 + (e.u)^2/(2cs4) - u^2/(2cs2))."""
        cs2 = self.fl.cs2
        eu = self.E @ u                                            # (Q, n)
        uu = (u * u).sum(0)
        return self.w[:, None] * rho * (1 + eu / cs2 + eu * eu / (2 * cs2 * cs2)
                                        - uu / (2 * cs2))

    def geq(self, T, u):
        """Scalar equilibrium w_i T (1 + e.u/cs2) (advection-diffusion)."""
        return self.ws[:, None] * T * (1 + (self.Es @ u) / self.sl.cs2)

    # --- porosity (Sec. 3.2) -------------------------------------------------
    def G(self, theta):
        """Switching function of the Darcy damping; G = 1 in fluid, 0 in solid."""
        P = self.P
        if P.porosity == "linear":
            return 1 - theta
        if P.porosity == "power":
            return 1 - theta ** P.porosity_q
        if P.porosity == "ramp":
            return (1 - theta) / (1 + P.porosity_q * theta)
        raise ValueError(P.porosity)

    def alpha(self, theta):
        """Linear interpolation of the scalar diffusivity (Sec. 3.2)."""
        return (1 - theta) * self.P.alpha_fluid + theta * self.P.alpha_solid

    # --- Zou-He on an x face ------------------------------------------------
    def zou_he(self, f, inward: int, u_n=None, rho=None):
        """Zou & He reconstruction of the unknown populations on an x face.

        ``inward`` is +1 on the x = 0 face and -1 on x = Lx-1.  The unknowns
        are the populations with e.n > 0 (n the inward normal).  Either the
        normal velocity ``u_n`` (velocity inlet) or ``rho`` (pressure outlet)
        is prescribed; transverse velocity is zero.  Mass and normal momentum
        give rho (1 - u_n) = s0 + 2 s_out.  Each unknown is its opposite plus
        the equilibrium difference 2 w_i rho (e_i.u)/cs2, minus the transverse
        correction sum_t e_it N_t with N_t = 1/2 sum_{e.n = 0} f_k e_kt
        - rho u_t/3, which restores the transverse momentum.
        Returns (f_reconstructed, rho, u).
        """
        E = self.fl.E
        en = E[:, 0] * inward
        zero = np.nonzero(en == 0)[0]
        out = np.nonzero(en < 0)[0]
        unk = np.nonzero(en > 0)[0]
        s0 = f[zero].sum(0)
        sout = f[out].sum(0)
        if u_n is not None:
            rho = (s0 + 2 * sout) / (1 - u_n)
            un = torch.full_like(s0, float(u_n))
        else:
            rho = torch.full_like(s0, float(rho))
            un = 1 - (s0 + 2 * sout) / rho
        zeros = torch.zeros_like(s0)
        u = torch.stack([un * inward, zeros, zeros])               # transverse u = 0
        N = {}
        for t in (1, 2):
            et = torch.tensor(E[zero, t], dtype=DT)
            N[t] = 0.5 * (et[:, None] * f[zero]).sum(0) - rho * u[t] / 3.0
        rows = [f[i] for i in range(self.Q)]
        for i in unk:
            eu = sum(float(E[i, a]) * u[a] for a in range(3))
            val = f[self.fl.opp[i]] + 2 * self.fl.w[i] * rho * eu / self.fl.cs2
            for t in (1, 2):
                if E[i, t] != 0:
                    val = val - float(E[i, t]) * N[t]
            rows[i] = val
        return torch.stack(rows), rho, u

    def inlet(self, f):
        """Zou-He reconstruction at the x = 0 face.  Velocity inlet: u_x =
        u_in.  Pressure inlet (Sec. 4: the inlet pressure is the pressure
        drop over the outlet's reference, p = cs2 rho): rho = rho_out + dp /
        cs2, giving u_x = 1 - (s0 + 2 s_out) / rho; where that exceeds the
        limit u_in the node is a velocity inlet at u_in instead."""
        P = self.P
        if P.inlet == "velocity":
            return self.zou_he(f, +1, u_n=P.u_in)[0]
        if P.inlet != "pressure":
            raise ValueError(P.inlet)
        f_p, _, u_p = self.zou_he(f, +1, rho=P.rho_out + P.dp / self.fl.cs2)
        f_c, _, _ = self.zou_he(f, +1, u_n=P.u_in)
        return torch.where(u_p[0] > P.u_in, f_c, f_p)

    def scalar_outlet(self, g, v):
        """Outlet scalar: unknown populations (e_x < 0) at equilibrium with the
        node's own value T*, solved from the known ones:
        T* = sum_known g / (1 - sum_unknown w_i (1 + e_i.v/cs2))."""
        Es = self.sl.E
        unk = np.nonzero(Es[:, 0] < 0)[0]
        known = np.nonzero(Es[:, 0] >= 0)[0]
        phi = 1 + (self.Es @ v) / self.sl.cs2                      # (Qs, n)
        denom = 1 - (self.ws[unk, None] * phi[unk]).sum(0)
        T = g[known].sum(0) / denom
        rows = [g[i] for i in range(self.Qs)]
        for i in unk:
            rows[i] = self.ws[i] * T * phi[i]
        return torch.stack(rows), T

    def inlet_scalar(self, s: int, y):
        """Inlet value of scalar s at row y ("halves": 0 below Ly/2, 1 above,
        odd scalars carry the complement 1 - c; "signed": -1 below Ly/2, +1
        above as in the paper's mixer (Sec. 4.1), odd scalars carry -c)."""
        P = self.P
        upper = (y >= P.dims[1] // 2).to(DT)
        if P.scalar_inlet == "halves":
            return 1 - upper if s % 2 == 1 else upper
        if P.scalar_inlet == "signed":
            c = 2 * upper - 1
            return -c if s % 2 == 1 else c
        return torch.zeros(y.shape, dtype=DT)

    # --- the node operator --------------------------------------------------
    def macroscopic(self, F, theta, flags):
        """Quantities the collision and the objectives share.

        Returns a dict with the reconstructed fluid populations ``fr``,
        ``rho``, ``u`` (pre-collision velocity), ``v`` (post-collision
        velocity G u + g), and per scalar the reconstructed populations and
        the scalar value ``T``.
        """
        P, Q, Qs = self.P, self.Q, self.Qs
        f = F[:Q]
        is_in = (flags == INLET)
        is_out = (flags == OUTLET)
        fr = f
        if P.channel == "inlet_outlet":
            f_in = self.inlet(f)
            f_out, _, _ = self.zou_he(f, -1, rho=P.rho_out)
            fr = torch.where(is_in, f_in, torch.where(is_out, f_out, f))
        rho = fr.sum(0)
        u = (self.E.T @ fr) / rho
        v = self.G(theta) * u + self.g[:, None]
        out = dict(f=f, fr=fr, rho=rho, u=u, v=v, gr=[], T=[])
        for s in range(self.NS):
            g = F[Q + s * Qs: Q + (s + 1) * Qs]
            gr = g
            if P.channel == "inlet_outlet":
                g_out, _ = self.scalar_outlet(g, v)
                gr = torch.where(is_out, g_out, g)
            out["gr"].append(gr)
            out["T"].append(gr.sum(0))
        return out

    def collide(self, F, theta, flags, y):
        """W^x(F(x), theta(x)) for every node of the list (Eq. normal:iteration)."""
        P, Q, Qs = self.P, self.Q, self.Qs
        m = self.macroscopic(F, theta, flags)
        fr, rho, u, v = m["fr"], m["rho"], m["u"], m["v"]
        feq_pre = self.feq(rho, u)
        feq_post = self.feq(rho, v)
        if P.collision == "BGK":
            # Eq. SRT plus the Exact-Difference forcing term of Sec. 3.1
            Wf = fr + self.omega * (feq_pre - fr) + (feq_post - feq_pre)
        else:
            # FMRT: U^-1 (m_eq^post + (I - T)(U f - m_eq^pre)), m_eq = U f_eq
            meq_post = self.U @ feq_post
            meq_pre = self.U @ feq_pre
            Wf = self.Uinv @ (meq_post + self.I_minus_T[:, None] * (self.U @ fr - meq_pre))
        f = m["f"]
        bounce = (flags == WALL) | (flags == HOT)
        Wf = torch.where(bounce, f[self.fl.opp], Wf)
        outs = [Wf]
        for s in range(self.NS):
            g = F[Q + s * Qs: Q + (s + 1) * Qs]
            gr, T = m["gr"][s], m["T"][s]
            omT = 1.0 / (0.5 + self.alpha(theta) / self.sl.cs2)
            Wg = gr + omT * (self.geq(T, v) - gr)
            if P.channel == "inlet_outlet":
                # equilibrium at the inlet value and the node's inlet velocity
                g_in = self.geq(self.inlet_scalar(s, y), u)
                Wg = torch.where(flags == INLET, g_in, Wg)
            Wg = torch.where(flags == WALL, g[self.sl.opp], Wg)
            if P.hot:
                g_hot = (self.ws[:, None] * P.T_hot).expand(Qs, g.shape[1])
                Wg = torch.where(flags == HOT, g_hot, Wg)
            outs.append(Wg)
        return torch.cat(outs, 0)

    # --- objectives F^x (Eq. objective:function) ----------------------------
    def objective(self, F, theta, flags, y, n_inlet: int = 1, n_outlet: int = 1):
        """Objective of one state f^n as a sum of node terms (torch scalar).

        * dissipation: sum over FLUID nodes of 2 rho nu S:S with
          S_ab = -(3 omega / (2 rho)) sum_i e_ia e_ib (f_i - f_eq,i(rho, u)).
        * variance: mean over OUTLET nodes of (c - mean c)^2 for scalar 0,
          c the outlet value T*.
        * heatflux_dp: sum over OUTLET nodes of v_x T* (Eq. exchanger:obj)
          minus 0.1 (mean inlet rho - rho_out)/3.
        * heatflux: sum over OUTLET nodes of v_x T* alone (Eq. exchanger:obj).
        * mixflux: sum over OUTLET nodes of v_x (1 - T*^2) (Eq. mixing:obj).
        """
        P = self.P
        kind = P.objective
        if kind == "none":
            return torch.zeros((), dtype=DT)
        m = self.macroscopic(F, theta, flags)
        if kind == "dissipation":
            f, rho, u = m["f"], m["rho"], m["u"]
            fneq = f - self.feq(rho, u)
            Pi = torch.einsum("ia,ib,in->abn", self.E, self.E, fneq)
            S = -(3 * self.omega / (2 * rho)) * Pi
            phi = 2 * rho * self.nu * (S * S).sum((0, 1))
            return (phi * (flags == FLUID)).sum()
        out = (flags == OUTLET).to(DT)
        c = m["T"][0]
        if kind == "variance":
            mean = (c * out).sum() / n_outlet
            return (((c - mean) ** 2) * out).sum() / n_outlet
        vx = m["v"][0]
        if kind == "heatflux_dp":
            inl = (flags == INLET).to(DT)
            rho_in_mean = (m["rho"] * inl).sum() / n_inlet
            return (vx * c * out).sum() - 0.1 * (rho_in_mean - P.rho_out) / 3.0
        if kind == "heatflux":
            return (vx * c * out).sum()
        if kind == "mixflux":
            return (vx * (1 - c * c) * out).sum()
        raise ValueError(kind)

    def weights(self):
        """Time weights c_n, n = 0..N, of J = sum_n c_n F(f^n)."""
        N, K = int(self.P.nsteps), int(self.P.obj_window)
        c = np.zeros(N + 1)
        if K <= 0:
            c[N] = 1.0
        else:
            c[max(N - K + 1, 0):] = 1.0 / K
        return c
