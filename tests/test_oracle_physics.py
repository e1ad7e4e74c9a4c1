"""Pins of the oracle's primal iteration: Lemma 1, conservation laws, the
Poiseuille closed form, dissipation, Zou-He, porosity limits and scalar
diffusion (no GPU)."""
import math

import numpy as np
import pytest
import torch

from oracle.model import FLUID, INLET, OUTLET, WALL, HOT, build_flags
from oracle.solver import Oracle
from paper_1501_04741_gb300 import inputs


def _rand_state(o, seed, scale=0.02):
    rng = np.random.default_rng(seed)
    m = o.model
    F = o.initial().clone()
    F[:m.Q] *= torch.tensor(1 + scale * rng.standard_normal(F[:m.Q].shape))
    if m.NS:
        F[m.Q:] = torch.tensor(0.1 * rng.random(F[m.Q:].shape))
    return F


@pytest.mark.parametrize("lattice,dims,ns", [("D2Q9", (7, 5, 1), 1), ("D3Q19", (5, 4, 3), 2)])
def test_lemma1_streaming_is_a_permutation(lattice, dims, ns):
    # Lemma 1 (Sec. 2.2): S is unitary; S^-1 S = identity bit-exactly, sums
    # are invariant and <a, S b> = <S^-1 a, b>.
    P = inputs.Problem(lattice=lattice, dims=dims, walls="", nscalars=ns, objective="none")
    o = Oracle(P, np.zeros(dims[::-1], np.float32))
    rng = np.random.default_rng(0)
    a = torch.tensor(rng.standard_normal((o.model.M,) + o.shape))
    b = torch.tensor(rng.standard_normal((o.model.M,) + o.shape))
    assert torch.equal(o.unstream(o.stream(a)), a)
    assert torch.equal(o.stream(o.unstream(a)), a)
    assert abs(float(o.stream(a).sum() - a.sum())) < 1e-12
    lhs = float((a * o.stream(b)).sum())
    rhs = float((o.unstream(a) * b).sum())
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    # the shift moves f_j from x to x + e_j (periodic)
    e = o.model.E_all[3]
    z, y, x = dims[2] - 1, 2, 3
    val = o.stream(a)[3, (z + e[2]) % dims[2], (y + e[1]) % dims[1], (x + e[0]) % dims[0]]
    assert float(val) == float(a[3, z, y, x])


@pytest.mark.parametrize("coll", ["BGK", "MRT"])
@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_periodic_mass_and_momentum_conservation(coll, lattice):
    dims = (6, 5, 1) if lattice == "D2Q9" else (4, 4, 3)
    P = inputs.Problem(lattice=lattice, collision=coll, dims=dims, walls="", tau=0.7,
                       objective="none")
    o = Oracle(P, np.zeros(dims[::-1], np.float32))
    F = _rand_state(o, 1)
    m = o.model
    mass0 = float(F[:m.Q].sum())
    mom0 = torch.einsum("qa,q...->a", m.E, F[:m.Q])
    with torch.no_grad():
        for _ in range(100):
            F = o.step(F)
    assert abs(float(F[:m.Q].sum()) - mass0) < 1e-12 * mass0
    mom = torch.einsum("qa,q...->a", m.E, F[:m.Q])
    assert (mom - mom0).abs().max() < 1e-12 * mass0


def test_body_force_momentum_growth_is_exact():
    # Exact-Difference forcing (Sec. 3.1): u_post = u_pre + g, so the total
    # momentum grows by exactly (total mass) * g per step.
    dims = (5, 4, 1)
    g = (3e-5, -2e-5, 0.0)
    P = inputs.Problem(lattice="D2Q9", dims=dims, walls="", force=g, objective="none")
    o = Oracle(P, np.zeros(dims[::-1], np.float32))
    F = _rand_state(o, 2)
    m = o.model
    mass = float(F[:m.Q].sum())
    mom0 = torch.einsum("qa,q...->a", m.E, F[:m.Q])
    nsteps = 50
    with torch.no_grad():
        for _ in range(nsteps):
            F = o.step(F)
    mom = torch.einsum("qa,q...->a", m.E, F[:m.Q])
    expect = mom0 + nsteps * mass * torch.tensor(g, dtype=torch.float64)
    assert (mom - expect).abs().max() < 1e-13


def test_walls_conserve_mass():
    P = inputs.channel2d(dims=(9, 7, 1), design=(2, 6, 2, 5, 0, 1), objective="none")
    th = inputs.theta_uniform(P, 3)
    o = Oracle(P, th)
    F = _rand_state(o, 3)
    mass0 = float(F[:9].sum())
    with torch.no_grad():
        for _ in range(200):
            F = o.step(F)
    assert abs(float(F[:9].sum()) - mass0) < 1e-13 * mass0


def _poiseuille(coll, tau, Ly=10, g=1e-6, viscous_times=14):
    P = inputs.channel2d(dims=(3, Ly, 1), collision=coll, tau=tau, force=(g, 0, 0),
                         design=(0, 0, 0, 0, 0, 1), objective="dissipation")
    o = Oracle(P, np.zeros((1, Ly, 3), np.float32))
    nu = (tau - 0.5) / 3
    F = o.initial()
    with torch.no_grad():
        for _ in range(int(viscous_times * (Ly - 2) ** 2 / nu)):
            F = o.step(F)
    m = o.model
    f = F[:9].reshape(9, -1)
    rho = f.sum(0)
    # physical velocity of the Exact-Difference scheme: mean of pre and post
    ux = ((m.E.T @ f)[0] / rho + g / 2).reshape(Ly, 3)[:, 0].numpy()
    return o, F, ux, nu


def test_poiseuille_exact_at_magic_tau():
    # BGK with bounce-back walls reproduces the parabolic Poiseuille profile
    # exactly, with the wall half-way between wall and fluid nodes, when
    # (tau - 1/2)^2 = 3/16 (He, Zou, Luo & Dembo 1997): a closed-form pin of
    # the collision, the forcing, bounce-back and periodic streaming.
    g, Ly = 1e-6, 10
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    o, F, ux, nu = _poiseuille("BGK", tau, Ly=Ly, g=g)
    y = np.arange(Ly)
    a, b = 0.5, Ly - 1.5
    exact = g / (2 * nu) * (y - a) * (b - y)
    rel = np.abs(ux[1:-1] - exact[1:-1]).max() / exact.max()
    assert rel < 1e-9


@pytest.mark.parametrize("tau", [0.8, 0.6])
def test_poiseuille_profile_with_bgk_slip(tau):
    # Away from the magic tau, BGK + bounce-back adds a uniform slip
    # u_s = g (16 (tau-1/2)^2 - 3) / (24 nu) to the parabola (same reference).
    g, Ly = 1e-6, 10
    o, F, ux, nu = _poiseuille("BGK", tau, Ly=Ly, g=g)
    y = np.arange(Ly)
    a, b = 0.5, Ly - 1.5
    exact = g / (2 * nu) * (y - a) * (b - y) + g * (16 * (tau - 0.5) ** 2 - 3) / (24 * nu)
    rel = np.abs(ux[1:-1] - exact[1:-1]).max() / exact.max()
    assert rel < 2e-3
    # u_max within 1e-3 of the closed form once the stated slip is included
    assert abs(ux.max() - exact.max()) / exact.max() < 1e-3 + 1e-2 * abs(exact.max() - exact[1])


def test_dissipation_objective_closed_form():
    # Steady Poiseuille: 2 rho nu S:S = rho nu (du/dy)^2 with
    # du/dy = g (a + b - 2y) / (2 nu), summed over fluid nodes (3 columns).
    g, Ly, tau = 1e-6, 10, 0.8
    o, F, ux, nu = _poiseuille("BGK", tau, Ly=Ly, g=g)
    a, b = 0.5, Ly - 1.5
    phi = sum(nu * (g / (2 * nu) * (a + b - 2 * y)) ** 2 for y in range(1, Ly - 1)) * 3
    J = float(o.F_obj(F))
    assert abs(J - phi) / phi < 1e-6


def _mixer_small(**kw):
    return inputs.scaled(inputs.mixer3d(), (10, 6, 6), nsteps=20, obj_window=4, **kw)


def test_flags_channel_geometry():
    P = inputs.scaled(inputs.exchanger3d(), (14, 8, 8))
    fl = build_flags(P)
    assert fl.dtype == np.uint8
    assert (fl[1:-1, 1:-1, 0] == INLET).all() and (fl[1:-1, 1:-1, -1] == OUTLET).all()
    x0, x1, z0, z1 = P.hot
    assert (fl[z0:z1, 0, x0:x1] == HOT).all()
    hot = np.zeros_like(fl, dtype=bool)
    hot[z0:z1, 0, x0:x1] = True
    assert (fl[0][~hot[0]] == WALL).all() and (fl[-1][~hot[-1]] == WALL).all()
    assert (fl[1:-1, -1, :] == WALL).all()
    assert (fl[:, 0, :][~hot[:, 0, :]] == WALL).all()
    assert (fl[1:-1, 1:-1, 1:-1] == FLUID).all()


def test_wall_and_hot_nodes_after_collision():
    # Walls: full bounce-back of fluid and scalar populations; the hot patch
    # is a wall for the fluid and holds the scalar at the rest equilibrium
    # of T_hot (Dirichlet).
    P = inputs.scaled(inputs.exchanger3d(), (14, 8, 8), T_hot=0.8)
    o = Oracle(P, np.zeros(P.dims[::-1], np.float32))
    F = _rand_state(o, 9, scale=0.02)
    m = o.model
    pre = F.reshape(m.M, -1)
    post = o.collide(F).reshape(m.M, -1)
    opp = torch.tensor([int(v) for v in m.fl.opp])
    opps = torch.tensor([int(v) for v in m.sl.opp])
    wall = o.flags == WALL
    hot = o.flags == HOT
    assert int(hot.sum()) > 0 and int(wall.sum()) > 0
    for sel in (wall, hot):
        assert torch.equal(post[:m.Q][:, sel], pre[:m.Q][opp][:, sel])
    assert torch.equal(post[m.Q:][:, wall], pre[m.Q:][opps][:, wall])
    want = torch.as_tensor(np.asarray(m.sl.w, dtype=np.float64) * 0.8)[:, None]
    assert (post[m.Q:][:, hot] - want).abs().max() < 1e-15


def test_zou_he_prescribed_values_after_collision():
    # Zou & He (Sec. 3): after the node operator the inlet node carries
    # u = u_in and the outlet node rho = rho_out.
    P = _mixer_small(collision="BGK")
    o = Oracle(P, np.zeros(P.dims[::-1], np.float32))
    F = _rand_state(o, 5, scale=0.01)
    post = o.collide(F).reshape(o.model.M, -1)
    m = o.model
    f = post[:m.Q]
    rho = f.sum(0)
    u = (m.E.T @ f) / rho
    inl = o.flags == INLET
    out = o.flags == OUTLET
    assert (u[0, inl] - P.u_in).abs().max() < 1e-14
    assert u[1:, inl].abs().max() < 1e-14
    assert (rho[out] - P.rho_out).abs().max() < 1e-14
    assert u[1:, out].abs().max() < 1e-14
    # inlet scalars sit at equilibrium with the prescribed halves profile
    T0 = post[m.Q:m.Q + m.Qs].sum(0)
    T1 = post[m.Q + m.Qs:].sum(0)
    c = (o.y >= P.dims[1] // 2).double()
    assert (T0[inl] - c[inl]).abs().max() < 1e-14
    assert (T1[inl] - (1 - c[inl])).abs().max() < 1e-14


def test_porosity_limits():
    # Sec. 3.2: G(fluid) = 1 leaves the run unchanged (bit-exact with theta = 0)
    # and G(solid) = 0 gives u_post = 0 (no body force).
    P = inputs.channel2d(dims=(12, 8, 1), design=(3, 9, 2, 6, 0, 1), force=(0, 0, 0),
                         objective="none")
    o0 = Oracle(P, np.zeros((1, 8, 12), np.float32))
    F = _rand_state(o0, 7)
    o_same = Oracle(P.replace(design=(0, 0, 0, 0, 0, 1)), np.zeros((1, 8, 12), np.float32))
    assert torch.equal(o0.step(F), o_same.step(F))
    th = np.zeros((1, 8, 12), np.float32)
    th[0, 2:6, 3:9] = 1.0
    o1 = Oracle(P, th)
    post = o1.collide(F).reshape(o1.model.M, -1)
    j = o1.model.E.T @ post[:9]
    solid = torch.tensor(th.reshape(-1) == 1.0)
    assert j[:, solid].abs().max() < 1e-16


@pytest.mark.parametrize("law,q", [("linear", 1.0), ("power", 3.0), ("ramp", 2.0)])
@pytest.mark.parametrize("c", [0.25, 0.6])
def test_porosity_law_at_intermediate_theta(law, q, c):
    # Sec. 3.2: u_post = G(theta) u_pre.  An equilibrium state at uniform
    # velocity U in a periodic box with uniform theta = c and no force
    # collides to f_eq(rho, G(c) U), so its momentum is rho G(c) U exactly;
    # G by the readings of the laws: 1 - c, 1 - c^q, (1 - c) / (1 + q c).
    for coll in ("BGK", "MRT"):
        P = inputs.Problem(lattice="D3Q19", dims=(6, 5, 4), walls="", collision=coll, tau=0.7,
                           porosity=law, porosity_q=q, objective="none")
        o = Oracle(P, np.full((4, 5, 6), c, np.float32))
        U = (0.03, -0.02, 0.01)
        m = o.model
        n = o.n
        u = torch.tensor(U, dtype=torch.float64)[:, None].expand(3, n)
        F = m.feq(torch.ones(n, dtype=torch.float64), u).view(m.Q, *o.shape)
        post = o.collide(F).reshape(m.Q, -1)
        j = m.E.T @ post
        # theta is held in FP32: evaluate G on the stored value
        cf = float(np.float32(c))
        Gf = {"linear": 1 - cf, "power": 1 - cf ** q, "ramp": (1 - cf) / (1 + q * cf)}[law]
        want = Gf * torch.tensor(U, dtype=torch.float64)
        assert (j - want[:, None]).abs().max() < 1e-15, (law, coll, c)


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.0])
def test_scalar_diffusivity_interpolates_in_theta(theta):
    # Sec. 3.2: alpha = (1 - theta) alpha_fluid + theta alpha_solid; a Fourier
    # mode of a pure-diffusion field in a box of uniform theta decays at
    # alpha(theta) k^2 (up to O(k^2) lattice corrections).
    L, a_f, a_s = 32, 0.05, 0.15
    P = inputs.Problem(lattice="D3Q19", dims=(L, 2, 2), walls="", nscalars=1,
                       alpha_fluid=a_f, alpha_solid=a_s, objective="none")
    th = float(np.float32(theta))
    o = Oracle(P, np.full((2, 2, L), theta, np.float32))
    alpha = (1 - th) * a_f + th * a_s
    m = o.model
    F = o.initial().clone()
    k = 2 * math.pi / L
    x = torch.arange(L, dtype=torch.float64)
    F[m.Q:] = (m.ws[:, None] * (0.5 + 0.1 * torch.sin(k * x))[None, :]).view(m.Qs, 1, 1, L)
    nsteps = 200
    with torch.no_grad():
        for _ in range(nsteps):
            F = o.step(F)
    T = F[m.Q:].sum(0)[0, 0]
    amp = float(((T - 0.5) * torch.sin(k * x)).sum() * 2 / L)
    rate = -math.log(amp / 0.1) / nsteps
    assert abs(rate - alpha * k * k) / (alpha * k * k) < 0.02


def test_scalar_diffusion_decay_and_conservation():
    # Pure diffusion (u = 0, periodic): sum T is conserved and a Fourier mode
    # decays at rate alpha k^2 up to O(k^2) lattice corrections.
    L = 32
    alpha = 0.05
    P = inputs.Problem(lattice="D3Q19", dims=(L, 2, 2), walls="", nscalars=1,
                       alpha_fluid=alpha, alpha_solid=alpha, objective="none")
    o = Oracle(P, np.zeros((2, 2, L), np.float32))
    F = o.initial().clone()
    k = 2 * math.pi / L
    x = torch.arange(L, dtype=torch.float64)
    T0 = 0.5 + 0.1 * torch.sin(k * x)
    m = o.model
    F[m.Q:] = (m.ws[:, None] * T0[None, :]).view(m.Qs, 1, 1, L)
    total0 = float(F[m.Q:].sum())
    nsteps = 200
    with torch.no_grad():
        for _ in range(nsteps):
            F = o.step(F)
    T = F[m.Q:].sum(0)[0, 0]
    amp = float(((T - 0.5) * torch.sin(k * x)).sum() * 2 / L)
    rate = -math.log(amp / 0.1) / nsteps
    assert abs(rate - alpha * k * k) / (alpha * k * k) < 0.02
    assert abs(float(F[m.Q:].sum()) - total0) < 1e-12 * total0


def test_uniform_scalar_has_zero_variance():
    P = _mixer_small(scalar_inlet="zero", nscalars=1)
    o = Oracle(P, np.zeros(P.dims[::-1], np.float32))
    F = o.initial().clone()
    m = o.model
    F[m.Q:] = 0.3 * m.ws.view(-1, 1, 1, 1)
    assert abs(float(o.F_obj(F))) < 1e-15


def _uniform_flow_state(o, U, T_of_y=None, rho=1.0):
    """Every node at equilibrium with (rho, u = (U,0,0)) and scalar 0 at T(y)."""
    m = o.model
    n = o.n
    u = torch.zeros(3, n, dtype=torch.float64)
    u[0] = U
    F = torch.zeros(m.M, n, dtype=torch.float64)
    F[:m.Q] = m.feq(torch.full((n,), rho, dtype=torch.float64), u)
    if m.NS:
        T = torch.zeros(n, dtype=torch.float64) if T_of_y is None else T_of_y(o.y.double())
        F[m.Q:m.Q + m.Qs] = m.geq(T, u)
    return F.view(m.M, *o.shape)


@pytest.mark.parametrize("T", [0.0, 0.3, 1.0])
def test_heat_flux_and_mixing_flux_closed_forms(T):
    # Uniform flow u = (U,0,0) at rho = 1 with a uniform scalar T: at the
    # outlet Zou-He gives u_x = U and the outlet scalar T* = T, and at the
    # inlet rho = (s0 + 2 s_out)/(1 - U) = 1 when u_in = U, so Delta p = 0:
    #   Eq. exchanger:obj sum_outlet u_x T = A U T,
    #   Eq. mixing:obj    sum_outlet u_x (1 - T^2) = A U (1 - T^2).
    U = 0.04
    P = inputs.scaled(inputs.exchanger3d(), (12, 7, 6), u_in=U, hot=())
    o = Oracle(P, np.zeros(P.dims[::-1], np.float32))
    F = _uniform_flow_state(o, U, lambda y: torch.full_like(y, T))
    A = o.n_out
    assert abs(float(o.F_obj(F)) - A * U * T) < 1e-13
    Pm = P.replace(objective="mixflux")
    om = Oracle(Pm, np.zeros(P.dims[::-1], np.float32))
    assert abs(float(om.F_obj(F)) - A * U * (1 - T * T)) < 1e-13


def test_heat_flux_pressure_drop_term():
    # A uniform equilibrium state at rho_0 != 1 and u = (U,0,0) with u_in = U
    # gives inlet rho = (s0 + 2 s_out)/(1 - U) = rho_0 (Zou-He), so the
    # pressure term is -0.1 (rho_0 - rho_out)/3; at the outlet Zou-He gives
    # u_x = (s0 + 2 s_out)/rho_out - 1 = rho_0 (1 + U) - 1 for rho_out = 1.
    U, rho0 = 0.03, 1.02
    P = inputs.scaled(inputs.exchanger3d(), (12, 7, 6), u_in=U, hot=())
    o = Oracle(P, np.zeros(P.dims[::-1], np.float32))
    T = 0.5
    F = _uniform_flow_state(o, U, lambda y: torch.full_like(y, T), rho=rho0)
    A = o.n_out
    ux_out = rho0 * (1 + U) - 1.0
    # outlet scalar: unknown populations at equilibrium with T* and v = u_x
    # leave T* = T because the known ones carry equilibrium at the inlet speed U
    m = o.model
    Es = m.sl.E
    known = Es[:, 0] >= 0
    phiU = 1 + Es[:, 0] * U / m.sl.cs2
    phi_out = 1 + Es[:, 0] * ux_out / m.sl.cs2
    Tstar = T * float((m.sl.w * phiU)[known].sum()) / (1 - float((m.sl.w * phi_out)[~known].sum()))
    expect = A * ux_out * Tstar - 0.1 * (rho0 - 1.0) / 3.0
    assert abs(float(o.F_obj(F)) - expect) < 1e-13
    # the heat flux alone (Eq. exchanger:obj) has no pressure term
    oh = Oracle(P.replace(objective="heatflux"), np.zeros(P.dims[::-1], np.float32))
    assert abs(float(oh.F_obj(F)) - A * ux_out * Tstar) < 1e-13


def test_signed_inlet_values_after_collision():
    # the paper's mixer inlet (Sec. 4.1): T = -1 for y < Ly/2 and +1 above;
    # the second scalar carries -T
    P = _mixer_small(collision="BGK", scalar_inlet="signed")
    o = Oracle(P, np.zeros(P.dims[::-1], np.float32))
    F = _rand_state(o, 6, scale=0.01)
    post = o.collide(F).reshape(o.model.M, -1)
    m = o.model
    inl = o.flags == INLET
    T0 = post[m.Q:m.Q + m.Qs].sum(0)
    T1 = post[m.Q + m.Qs:].sum(0)
    c = torch.where(o.y >= P.dims[1] // 2, 1.0, -1.0).double()
    assert (T0[inl] - c[inl]).abs().max() < 1e-14
    assert (T1[inl] + c[inl]).abs().max() < 1e-14


@pytest.mark.parametrize("coll", ["BGK", "MRT"])
def test_signed_inlet_field_is_antisymmetric(coll):
    # The channel, its walls and its inflow are symmetric under y -> Ly-1-y
    # (Ly even) and the signed inlet changes sign under it, so the scalar
    # field (a linear response to the inlet, starting from 0) is odd in y at
    # every step, and its outlet mean vanishes.
    P = inputs.scaled(inputs.mixer3d(), (12, 8, 6), nsteps=30, obj_window=0,
                      collision=coll, scalar_inlet="signed", nscalars=1)
    o = Oracle(P, np.zeros(P.dims[::-1], np.float32))
    _, traj = o.primal(keep=False)
    F = traj[-1]
    m = o.model
    T = F[m.Q:m.Q + m.Qs].sum(0)                       # (Lz, Ly, Lx)
    assert float(T.abs().max()) > 1e-3
    assert float((T + T.flip(1)).abs().max()) < 1e-13


def test_outlet_variance_of_a_two_level_profile():
    # Outlet scalar 0 below y = Ly/2 and 1 above, fluid at rest: the outlet
    # variance is p (1 - p), p the fraction of outlet nodes with value 1.
    P = inputs.scaled(inputs.mixer3d(), (10, 9, 6), obj_window=0)
    o = Oracle(P, np.zeros(P.dims[::-1], np.float32))
    half = P.dims[1] // 2
    F = _uniform_flow_state(o, 0.0, lambda y: (y >= half).double())
    out = (o.flags == 4 - 1)
    ys = o.y[out]
    p = float((ys >= half).double().mean())
    assert abs(float(o.F_obj(F)) - p * (1 - p)) < 1e-14


def test_paper_presets_follow_the_printed_cases():
    # inputs.paper_*_empty carry Tab. tab:cases: sizes, nu (tau = 3 nu + 1/2),
    # the diffusivities, the design span (nodes x_first..x_last) and the
    # pressure drop of the pressure inlet, whose velocity limit is 0.05 (Sec. 4).
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_table_cases.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        c, *v = line.split()
        rows[c] = [float(x) for x in v]
    for case, P in (("mixer", inputs.paper_mixer_empty()), ("exchanger", inputs.paper_exchanger_empty())):
        Lx, Ly, Lz, x0, x1, dp, nu, a_f, a_s = rows[case]
        assert tuple(P.dims) == (int(Lx), int(Ly), int(Lz))
        assert abs(P.tau - (3 * nu + 0.5)) < 1e-12
        assert P.alpha_fluid == a_f and P.alpha_solid == a_s
        assert P.design[0] == int(x0) and P.design[1] == int(x1) + 1
        assert P.u_in == 0.05 and P.collision == "MRT" and P.nscalars == 1
        assert P.inlet == "pressure" and P.dp == dp and P.rho_out == 1.0



# ---------------------------------------------------------------------------
# time weights of the window objective, outlet scalar reconstruction
# ---------------------------------------------------------------------------

def _ghost_mode(lattice, dims, tau, eps):
    """A spatially uniform non-equilibrium state of a fully periodic box:
    f_i = w_i (1 + eps (e_ix^2 - e_iy^2)).  The perturbation carries no
    mass and no momentum, so rho = 1 and u = 0 at every node; streaming a
    uniform field changes nothing, and BGK without force or porosity scales
    f - f_eq by (1 - omega) per step.  Hence f^n - f_eq = (1 - omega)^n
    (f^0 - f_eq) exactly, and the stress Pi_ab = sum_i e_ia e_ib (f_i - f_eq,i)
    is diag(2/9, -2/9, 0) eps (1 - omega)^n on D2Q9 and D3Q19 (sum w e_x^4 =
    1/3, sum w e_x^2 e_y^2 = 1/9 on both).  The dissipation 2 rho nu S:S with
    S = -(3 omega / 2) Pi is then (4/9) nu omega^2 eps^2 (1 - omega)^(2n) per
    node."""
    P = inputs.Problem(lattice=lattice, dims=dims, collision="BGK", tau=tau, walls="",
                       channel="periodic", objective="dissipation")
    o = Oracle(P, np.zeros(dims[::-1], np.float32))
    m = o.model
    E = m.E.numpy()
    h = torch.tensor(E[:, 0] ** 2 - E[:, 1] ** 2, dtype=torch.float64)
    F = (m.w * (1 + eps * h))[:, None].expand(m.Q, o.n).clone().view(m.Q, *o.shape)
    omega = 1.0 / tau
    nu = (tau - 0.5) / 3.0
    F0 = o.n * 4.0 / 9.0 * nu * omega ** 2 * eps ** 2

    def closed(n):
        return F0 * (1.0 - omega) ** (2 * n)
    return P, o, F, closed


@pytest.mark.parametrize("lattice,dims", [("D2Q9", (6, 5, 1)), ("D3Q19", (4, 3, 5))])
@pytest.mark.parametrize("N,K", [(7, 0), (7, 3), (6, 1), (5, 6)])
def test_window_objective_is_the_mean_of_the_last_K_steps(lattice, dims, N, K):
    # J = sum_n c_n F(f^n) with c_n = 1/K on n = N-K+1 .. N (K > 0), or the
    # final step alone (K = 0), against the closed-form F(f^n) of the ghost
    # mode: a window of K+1 terms, a weight 1/(K+1) or a shifted window
    # fails it.  Both weight constructions of the oracle are checked (the
    # problem's horizon and an explicit one).
    tau = 0.7
    P, o, F, closed = _ghost_mode(lattice, dims, tau, eps=0.03)
    for n in range(3):                     # the closed form itself, step by step
        assert abs(float(o.F_obj(F)) - closed(n)) <= 1e-12 * closed(0)
        with torch.no_grad():
            F = o.step(F)
    want = closed(N) if K == 0 else sum(closed(n) for n in range(N - K + 1, N + 1)) / K
    _, o, F0, _ = _ghost_mode(lattice, dims, tau, eps=0.03)
    o.P = P.replace(nsteps=N, obj_window=K)
    o.model.P = o.P
    J_model, _ = o.primal(F0=F0, keep=False)              # weights of the problem (Model.weights)
    J_explicit, _ = o.primal(nsteps=N, F0=F0, keep=False)  # weights of an explicit horizon
    assert abs(J_model - want) <= 1e-12 * want
    assert abs(J_explicit - want) <= 1e-12 * want


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_outlet_scalar_reconstruction_worked_example(lattice):
    # One outlet node, fluid at equilibrium with u = (0.05, 0, 0) so that
    # the Zou-He outlet (rho_out = 1) returns v = u.  The scalar populations
    # that stream in from the interior (e_x >= 0) are set by hand to values
    # summing to S = 0.45; the ones with e_x < 0, which would stream in from
    # outside the box, hold garbage (7.0 each).  The outlet condition puts
    # the unknowns at equilibrium with the node's own value T*, w_i T*
    # (1 + e_i.v / cs2), and T* must be the zeroth moment of the
    # reconstructed populations: T* = S + T* sum_unknown w_i (1 - 0.05 /
    # cs2).  D3Q7 (cs2 = 1/4, one unknown of weight 1/8):
    # T* = 0.45 / (1 - 0.8 / 8) = 0.5 exactly.  D2Q9 scalar (cs2 = 1/3,
    # unknown weights 1/9, 1/36, 1/36): T* = 0.45 / (1 - 0.85 / 6).  A
    # reconstruction that takes T* = sum g (here 0.45 + garbage) fails.
    is3d = lattice == "D3Q19"
    P = inputs.Problem(lattice=lattice, dims=(3, 1, 1), collision="BGK", tau=0.8, walls="",
                       channel="inlet_outlet", u_in=0.05, rho_out=1.0, nscalars=1,
                       alpha_fluid=0.1, alpha_solid=0.1, objective="heatflux")
    o = Oracle(P, np.zeros((1, 1, 3), np.float32))
    m = o.model
    ux = 0.05
    E = m.E.numpy()
    w = m.w.numpy()
    eu = E[:, 0] * ux
    f = w * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * ux ** 2)
    Es = m.sl.E
    known = np.nonzero(Es[:, 0] >= 0)[0]
    unk = np.nonzero(Es[:, 0] < 0)[0]
    g = np.full(m.Qs, 7.0)
    vals = [0.02, 0.05, 0.08, 0.11, 0.06, 0.09, 0.04, 0.0, 0.0][:len(known)]
    vals[-1] += 0.45 - sum(vals)
    g[known] = vals
    F = torch.tensor(np.concatenate([f, g]), dtype=torch.float64)[:, None]
    flags = torch.tensor([OUTLET])
    mac = m.macroscopic(F, torch.zeros(1, dtype=torch.float64), flags)
    v = mac["v"][:, 0].numpy()
    assert abs(v[0] - ux) <= 1e-15 and abs(v[1]) <= 1e-15 and abs(v[2]) <= 1e-15
    T_star = 0.5 if is3d else 0.45 / (1 - 0.85 / 6)
    assert abs(float(mac["T"][0][0]) - T_star) <= 1e-14
    gr = mac["gr"][0][:, 0].numpy()
    np.testing.assert_allclose(gr[known], g[known], rtol=0, atol=0)
    cs2 = 0.25 if is3d else 1.0 / 3.0
    want_unk = m.sl.w[unk] * T_star * (1 - ux / cs2)
    np.testing.assert_allclose(gr[unk], want_unk, rtol=0, atol=1e-15)
    # the heat flux of this node is v_x T*
    assert abs(float(o.model.objective(F, torch.zeros(1, dtype=torch.float64), flags,
                                       torch.zeros(1, dtype=torch.long))) - ux * T_star) <= 1e-15


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_pressure_inlet_prescribed_values(lattice):
    # Zou-He pressure inlet with the velocity cap of Sec. 4, at one node whose
    # incoming populations are those of the equilibrium at rho = 1.02, u =
    # (0.03, 0, 0): mass and normal momentum give s0 + 2 s_out = rho (1 - u)
    # = 0.9894.  With dp = 0.03 (rho_in = 1.09) the pressure condition would
    # give u = 1 - 0.9894 / 1.09 = 0.0923 > 0.05, so the node is a velocity
    # inlet at the cap: u = 0.05, rho = 0.9894 / 0.95.  With dp = 0.001
    # (rho_in = 1.003) it stays a pressure inlet: rho = 1.003, u = 1 -
    # 0.9894 / 1.003.  Either way the reconstructed node carries that mass
    # and normal momentum, with no transverse momentum.
    dims = (3, 1, 1)
    for dp, rho_want, u_want in ((0.03, 0.9894 / 0.95, 0.05),
                                 (0.001, 1.003, 1.0 - 0.9894 / 1.003)):
        P = inputs.Problem(lattice=lattice, dims=dims, collision="BGK", tau=0.8, walls="",
                           channel="inlet_outlet", inlet="pressure", dp=dp, u_in=0.05,
                           rho_out=1.0, objective="none")
        o = Oracle(P, np.zeros(dims[::-1], np.float32))
        m = o.model
        E = m.E.numpy()
        eu = E[:, 0] * 0.03
        f = 1.02 * m.w.numpy() * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * 0.03 ** 2)
        F = torch.tensor(f, dtype=torch.float64)[:, None]
        mac = m.macroscopic(F, torch.zeros(1, dtype=torch.float64), torch.tensor([INLET]))
        fr = mac["fr"][:, 0].numpy()
        assert abs(fr.sum() - rho_want) <= 1e-14
        assert abs((E[:, 0] * fr).sum() - rho_want * u_want) <= 1e-14
        assert abs((E[:, 1] * fr).sum()) <= 1e-15 and abs((E[:, 2] * fr).sum()) <= 1e-15
        assert abs(float(mac["rho"][0]) - rho_want) <= 1e-14
        assert abs(float(mac["u"][0, 0]) - u_want) <= 1e-14


def test_pressure_driven_channel_carries_the_inlet_density():
    # a short pressure-driven channel below the cap: every inlet node holds
    # rho_in exactly after its reconstruction, and the flow runs from the
    # inlet to the outlet
    P = inputs.Problem(lattice="D3Q19", dims=(16, 7, 7), collision="BGK", tau=0.8, walls="yz",
                       channel="inlet_outlet", inlet="pressure", dp=0.002, u_in=0.05,
                       rho_out=1.0, objective="none", nsteps=200)
    o = Oracle(P, np.zeros((7, 7, 16), np.float32))
    _, traj = o.primal(keep=False)
    F = traj[-1].reshape(o.model.M, -1)
    mac = o.model.macroscopic(F, o.theta, o.flags)
    inl = (o.flags == INLET) & (mac["u"][0] <= P.u_in)
    assert int(inl.sum()) > 0
    assert float((mac["rho"][inl] - (1.0 + 3 * P.dp)).abs().max()) <= 1e-12
    fl = o.flags == FLUID
    assert float(mac["u"][0][fl].mean()) > 0.0
