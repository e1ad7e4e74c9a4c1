"""Seeded synthetic workloads shared by the CUDA path and the FP64 oracle.

This module holds problem *descriptions* and seeded random inputs only: it
contains none of the method's arithmetic (no equilibria, no collision, no
streaming, no objective).  Both implementations read a :class:`Problem` and
build their own node flags, tables and initial states from it.

Workloads follow the paper's two channel test cases (Sec. 4, Tab. "tab:cases")
and the synthetic stand-ins derived from them:

* ``channel2d``  - D2Q9 BGK channel 128x64, body force, bounce-back walls on
  y, periodic x, porosity on a central 32x32 design block; viscous dissipation.
* ``mixer3d``    - D3Q19 MRT square-channel mixer 256x128x128 with two D3Q7
  passive scalars (inlet halves c=0/1 and the complement), velocity inlet,
  pressure outlet; outlet scalar variance averaged over the last 500 steps
  (Sec. 4.1, Eq. "mixing:obj" is offered as ``mixflux``).
* ``exchanger3d`` - D3Q19 BGK + D3Q7 temperature heat exchanger 512x256x256,
  hot bottom patch T=1, inlet T=0, Pr=0.7; outlet heat flux minus 0.1 times
  the pressure drop (Sec. 4.2, Eq. "exchanger:obj").
* ``paper_mixer_empty``, ``paper_exchanger_empty`` - the paper's own empty
  channels (450x50x50 and 352x50x50, Tab. "tab:cases") for comparison with
  its printed results.
* ``batch_instances``, ``serving_requests`` - seeded families of instances
  and timed requests for the batched and served forms.

Porosity naming: ``theta`` is the solid fraction (0 = fluid, 1 = solid), i.e.
``theta = 1 - w`` with the paper's ``w`` of Sec. 3.2.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Problem:
    """Plain description of one adjoint-LBM problem (no arithmetic)."""

    lattice: str = "D2Q9"            # "D2Q9" | "D3Q19" (fluid lattice, Sec. 3)
    dims: tuple = (128, 64, 1)       # (Lx, Ly, Lz); Lz == 1 for 2D
    collision: str = "BGK"           # "BGK" (Eq. SRT) | "MRT" (Sec. 3.1)
    tau: float = 0.8                 # 1/omega = tau = 0.5 + 3 nu (Sec. 3.1)
    s_other: float = 1.2             # MRT rate of non-stress, non-conserved moments
    force: tuple = (0.0, 0.0, 0.0)   # body acceleration g (EDM forcing, Sec. 3.1)
    walls: str = "y"                 # axes carrying bounce-back wall planes at both ends
    channel: str = "periodic"        # "periodic" in x | "inlet_outlet" (Zou-He x faces)
    inlet: str = "velocity"          # "velocity": u = u_in | "pressure": rho = rho_out + 3 dp
    #                                  with the inlet velocity capped at u_in (Sec. 4)
    dp: float = 0.0                  # pressure drop of a pressure inlet (lattice units)
    u_in: float = 0.05               # velocity inlet speed (x = 0 face), or its cap
    rho_out: float = 1.0             # pressure outlet density (x = Lx-1 face)
    nscalars: int = 0                # passive scalar lattices (D3Q7 in 3D, D2Q9 in 2D)
    alpha_fluid: float = 0.0         # scalar diffusivity in fluid (theta = 0)
    alpha_solid: float = 0.0         # scalar diffusivity in solid (theta = 1)
    scalar_inlet: str = "zero"       # "zero" | "halves" (c = 0 for y < Ly/2, else 1)
    #                                  | "signed" (-1 for y < Ly/2, else +1)
    hot: tuple = ()                  # (x0, x1, z0, z1): y = 0 wall nodes with T = T_hot
    T_hot: float = 1.0
    porosity: str = "linear"         # G(theta): "linear" 1-theta | "power" 1-theta^q | "ramp"
    porosity_q: float = 1.0
    objective: str = "dissipation"   # "none"|"dissipation"|"variance"|"heatflux_dp"|"mixflux"|"heatflux"
    obj_window: int = 0              # 0: J = F(f^N); K > 0: mean of F(f^n), N-K < n <= N
    nsteps: int = 2000               # horizon N of the unsteady problem
    design: tuple = (48, 80, 16, 48, 0, 1)   # (x0, x1, y0, y1, z0, z1) design box
    precision: str = "fp32"          # population storage on the GPU: fp32 | bf16 | fp16
    ckpt_every: int = 0              # level-1 checkpoint stride of the adjoint schedule
    kernel: str = "auto"             # GPU step kernels: auto | plain | tiles (staged rows)
    adjoint_mode: str = "unsteady"   # "unsteady" (exact gradient over the horizon) | "frozen"
    #                                  (the paper's fixed-point ALBS at f^N, Sec. 2.2)

    @property
    def n_nodes(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])

    @property
    def is3d(self) -> bool:
        return self.lattice == "D3Q19"

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# Workload presets (parameters only)
# ---------------------------------------------------------------------------

def channel2d(**kw) -> Problem:
    """D2Q9 BGK channel 128x64, tau=0.8, g=(1e-5,0), walls y, periodic x."""
    p = Problem(lattice="D2Q9", dims=(128, 64, 1), collision="BGK", tau=0.8,
                force=(1e-5, 0.0, 0.0), walls="y", channel="periodic",
                objective="dissipation", obj_window=0, nsteps=2000,
                design=(48, 80, 16, 48, 0, 1))
    return p.replace(**kw)


def channel3d(**kw) -> Problem:
    """The config-1 channel in 3D: D3Q19 BGK 128x64x64, tau=0.8, body force
    g=(1e-5,0,0), bounce-back walls on y and z, periodic x, porosity on a
    central box; viscous dissipation.  The flow rate adapts to the porous
    resistance, so any theta field gives a bounded state."""
    p = Problem(lattice="D3Q19", dims=(128, 64, 64), collision="BGK", tau=0.8,
                force=(1e-5, 0.0, 0.0), walls="yz", channel="periodic",
                objective="dissipation", obj_window=0, nsteps=2000,
                design=(48, 80, 16, 48, 16, 48))
    return p.replace(**kw)


def mixer3d(**kw) -> Problem:
    """D3Q19 MRT mixer 256x128x128 + two D3Q7 scalars, tau=0.6.

    The scalar diffusivity is alpha = nu (Schmidt number 1) in both phases
    (alpha_solid = alpha_fluid, as in the paper's mixer).  The paper's own
    ratio nu/alpha = 0.02/0.003 puts the D3Q7 relaxation time at 0.52, and
    with theta ~ U[0,1] filling the design box the flow squeezes around it
    at |u| up to about 0.25 = c_s^2 of D3Q7; the scalar then diverges within
    2000 steps, while alpha = nu (tau_T = 0.633) stays within [0, 1.09]
    over the 10000 steps.
    """
    tau = 0.6
    nu = (tau - 0.5) / 3.0
    alpha = nu
    Lx, Ly, Lz = 256, 128, 128
    p = Problem(lattice="D3Q19", dims=(Lx, Ly, Lz), collision="MRT", tau=tau,
                walls="yz", channel="inlet_outlet", u_in=0.05, rho_out=1.0,
                nscalars=2, alpha_fluid=alpha, alpha_solid=alpha,
                scalar_inlet="halves", objective="variance", obj_window=500,
                nsteps=10000, design=(64, 192, 16, 112, 16, 112), ckpt_every=500)
    return p.replace(**kw)


def exchanger3d(**kw) -> Problem:
    """D3Q19 BGK + D3Q7 temperature heat exchanger 512x256x256, tau=0.55.

    Pr = nu/alpha_fluid = 0.7, alpha_solid = 1 (Tab. "tab:cases"); the D x D
    hot plate sits on the bottom wall in the middle of the channel and the
    design region is the middle 3/7 of the length (Sec. 4.2).
    """
    tau = 0.55
    nu = (tau - 0.5) / 3.0
    Lx, Ly, Lz = 512, 256, 256
    x0 = Lx // 2 - Ly // 2
    p = Problem(lattice="D3Q19", dims=(Lx, Ly, Lz), collision="BGK", tau=tau,
                walls="yz", channel="inlet_outlet", u_in=0.05, rho_out=1.0,
                nscalars=1, alpha_fluid=nu / 0.7, alpha_solid=1.0,
                scalar_inlet="zero", hot=(x0, x0 + Ly, 0, Lz), T_hot=1.0,
                objective="heatflux_dp", obj_window=0, nsteps=1000,
                design=(2 * Lx // 7, 5 * Lx // 7, 1, Ly - 1, 1, Lz - 1))
    return p.replace(**kw)


def paper_mixer_empty(**kw) -> Problem:
    """The paper's mixing channel without obstacle (Tab. tab:cases, Sec. 4.1):
    D3Q19 MRT 450x50x50, nu = 0.02 (tau = 0.56), one D3Q7 scalar with
    alpha = 0.003 in both phases, inlet T = -1 for y < 25 and +1 above,
    objective the outlet mixing flux of Eq. mixing:obj, theta = 0.  Driven
    by the pressure drop 0.016666 between inlet and outlet (Sec. 4), with
    the inlet velocity limited to 0.05.  40 000 steps (the iterations
    Tab. tab:results lists for the empty mixer)."""
    nu = 0.02
    p = Problem(lattice="D3Q19", dims=(450, 50, 50), collision="MRT", tau=3 * nu + 0.5,
                walls="yz", channel="inlet_outlet", inlet="pressure", dp=0.016666,
                u_in=0.05, rho_out=1.0,
                nscalars=1, alpha_fluid=0.003, alpha_solid=0.003, scalar_inlet="signed",
                objective="mixflux", obj_window=0, nsteps=40000,
                design=(61, 391, 1, 49, 1, 49), ckpt_every=0)
    return p.replace(**kw)


def paper_exchanger_empty(**kw) -> Problem:
    """The paper's heat-exchanger channel without obstacle (Tab. tab:cases,
    Sec. 4.2): D3Q19 MRT 352x50x50, nu = 0.01 (tau = 0.53), one D3Q7
    temperature with alpha = 0.003 in the fluid and 1 in the solid, inlet
    T = 0, a D x D plate at T = 1 on the bottom wall in the middle, objective
    the outlet heat flux of Eq. exchanger:obj, theta = 0.  Driven by the
    pressure drop 0.03 (Sec. 4) with the inlet velocity limited to 0.05;
    30 000 steps (Tab. tab:results)."""
    nu = 0.01
    Lx, Ly, Lz = 352, 50, 50
    x0 = Lx // 2 - Ly // 2
    p = Problem(lattice="D3Q19", dims=(Lx, Ly, Lz), collision="MRT", tau=3 * nu + 0.5,
                walls="yz", channel="inlet_outlet", inlet="pressure", dp=0.03,
                u_in=0.05, rho_out=1.0,
                nscalars=1, alpha_fluid=0.003, alpha_solid=1.0, scalar_inlet="zero",
                hot=(x0, x0 + Ly, 0, Lz), T_hot=1.0, objective="heatflux", obj_window=0,
                nsteps=30000, design=(101, 253, 1, 49, 1, 49), ckpt_every=0)
    return p.replace(**kw)


def scaled(p: Problem, dims, nsteps=None, **kw) -> Problem:
    """The same physics on another lattice size (design box and hot patch scaled)."""
    Lx0, Ly0, Lz0 = p.dims
    Lx, Ly, Lz = dims
    d = p.design

    def sx(a):
        return int(round(a * Lx / Lx0))

    def sy(a):
        return int(round(a * Ly / Ly0))

    def sz(a):
        return int(round(a * Lz / Lz0)) if Lz0 > 1 else a

    design = (sx(d[0]), max(sx(d[1]), sx(d[0]) + 1), sy(d[2]), max(sy(d[3]), sy(d[2]) + 1),
              sz(d[4]), max(sz(d[5]), sz(d[4]) + 1))
    hot = p.hot
    if hot:
        hot = (sx(hot[0]), sx(hot[1]), sz(hot[2]), sz(hot[3]))
    out = p.replace(dims=tuple(int(v) for v in dims), design=design, hot=hot)
    if nsteps is not None:
        out = out.replace(nsteps=int(nsteps))
    return out.replace(**kw)


# ---------------------------------------------------------------------------
# Seeded porosity fields (FP32, the same bytes go to both implementations)
# ---------------------------------------------------------------------------

def fins_theta(p: Problem, n: int, width: int, min_gap: int = 3) -> np.ndarray:
    """The finned exchanger of Sec. 4.2: `n` evenly spaced parallel plates of
    thickness `width` (z) standing on the heating plate, spanning its length
    (x over the hot patch) and the channel's interior height (y); theta = 1
    (solid, with the solid diffusivity) on the plates, 0 elsewhere.  Raises
    ValueError when the gaps between the plates and the walls fall below
    `min_gap` nodes.  Returns float32 (Lz, Ly, Lx)."""
    Lx, Ly, Lz = p.dims
    if not p.hot:
        raise ValueError("the finned exchanger needs a hot patch")
    x0, x1 = p.hot[0], p.hot[1]
    span = Lz - 2                                  # interior nodes across z
    gap = (span - n * width) / (n + 1)
    if n < 1 or width < 1 or gap < min_gap:
        raise ValueError(f"{n} fins of width {width} leave gaps of {gap:.2f} < {min_gap}")
    th = np.zeros((Lz, Ly, Lx), dtype=np.float32)
    for k in range(n):
        z0 = 1 + int(round(gap * (k + 1) + width * k))
        th[z0:z0 + width, 1:Ly - 1, x0:x1] = 1.0
    return th


def fin_sweep(p: Problem, counts=range(1, 8), widths=range(3, 11), min_gap: int = 3):
    """(n, width) pairs of the fin study of Sec. 4.2 that keep the gaps."""
    out = []
    for n in counts:
        for w in widths:
            if (p.dims[2] - 2 - n * w) / (n + 1) >= min_gap:
                out.append((n, w))
    return out


def design_mask(p: Problem) -> np.ndarray:
    """Boolean (Lz, Ly, Lx) mask of the design box."""
    Lx, Ly, Lz = p.dims
    x0, x1, y0, y1, z0, z1 = p.design
    m = np.zeros((Lz, Ly, Lx), dtype=bool)
    m[max(z0, 0):min(z1, Lz), max(y0, 0):min(y1, Ly), max(x0, 0):min(x1, Lx)] = True
    return m


def theta_uniform(p: Problem, seed: int) -> np.ndarray:
    """theta ~ U[0,1] on the design box, 0 elsewhere; float32 (Lz, Ly, Lx)."""
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = p.dims
    th = np.zeros((Lz, Ly, Lx), dtype=np.float32)
    m = design_mask(p)
    th[m] = rng.random(int(m.sum()), dtype=np.float64).astype(np.float32)
    return th


def theta_grf(p: Problem, seed: int, sigma: float = 4.0) -> np.ndarray:
    """Smoothed Gaussian random field in [0,1] on the design box.

    White noise filtered by a Gaussian of width ``sigma`` lattice units (FFT,
    periodic), min-max rescaled to [0,1] over the design box in FP64, then cast
    to float32 once.  Zero outside the design box.
    """
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = p.dims
    noise = rng.standard_normal((Lz, Ly, Lx))
    kz = np.fft.fftfreq(Lz)[:, None, None]
    ky = np.fft.fftfreq(Ly)[None, :, None]
    kx = np.fft.fftfreq(Lx)[None, None, :]
    k2 = (2 * math.pi) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2)
    field_ = np.real(np.fft.ifftn(np.fft.fftn(noise) * np.exp(-0.5 * sigma ** 2 * k2)))
    m = design_mask(p)
    th = np.zeros((Lz, Ly, Lx), dtype=np.float32)
    if m.any():
        v = field_[m]
        lo, hi = float(v.min()), float(v.max())
        th[m] = ((v - lo) / max(hi - lo, 1e-300)).astype(np.float32)
    return th


def random_state(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded float64 normal array (for duality tests and random adjoints)."""
    return np.random.default_rng(seed).standard_normal(shape) * scale


# ---------------------------------------------------------------------------
# Batched and served workloads
# ---------------------------------------------------------------------------

def batch_instances(count: int = 64, seed: int = 0, size_scale: float = 1.0,
                    steps=(1000, 5000)):
    """Seeded mixed batch: a coin picks the D2Q9 channel (config-1 geometry,
    aspect 2:1, sizes log-uniform 64^2..1024^2 nodes) or its 3D analogue
    ``channel3d`` (D3Q19 BGK, aspect 2:1:1, sizes log-uniform 48^3..192^3
    nodes); steps uniform in ``steps``; theta ~ U[0,1] on each design box
    (seed ``seed + i``).  ``size_scale`` shrinks the linear sizes (tests).
    Returns a list of (Problem, theta).

    The 3D instances are body-force driven.  The velocity-inlet channels do
    not suit random designs at these sizes and horizons: in the heat
    exchanger the design region spans the cross-section, blocks the flow and
    the upstream density grows by about u_in / L_upstream per step (no
    steady state); in the mixer scaled below ~100 nodes across, the bypass
    gaps are a few nodes wide and the jets through them diverge."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        steps_i = int(rng.integers(steps[0], steps[1] + 1))
        if rng.random() < 0.5:
            area = math.exp(rng.uniform(math.log(64 ** 2), math.log(1024 ** 2)))
            Ly = max(8, int(round(math.sqrt(area / 2.0) * size_scale)))
            P = scaled(channel2d(), (2 * Ly, Ly, 1), nsteps=steps_i)
        else:
            vol = math.exp(rng.uniform(math.log(48 ** 3), math.log(192 ** 3)))
            m = max(8, int(round((vol / 2.0) ** (1.0 / 3.0) * size_scale)))
            P = scaled(channel3d(), (2 * m, m, m), nsteps=steps_i)
        out.append((P, theta_uniform(P, seed + i)))
    return out


def serving_requests(count: int, rate: float, seed: int = 0, node_range=(1e4, 3e7),
                     steps=(500, 5000)):
    """Poisson-arriving sensitivity requests: arrival times (s) with mean
    rate ``rate``/s; D2Q9 channel or D3Q19 channel at 50/50 (the geometries
    of ``batch_instances``); node counts log-uniform in
    ``node_range`` factored to aspect 2:1 (2D) or 2:1:1 (3D); steps uniform
    in ``steps``.  Returns a list of (arrival_s, Problem, theta)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        nodes = math.exp(rng.uniform(math.log(node_range[0]), math.log(node_range[1])))
        steps_i = int(rng.integers(steps[0], steps[1] + 1))
        if rng.random() < 0.5:
            Ly = max(8, int(round(math.sqrt(nodes / 2.0))))
            P = scaled(channel2d(), (2 * Ly, Ly, 1), nsteps=steps_i)
        else:
            m = max(8, int(round((nodes / 2.0) ** (1.0 / 3.0))))
            P = scaled(channel3d(), (2 * m, m, m), nsteps=steps_i)
        out.append((t, P, theta_uniform(P, seed * 100003 + i)))
    return out
