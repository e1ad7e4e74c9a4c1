"""Pins of the oracle's lattices and MRT bases against what the paper and the
mathematics fix (no GPU)."""
import itertools
import os

import numpy as np
import pytest
import torch

from oracle.lattice import Lattice, moment_basis
from oracle.model import Model
from paper_1501_04741_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_d3q19_matches_paper_list():
    # Sec. 3 prints e1..e19 explicitly.
    E = _golden("d3q19_velocities.txt").astype(np.int64)
    assert (Lattice("D3Q19").E == E).all()
    # "For the heat transfer equation we use the first 7 of the above."
    assert (Lattice("D3Q7").E == E[:7]).all()
    # 2D: reduced to 9 vectors (the z = 0 members, kept in paper order)
    assert (Lattice("D2Q9").E == E[[0, 1, 2, 3, 4, 7, 8, 9, 10]]).all()


def test_dof_per_node_matches_paper_tables():
    # Tab. "tab:cases" and Sec. 4.3 print nodes and DoF; D3Q19 + D3Q7 = 26.
    rows = _golden("paper_counts.txt")
    P = inputs.exchanger3d()
    M = Model(P.replace(dims=(4, 4, 4))).M
    assert M == 26
    for Lx, Ly, Lz, dof, unit in rows:
        # M densities per node, truncated to the printed digit
        assert 0 <= Lx * Ly * Lz * M - dof < unit


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q7"])
def test_weights_isotropy(name):
    lat = Lattice(name)
    w, E = lat.w, lat.E.astype(np.float64)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs((w[:, None] * E).sum(0)).max() < 1e-15
    dim = 2 if name == "D2Q9" else 3
    second = np.einsum("i,ia,ib->ab", w, E, E)
    assert np.abs(second[:dim, :dim] - lat.cs2 * np.eye(dim)).max() < 1e-15
    # third moments vanish
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, E, E, E)).max() < 1e-15
    if name != "D3Q7":
        # fourth-order isotropy of the fluid lattices (needed by the
        # second-order equilibrium): sum w e_a e_b e_c e_d = cs^4 (dd + dd + dd)
        fourth = np.einsum("i,ia,ib,ic,id->abcd", w, E, E, E, E)
        d = np.eye(3)
        iso = lat.cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                              + np.einsum("ad,bc->abcd", d, d))
        sl = slice(0, dim)
        assert np.abs(fourth[sl, sl, sl, sl] - iso[sl, sl, sl, sl]).max() < 1e-15


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D3Q7"])
def test_opposites(name):
    lat = Lattice(name)
    assert (lat.opp[lat.opp] == np.arange(lat.Q)).all()
    assert (lat.E[lat.opp] == -lat.E).all()


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_moment_basis_orthogonal_and_conserved_rows(name):
    lat = Lattice(name)
    U, conserved, stress = moment_basis(lat)
    G = U @ U.T
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-12
    assert np.linalg.matrix_rank(U) == lat.Q
    # conserved rows are density and momentum
    assert np.allclose(U[conserved[0]], 1.0)
    for a, r in enumerate(conserved[1:]):
        assert np.allclose(U[r], lat.E[:, a])
    # the stress rows span the traceless second moments
    dim = 2 if name == "D2Q9" else 3
    E = lat.E.astype(np.float64)
    sec = []
    for a, b in itertools.product(range(dim), range(dim)):
        sec.append(E[:, a] * E[:, b])
    sec = np.array(sec)
    for r in stress:
        # each stress row is a combination of second moments with zero trace
        coef, *_ = np.linalg.lstsq(sec.T, U[r], rcond=None)
        assert np.abs(sec.T @ coef - U[r]).max() < 1e-12
        assert abs(sum(coef[a * dim + a] for a in range(dim))) < 1e-12


def _random_nodes(model, n, seed, scale=0.01):
    rng = np.random.default_rng(seed)
    F = np.zeros((model.M, n))
    F[:model.Q] = model.fl.w[:, None] * (1 + scale * rng.standard_normal((model.Q, n)))
    if model.NS:
        F[model.Q:] = 0.05 * rng.random((model.M - model.Q, n))
    return torch.tensor(F)


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_mrt_with_T_equal_omega_is_bgk(lattice):
    # Sec. 3.1: with T = omega I the MRT collision reduces to Eq. SRT.
    base = dict(lattice=lattice, dims=(4, 4, 4 if lattice == "D3Q19" else 1), walls="",
                force=(2e-4, -1e-4, 0.0 if lattice == "D2Q9" else 3e-4), tau=0.7)
    Pm = inputs.Problem(collision="MRT", s_other=1 / 0.7, **base)
    Pb = inputs.Problem(collision="BGK", **base)
    mm, mb = Model(Pm), Model(Pb)
    n = 64
    F = _random_nodes(mm, n, 1)
    theta = torch.tensor(np.random.default_rng(2).random(n))
    flags = torch.zeros(n, dtype=torch.int64)
    y = torch.zeros(n, dtype=torch.int64)
    # conserved-moment rates do not matter (their non-equilibrium part is zero)
    mm.I_minus_T = torch.full_like(mm.I_minus_T, 1 - 1 / 0.7)
    a = mm.collide(F, theta, flags, y)
    b = mb.collide(F, theta, flags, y)
    assert (a - b).abs().max().item() < 1e-14


@pytest.mark.parametrize("coll", ["BGK", "MRT"])
@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q19"])
def test_collision_conserves_mass_and_forced_momentum(coll, lattice):
    P = inputs.Problem(lattice=lattice, collision=coll, dims=(4, 4, 4 if lattice == "D3Q19" else 1),
                       walls="", force=(1e-4, 2e-4, 0.0), tau=0.65)
    m = Model(P)
    n = 50
    F = _random_nodes(m, n, 3)
    theta = torch.tensor(np.random.default_rng(4).random(n))
    flags = torch.zeros(n, dtype=torch.int64)
    W = m.collide(F, theta, flags, torch.zeros(n, dtype=torch.int64))
    f, Wf = F[:m.Q], W[:m.Q]
    rho = f.sum(0)
    assert (Wf.sum(0) - rho).abs().max() < 1e-15
    # Exact-Difference forcing with Darcy damping: rho u_post = rho (G u + g)
    u = (m.E.T @ f) / rho
    v = (1 - theta) * u + m.g[:, None]
    assert ((m.E.T @ Wf) - rho * v).abs().max() < 1e-15
