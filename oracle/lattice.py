"""Velocity sets, weights and MRT moment bases (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

* D3Q19 is the list e1..e19 of Sec. 3 in the paper's order (index 0 = e1 =
  rest vector).
* D3Q7 is e1..e7, the first seven vectors of that list (Sec. 3).
* D2Q9 is the set of z = 0 members of the D3Q19 list in paper order,
  {e1, e2, e3, e4, e5, e8, e9, e10, e11} (Sec. 3 reduces the set to nine
  vectors in 2D).
* Weights are the standard ones of each set (the paper does not print them):
  D2Q9 4/9, 1/9, 1/36; D3Q19 1/3, 1/18, 1/36 (c_s^2 = 1/3); D3Q7 1/4, 1/8
  (c_s^2 = 1/4).  Tests pin them by the isotropy conditions.
* ``opp`` is found by search, not tabulated.
* MRT bases: the D3Q19 orthogonal polynomial basis of d'Humieres et al. 2002
  (the matrix Sec. 3.1 cites) and the D2Q9 basis of Lallemand & Luo 2000,
  written as polynomials of the velocity components.
"""
from __future__ import annotations

import numpy as np

# e1 .. e19 of Sec. 3, in the paper's order.
_E19 = np.array([
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, 1, 0), (1, -1, 0), (-1, -1, 0),
    (1, 0, 1), (-1, 0, 1), (1, 0, -1), (-1, 0, -1),
    (0, 1, 1), (0, -1, 1), (0, 1, -1), (0, -1, -1),
], dtype=np.int64)


class Lattice:
    """A velocity set with weights, sound speed and opposite directions."""

    def __init__(self, name: str):
        self.name = name
        if name == "D3Q19":
            E = _E19.copy()
            wmap = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}
            cs2 = 1.0 / 3.0
        elif name == "D2Q9":
            # z = 0 members of the D3Q19 list, kept in paper order
            E = np.array([e for e in _E19 if e[2] == 0], dtype=np.int64)
            wmap = {0: 4.0 / 9.0, 1: 1.0 / 9.0, 2: 1.0 / 36.0}
            cs2 = 1.0 / 3.0
        elif name == "D3Q7":
            E = _E19[:7].copy()
            wmap = {0: 1.0 / 4.0, 1: 1.0 / 8.0}
            cs2 = 1.0 / 4.0
        else:
            raise ValueError(f"unknown lattice {name!r}")
        self.E = E
        self.Q = len(E)
        self.w = np.array([wmap[int((e * e).sum())] for e in E], dtype=np.float64)
        self.cs2 = cs2
        opp = []
        for e in E:
            hits = [j for j, e2 in enumerate(E) if (e2 == -e).all()]
            assert len(hits) == 1
            opp.append(hits[0])
        self.opp = np.array(opp, dtype=np.int64)


def moment_basis(lat: Lattice):
    """Rows of the orthogonal MRT moment matrix U, plus row roles.

    Returns (U, conserved_rows, stress_rows).  U[k, i] is the k-th moment
    polynomial evaluated at e_i.
    """
    ex, ey, ez = (lat.E[:, a].astype(np.float64) for a in range(3))
    c2 = ex * ex + ey * ey + ez * ez
    if lat.name == "D3Q19":
        rows = [
            np.ones_like(c2),                        # rho
            19 * c2 - 30,                            # e
            (21 * c2 * c2 - 53 * c2 + 24) / 2,       # epsilon
            ex,                                      # j_x
            (5 * c2 - 9) * ex,                       # q_x
            ey,                                      # j_y
            (5 * c2 - 9) * ey,                       # q_y
            ez,                                      # j_z
            (5 * c2 - 9) * ez,                       # q_z
            3 * ex * ex - c2,                        # 3 p_xx
            (3 * c2 - 5) * (3 * ex * ex - c2),       # 3 pi_xx
            ey * ey - ez * ez,                       # p_ww
            (3 * c2 - 5) * (ey * ey - ez * ez),      # pi_ww
            ex * ey,                                 # p_xy
            ey * ez,                                 # p_yz
            ex * ez,                                 # p_xz
            (ey * ey - ez * ez) * ex,                # m_x
            (ez * ez - ex * ex) * ey,                # m_y
            (ex * ex - ey * ey) * ez,                # m_z
        ]
        conserved = [0, 3, 5, 7]
        stress = [9, 11, 13, 14, 15]
    elif lat.name == "D2Q9":
        rows = [
            np.ones_like(c2),                        # rho
            -4 + 3 * c2,                             # e
            4 - 10.5 * c2 + 4.5 * c2 * c2,           # epsilon
            ex,                                      # j_x
            (-5 + 3 * c2) * ex,                      # q_x
            ey,                                      # j_y
            (-5 + 3 * c2) * ey,                      # q_y
            ex * ex - ey * ey,                       # p_xx
            ex * ey,                                 # p_xy
        ]
        conserved = [0, 3, 5]
        stress = [7, 8]
    else:
        raise ValueError("MRT basis defined for D2Q9 and D3Q19 only")
    U = np.stack(rows).astype(np.float64)
    return U, conserved, stress
