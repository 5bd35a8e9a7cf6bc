"""Local polynomial spaces and bases (Sec. 3.2 and Sec. 3.3 of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Equal order k' = k (the ERK setting, Sec. 3.3 and Sec. 5).  Per cell T:
  fluid: m_T in P^k(T)^2 (dG dual), p_T in P^k(T) (HHO primal);
  solid: s_T in P^k_sym(T) (3 components in 2D), v_T in P^k(T)^2.
Per face F: fluid p_F in P^k(F); solid v_F in P^k(F)^2; interface both
(Sec. 3.2).

Bases: monomials centred at the barycentre (Sec. 3.3, the sentence after the
basis list), scaled by the cell diameter:
  phi_(a,b) = X^a Y^b with X = (x - x_T)/h_T, Y = (y - y_T)/h_T,
ordered by total degree, then by decreasing a: 1, X, Y, X^2, XY, Y^2, ...
Face basis: xi^l, l = 0..k, xi in [-1, 1] the affine coordinate from the
canonical start point A to the end point B of the face.
Vector fields: component blocks [x-block, y-block].  Symmetric tensors:
basis E_xx, E_yy, E_xy = e_x (x) e_y + e_y (x) e_x, so the coefficients are the
physical components.

Cell DOF order: fluid [m_x, m_y, p], solid [s_xx, s_yy, s_xy, v_x, v_y] (the
row order of the paper's block system).
"""
from __future__ import annotations

import numpy as np


def exponents(k: int):
    """List of (a, b) with a + b <= k, by total degree then decreasing a."""
    out = []
    for d in range(k + 1):
        for a in range(d, -1, -1):
            out.append((a, d - a))
    return out


def n_cell(k: int) -> int:
    """dim P^k(T) in 2D."""
    return (k + 1) * (k + 2) // 2


def n_face(k: int) -> int:
    """dim P^k(F) in 2D (F is a segment)."""
    return k + 1


def cell_dofs(k: int, domain: int) -> int:
    """3 n for a fluid cell (m: 2n, p: n); 5 n for a solid cell (s: 3n, v: 2n)."""
    return (3 if domain == 0 else 5) * n_cell(k)


def face_dofs(k: int, face_type: int) -> int:
    """Unknowns on a face: f fluid, 2f solid, 3f interface, 0 boundary."""
    f = n_face(k)
    return {0: f, 1: 2 * f, 2: 3 * f, 3: 0, 4: 0}[int(face_type)]


def eval_cell_basis(k: int, xT, yT, hT, x, y):
    """Matrix [len(x), n] of phi_i(x, y)."""
    X = (np.asarray(x, dtype=np.float64) - xT) / hT
    Y = (np.asarray(y, dtype=np.float64) - yT) / hT
    return np.stack([X ** a * Y ** b for (a, b) in exponents(k)], axis=-1)
