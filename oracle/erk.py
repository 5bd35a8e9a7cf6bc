"""Explicit Runge-Kutta time stepping (Sec. 4.2 of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Tableaux: Eq. ERK (ERK(2) explicit midpoint, ERK(3), classical ERK(4)), with
the paper's convention a_{s+1,i} := b_i (Sec. 4, after the generic tableaux).

One time step from U^{n-1} follows Eq. ERK_compact with the face elimination
of Eq. ex_solve, in the paper's order: U^{n,1} = U^{n-1}; for i = 2..s+1,
first solve K_F U_F^{n,i-1} = -K_FT U_T^{n,i-1}, then
M U^{n,i} = M U^{n-1} + dt sum_{j<i} a_ij (F^{n-1+c_j} - K_T U^{n,j} - K_TF U_F^{n,j});
finally U^n := U^{n,s+1} (read of the paper's "U^{n+1} := U^{n,s+1}").

Both solves are done with a generic sparse LU of the *global* K_F and M
(scipy's SuperLU), with no use of their block-diagonal structure.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np
import scipy.sparse.linalg as spla

TABLEAUX = {
    # name: (A strictly lower triangular, b, c) as exact rationals (Eq. ERK)
    "erk2": ([[0, 0], [Fr(1, 2), 0]], [0, 1], [0, Fr(1, 2)]),
    "erk3": ([[0, 0, 0], [Fr(1, 2), 0, 0], [-1, 2, 0]], [Fr(1, 6), Fr(2, 3), Fr(1, 6)], [0, Fr(1, 2), 1]),
    "erk4": ([[0, 0, 0, 0], [Fr(1, 2), 0, 0, 0], [0, Fr(1, 2), 0, 0], [0, 0, 1, 0]],
             [Fr(1, 6), Fr(1, 3), Fr(1, 3), Fr(1, 6)], [0, Fr(1, 2), Fr(1, 2), 1]),
}


def tableau(name: str):
    """(A, b, c) as float arrays, with the extended row a_{s+1,:} = b appended to A."""
    A, b, c = TABLEAUX[name]
    s = len(b)
    Aext = np.zeros((s + 1, s))
    for i in range(s):
        for j in range(s):
            Aext[i, j] = float(A[i][j])
    Aext[s, :] = [float(x) for x in b]
    return Aext, np.array([float(x) for x in b]), np.array([float(x) for x in c])


class Stepper:
    """ERK stepping of an assembled ``System`` with an optional source F(t)."""

    def __init__(self, system, source=None):
        """``source(t)`` returns the load vector F_T(t) (length nT), or None."""
        self.sys = system
        self.source = source
        self.luF = spla.splu(system.KF.tocsc()) if system.nF > 0 else None
        self.luM = spla.splu(system.M.tocsc())

    def face_solve(self, UT):
        """U_F = K_F^{-1} (-K_FT U_T)  (first equation of Eq. ex_solve)."""
        if self.luF is None:
            return np.zeros(0)
        return self.luF.solve(-(self.sys.KFT @ UT))

    def F(self, t):
        if self.source is None:
            return np.zeros(self.sys.nT)
        return self.source(t)

    def residual(self, UT, t):
        """W = F(t) - K_T U_T - K_TF U_F with U_F from the face solve."""
        UF = self.face_solve(UT)
        return self.F(t) - self.sys.KT @ UT - self.sys.KTF @ UF

    def rate(self, UT, t):
        """d/dt U_T = M^{-1} (F(t) - (K_T - K_TF K_F^{-1} K_FT) U_T)."""
        return self.luM.solve(self.residual(UT, t))

    def step(self, U, t0: float, dt: float, name: str = "erk4", nsteps: int = 1):
        A, b, c = tableau(name)
        s = len(b)
        t = t0
        for _ in range(nsteps):
            MU0 = self.sys.M @ U
            stages = [U]
            W = []
            for i in range(1, s + 1):              # builds U^{n,i+1}, i.e. paper stage i+1
                W.append(self.residual(stages[i - 1], t + c[i - 1] * dt))
                rhs = MU0.copy()
                for j in range(i):
                    if A[i, j] != 0.0:
                        rhs += dt * A[i, j] * W[j]
                stages.append(self.luM.solve(rhs))
            U = stages[s]
            t = t + dt
        return U
