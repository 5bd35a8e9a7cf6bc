"""Singly diagonally implicit Runge-Kutta stepping (Sec. 4.1, Eq. SDIRK_compact
and Eq. cp_dirk of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Tableaux of Eq. SDIRK, with the diagonal a_* = a_11 = ... = a_ss:
  "sdirk2": the 2-stage tableau as printed (a_* = 1/4, c = (1/4, 3/4),
            b = (1/2, 1/2)).  Its order is 2, not the 3 its label SDIRK(2,3)
            suggests (the order-3 member of the same family has
            a_* = (3 + sqrt 3)/6); it is kept as printed.
  "sdirk23": that order-3 member, a_* = (3 + sqrt 3)/6.
  "sdirk34": the 3-stage tableau as printed, nu = cos(pi/18)/sqrt 3 + 1/2,
            xi = 1 / (6 (2 nu - 1)^2).
  "sdirk1":  the 1-stage member (implicit midpoint, a_* = 1/2, b = 1).

One step from U^{n-1}, in the paper's order: for i = 1..s solve the full
(non-condensed) stage system of Eq. cp_dirk,
    [M + a_* dt K_T,  a_* dt K_TF] [U_T^{n,i}]   [B_T^{n,i}]
    [a_* dt K_FT,     a_* dt K_F ] [U_F^{n,i}] = [B_F^{n,i}],
    B_T = M U^{n-1} + a_* dt F^{n-1+c_i}
          + dt sum_{j<i} a_ij (F^{n-1+c_j} - K_T U_T^{n,j} - K_TF U_F^{n,j}),
    B_F = -dt sum_{j<i} a_ij (K_FT U_T^{n,j} + K_F U_F^{n,j}),
then the last stage (a_{s+1,j} = b_j, a_{s+1,s+1} = 0) is a mass solve:
    M U^n = M U^{n-1} + dt sum_j b_j (F^{n-1+c_j} - K_T U_T^{n,j} - K_TF U_F^{n,j}).
The stage matrix is factorised once per dt by a generic sparse LU of the
whole system (no static condensation).  ``step_condensed`` applies the same
tableau to the condensed ODE M U' = F - K_cond U instead; the two agree
because every stage keeps K_FT U_T + K_F U_F = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _tableaux():
    nu = np.cos(np.pi / 18.0) / np.sqrt(3.0) + 0.5
    xi = 1.0 / (6.0 * (2.0 * nu - 1.0) ** 2)
    g3 = (3.0 + np.sqrt(3.0)) / 6.0
    return {
        "sdirk1": (np.array([[0.5]]), np.array([1.0]), np.array([0.5])),
        "sdirk2": (np.array([[0.25, 0.0], [0.5, 0.25]]), np.array([0.5, 0.5]), np.array([0.25, 0.75])),
        "sdirk23": (np.array([[g3, 0.0], [1.0 - 2.0 * g3, g3]]), np.array([0.5, 0.5]), np.array([g3, 1.0 - g3])),
        "sdirk34": (np.array([[nu, 0.0, 0.0], [0.5 - nu, nu, 0.0], [2.0 * nu, 1.0 - 4.0 * nu, nu]]),
                    np.array([xi, 1.0 - 2.0 * xi, xi]), np.array([nu, 0.5, 1.0 - nu])),
    }


TABLEAUX = _tableaux()


def tableau(name: str):
    """(A, b, c): A lower triangular with constant diagonal a_*."""
    A, b, c = TABLEAUX[name]
    return A.copy(), b.copy(), c.copy()


class Stepper:
    """SDIRK stepping of an assembled ``System`` with an optional source F(t)."""

    def __init__(self, system, source=None):
        self.sys = system
        self.source = source
        self.luM = spla.splu(system.M.tocsc())
        self._lu = {}

    def F(self, t):
        if self.source is None:
            return np.zeros(self.sys.nT)
        return self.source(t)

    def _stage_lu(self, a_dt):
        key = float(a_dt)
        if key not in self._lu:
            S = self.sys
            top = sp.hstack([S.M + a_dt * S.KT, a_dt * S.KTF])
            bot = sp.hstack([a_dt * S.KFT, a_dt * S.KF])
            self._lu[key] = spla.splu(sp.vstack([top, bot]).tocsc())
        return self._lu[key]

    def step(self, U, t0: float, dt: float, name: str = "sdirk34", nsteps: int = 1):
        """Eq. SDIRK_compact / Eq. cp_dirk on the full system."""
        A, b, c = tableau(name)
        s = len(b)
        a = A[0, 0]
        S = self.sys
        nT = S.nT
        lu = self._stage_lu(a * dt)
        t = t0
        for _ in range(nsteps):
            MU0 = S.M @ U
            R, G = [], []          # cell residuals F - K_T U_T - K_TF U_F and face residuals -(K_FT U_T + K_F U_F)
            for i in range(s):
                BT = MU0 + a * dt * self.F(t + c[i] * dt)
                BF = np.zeros(S.nF)
                for j in range(i):
                    BT += dt * A[i, j] * R[j]
                    BF += dt * A[i, j] * G[j]
                X = lu.solve(np.concatenate([BT, BF]))
                UT, UF = X[:nT], X[nT:]
                R.append(self.F(t + c[i] * dt) - S.KT @ UT - S.KTF @ UF)
                G.append(-(S.KFT @ UT + S.KF @ UF))
            rhs = MU0.copy()
            for j in range(s):
                rhs += dt * b[j] * R[j]
            U = self.luM.solve(rhs)
            t = t + dt
        return U

    def step_condensed(self, U, t0: float, dt: float, name: str = "sdirk34", nsteps: int = 1):
        """The same tableau on the condensed ODE M U' = F - K_cond U with
        K_cond = K_T - K_TF K_F^{-1} K_FT (dense; for small meshes)."""
        A, b, c = tableau(name)
        s = len(b)
        a = A[0, 0]
        S = self.sys
        KF = S.KF.toarray()
        Kc = S.KT.toarray() - S.KTF.toarray() @ np.linalg.solve(KF, S.KFT.toarray())
        M = S.M.toarray()
        L = M + a * dt * Kc
        t = t0
        for _ in range(nsteps):
            MU0 = M @ U
            R = []
            for i in range(s):
                rhs = MU0 + a * dt * self.F(t + c[i] * dt)
                for j in range(i):
                    rhs += dt * A[i, j] * R[j]
                Y = np.linalg.solve(L, rhs)
                R.append(self.F(t + c[i] * dt) - Kc @ Y)
            rhs = MU0.copy()
            for j in range(s):
                rhs += dt * b[j] * R[j]
            U = np.linalg.solve(M, rhs)
            t = t + dt
        return U
