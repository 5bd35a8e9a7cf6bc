"""Discrete adjoint of the ERK stepping, from the assembled matrices.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Forward (Sec. 4.2, Eq. ERK_compact with Eq. ex_solve): the semi-discrete rate
is k = A U + w(t) M^-1 b with A = -M^-1 (K_T - K_TF K_F^-1 K_FT), stage values
Y_i = U^{n-1} + dt sum_{j<i} a_ij k_j, U^n = U^{n-1} + dt sum_i b_i k_i; the
traces are d^n = R U^n (cell receivers: basis values; interface receivers:
the face values of the face solve).

Reverse mode for a cotangent G (dL/dd): lambda^n += R^T G^n; for stages in
reverse order mu_i = dt (b_i lambda + sum_{l>i} a_li nu_l), nu_i = A^T mu_i;
lambda^{n-1} = lambda^n + sum_i nu_i.  Here A^T is the plain transpose of the
dense matrix.

Material gradients with the stabilisation weights held fixed: K and b do not
depend on the materials, M does, so dk/dtheta = -M^-1 (dM/dtheta) k and
dL/dtheta = sum mu_i^T dk_i/dtheta.  dM/dtheta is assembled per cell from the
mass definitions (Eq. mass): rho multiplies the m / v blocks, 1/kappa the p
block, the plane-strain compliance the s block.  dL/dw(t_i) = mu_i^T M^-1 b.
"""
from __future__ import annotations

import numpy as np

from . import mesh as mmesh
from .assemble import E_BASIS, compliance_dlam, compliance_dmu
from .diagnostics import find_interface_face
from .assemble import locate_cell
from .erk import tableau
from .spaces import eval_cell_basis


def receiver_matrix(stepper, points):
    """Dense R with d = R U ([n_rec*5, nT]), rows ordered (receiver, field)."""
    S = stepper.sys
    m = S.mesh
    n = S.n
    R = np.zeros((5 * len(points), S.nT))
    KF = S.KF.toarray() if S.nF else None
    KFT = S.KFT.toarray() if S.nF else None
    for r, (x, y) in enumerate(points):
        F, xi = find_interface_face(m, x, y)
        if F is not None:
            psi = np.array([xi ** l for l in range(S.f)])
            E = np.zeros((3, S.nF))
            E[0, [S.idx_pF(F, l) for l in range(S.f)]] = psi
            for d in range(2):
                E[1 + d, [S.idx_vF(F, d, l) for l in range(S.f)]] = psi
            R[5 * r: 5 * r + 3] = -E @ np.linalg.solve(KF, KFT)
            continue
        c = locate_cell(m, x, y)
        xT, yT, h = S.cell_frame(c)
        phi = eval_cell_basis(S.k, xT, yT, h, [x], [y])[0]
        o = S.cell_off[c]
        fields = [2, 0, 1] if m.cell_domain[c] == mmesh.FLUID else [3, 4, 0, 1, 2]
        for j, fld in enumerate(fields):
            R[5 * r + j, o + fld * n: o + (fld + 1) * n] = phi
    return R


class DenseAdjoint:
    """Forward traces and reverse-mode gradients on a small assembled system."""

    def __init__(self, stepper, points, load=None, wavelet=None):
        S = stepper.sys
        self.S = S
        KT, KTF, KFT, KF, M = (x.toarray() for x in (S.KT, S.KTF, S.KFT, S.KF, S.M))
        Kc = KT - KTF @ np.linalg.solve(KF, KFT) if S.nF else KT
        self.M = M
        self.A = -np.linalg.solve(M, Kc)
        self.R = receiver_matrix(stepper, points)
        self.g = np.zeros(S.nT) if load is None else np.linalg.solve(M, load)
        self.wavelet = wavelet if wavelet is not None else (lambda t: 0.0)

    def run(self, U0, t0, dt, nsteps, scheme="erk4"):
        Aext, b, c = tableau(scheme)
        s = len(b)
        U = U0.copy()
        traces, stages = [], []
        for n in range(nsteps):
            tn = t0 + n * dt
            Y, K = [], []
            for i in range(s):
                Yi = U + dt * sum(Aext[i, j] * K[j] for j in range(i)) if i else U.copy()
                Y.append(Yi)
                K.append(self.A @ Yi + self.wavelet(tn + c[i] * dt) * self.g)
            U = U + dt * sum(b[i] * K[i] for i in range(s))
            stages.append((Y, K))
            traces.append(self.R @ U)
        return np.array(traces), stages

    def vjp(self, U0, t0, dt, nsteps, cotangent, scheme="erk4"):
        """Returns (grad [nc, 4] = dL/d(rho, kappa, lambda, mu), grad_w [nsteps, s])."""
        S = self.S
        m = S.mesh
        n = S.n
        Aext, b, c = tableau(scheme)
        s = len(b)
        _, stages = self.run(U0, t0, dt, nsteps, scheme)
        G = cotangent.reshape(nsteps, -1)
        lam = np.zeros(S.nT)
        grad = np.zeros((m.n_cells, 4))
        gw = np.zeros((nsteps, s))
        AT = self.A.T
        Minv = np.linalg.inv(self.M)
        for nn in range(nsteps - 1, -1, -1):
            lam = lam + self.R.T @ G[nn]
            Y, K = stages[nn]
            pend = [np.zeros(S.nT) for _ in range(s)]
            acc = lam.copy()
            for i in range(s - 1, -1, -1):
                mu_i = dt * (b[i] * lam + pend[i])
                nu = AT @ mu_i
                acc += nu
                for l in range(i):
                    if Aext[i, l] != 0.0:
                        pend[l] += Aext[i, l] * nu
                gw[nn, i] = mu_i @ self.g
                eta = Minv @ mu_i          # dL/dtheta = -eta^T (dM/dtheta) k
                k = K[i]
                for cc in range(m.n_cells):
                    M0 = S.M0[cc]
                    o = S.cell_off[cc]
                    blk = lambda f: slice(o + f * n, o + (f + 1) * n)
                    if m.cell_domain[cc] == mmesh.FLUID:
                        grad[cc, 0] -= sum(eta[blk(f)] @ M0 @ k[blk(f)] for f in (0, 1))
                        grad[cc, 1] -= eta[blk(2)] @ (-M0 / S.kappa[cc] ** 2) @ k[blk(2)]
                    else:
                        grad[cc, 0] -= sum(eta[blk(f)] @ M0 @ k[blk(f)] for f in (3, 4))
                        for p, dfun in ((2, compliance_dlam), (3, compliance_dmu)):
                            dD = np.array([[np.sum(dfun(S.lam[cc], S.mu[cc], E_BASIS[bb]) * E_BASIS[aa])
                                            for bb in range(3)] for aa in range(3)])
                            grad[cc, p] -= sum(dD[aa, bb] * (eta[blk(aa)] @ M0 @ k[blk(bb)])
                                               for aa in range(3) for bb in range(3))
            lam = acc
        return grad, gw
