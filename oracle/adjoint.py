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

Material gradients.  The materials enter through M (Eq. mass: rho
multiplies the m / v blocks, 1/kappa the p block, the plane-strain
compliance the s block) and through the stabilisation weights tau (Sec. 3.3:
tau^f = eta_f / (rho c_P), tau^s = eta_s rho c^s), which scale each cell's
least-squares stabilisation (Eq. stab).  So
    dL/dtheta = sum_i mu_i^T dk_i/dtheta + sum_c dL/dtau_c dtau_c/dtheta,
with dk/dtheta = -M^-1 (dM/dtheta) k for the mass part.  K is affine in tau
(dK/dtau_c = the stabilisation form of cell c, System.stab_form), so with the
face values Y_F = -K_F^-1 K_FT Y of a stage value, eta = M^-1 mu and the
adjoint face values eta_F = -K_F^-T K_TF^T eta,
    d(eta^T K_cond Y)/dtau_c = [eta; eta_F]^T (dK/dtau_c) [Y; Y_F]
(K_cond = K_T - K_TF K_F^-1 K_FT), and the stage term is minus that.  The
interface receivers read face values, which depend on tau as well: for
d = E U_F, d(G^T d)/dtau_c = [0; zeta]^T (dK/dtau_c) [U; U_F] with
zeta = -K_F^-T E^T G.  With tau given explicitly (tau_override) the weights
are constants and only the mass part remains.  dL/dw(t_i) = mu_i^T M^-1 b.
"""
from __future__ import annotations

import numpy as np

from . import mesh as mmesh
from .assemble import E_BASIS, compliance_dlam, compliance_dmu
from .diagnostics import find_interface_face
from .assemble import locate_cell
from .erk import tableau
from .spaces import eval_cell_basis


def receiver_matrix(stepper, points, with_face_rows=False):
    """Dense R with d = R U ([n_rec*5, nT]), rows ordered (receiver, field).
    With with_face_rows, also E ([n_rec*5, nF]): the rows of the interface
    receivers as point values of the face unknowns (d = E U_F there)."""
    S = stepper.sys
    m = S.mesh
    n = S.n
    R = np.zeros((5 * len(points), S.nT))
    Efull = np.zeros((5 * len(points), S.nF))
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
            Efull[5 * r: 5 * r + 3] = E
            continue
        c = locate_cell(m, x, y)
        xT, yT, h = S.cell_frame(c)
        phi = eval_cell_basis(S.k, xT, yT, h, [x], [y])[0]
        o = S.cell_off[c]
        fields = [2, 0, 1] if m.cell_domain[c] == mmesh.FLUID else [3, 4, 0, 1, 2]
        for j, fld in enumerate(fields):
            R[5 * r + j, o + fld * n: o + (fld + 1) * n] = phi
    return (R, Efull) if with_face_rows else R


class DenseAdjoint:
    """Forward traces and reverse-mode gradients on a small assembled system."""

    def __init__(self, stepper, points, load=None, wavelet=None):
        S = stepper.sys
        self.S = S
        KT, KTF, KFT, KF, M = (x.toarray() for x in (S.KT, S.KTF, S.KFT, S.KF, S.M))
        Kc = KT - KTF @ np.linalg.solve(KF, KFT) if S.nF else KT
        self.M = M
        self.A = -np.linalg.solve(M, Kc)
        self.R, self.E = receiver_matrix(stepper, points, with_face_rows=True)
        self.KF, self.KFT, self.KTF = KF, KFT, KTF
        self.dK = [S.stab_form(c) for c in range(S.mesh.n_cells)]
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
        self._U_end = U
        return np.array(traces), stages

    def face_values(self, U):
        """U_F = -K_F^-1 K_FT U (the face solve of Eq. ex_solve)."""
        return -np.linalg.solve(self.KF, self.KFT @ U) if self.S.nF else np.zeros(0)

    def adjoint_face_values(self, eta):
        """eta_F = -K_F^-T K_TF^T eta."""
        return -np.linalg.solve(self.KF.T, self.KTF.T @ eta) if self.S.nF else np.zeros(0)

    def tau_form(self, a, b):
        """[a^T (dK/dtau_c) b for every cell c] over stacked [U_T; U_F] vectors."""
        return np.array([a @ (dK @ b) for dK in self.dK])

    def vjp(self, U0, t0, dt, nsteps, cotangent, scheme="erk4", with_tau=False):
        """Returns (grad [nc, 4] = dL/d(rho, kappa, lambda, mu), grad_w [nsteps, s]),
        and dL/dtau [nc] as a third value when with_tau."""
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
        gtau = np.zeros(m.n_cells)
        for nn in range(nsteps - 1, -1, -1):
            lam = lam + self.R.T @ G[nn]
            if np.any(self.E):
                # interface receivers: d = E U_F(U^n), U^n = the next step's first stage value
                Un = stages[nn + 1][0][0] if nn + 1 < nsteps else self._U_end
                zeta = -np.linalg.solve(self.KF.T, self.E.T @ G[nn])
                gtau += self.tau_form(np.concatenate([np.zeros(S.nT), zeta]),
                                      np.concatenate([Un, self.face_values(Un)]))
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
                gtau -= self.tau_form(np.concatenate([eta, self.adjoint_face_values(eta)]),
                                      np.concatenate([Y[i], self.face_values(Y[i])]))
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
        grad += gtau[:, None] * S.tau_material_derivatives()
        return (grad, gw, gtau) if with_tau else (grad, gw)
