"""Full, non-condensed HHO algebraic system (Sec. 3.3 of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Assembles, as scipy sparse matrices, the blocks of the compact form
(Eq. compact_AR)

    [ M 0 ] d/dt [U_T]   [ K_T   K_TF ] [U_T]   [F_T]
    [ 0 0 ]      [U_F] + [ K_FT  K_F  ] [U_F] = [ 0 ]

directly from the defining integrals:

* mass matrices, Eq. mass: rho (m, r)_T, (1/kappa) (p, q)_T,
  (C^-1 s, b)_T, rho (v, w)_T;
* gradient reconstruction, Eq. rec_a:
  (G_T P_T + G_TF P_F)^T R = (grad p_T, r)_T - (p_T - p_dT, r.n_T)_dT,
  and the symmetric-gradient reconstruction, Eq. rec_e, with grad_sym and b.n_T;
* least-squares stabilisation for equal order (Eq. stab with
  S_dT(p_T, p_dT) = p_T|dT - p_dT), weights tau^f = eta^f / (rho c_P) and
  tau^s = eta^s rho c^s (alpha = 0, so the normalised diameter drops out);
* the coupling block, Q_F^T C V_F = (v_F . n_Gamma, q_F)_Gamma, nonzero only
  on interface faces;
* source vectors as load vectors (f, q)_T and (f^s, w)_T.

Readings of the paper taken here:

* Signs of the dual variables: the weak form (Eq. HHO1/HHO2) is used, i.e.
  d/dt m = g(p) and d/dt s = C g_sym(v).  The printed block matrix carries the
  opposite sign on the dual rows and columns; the two systems are the same
  under m -> -m, s -> -s, and the primal fields agree.  With this choice
  K_FT = (S K_TF)^T with S = -1 on dual rows and +1 on primal rows.
* Dirichlet boundary faces carry no unknowns (face values are zero); they
  still contribute their terms with p_dT = 0 / v_dT = 0.
* The source enters as the load vector (f, phi_i)_T.
* c^s in tau^s is c_P by default ("cp"), c_S on request ("cs").
* Plane strain: C^-1 s = (s - lambda/(2(lambda+mu)) tr(s) I) / (2 mu).

Every integral is exact up to rounding: cell integrals of monomials by
Green's theorem, face integrals by Gauss-Legendre with k+2 points (exact for
degree 2k+3).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import mesh as mmesh
from .quadrature import gauss_legendre, polygon_monomial, fan_rule
from .spaces import exponents, n_cell, n_face, eval_cell_basis

# Symmetric-tensor basis E_xx, E_yy, E_xy = e_x (x) e_y + e_y (x) e_x.
E_BASIS = [np.array([[1.0, 0.0], [0.0, 0.0]]),
           np.array([[0.0, 0.0], [0.0, 1.0]]),
           np.array([[0.0, 1.0], [1.0, 0.0]])]


def compliance(lam: float, mu: float, S: np.ndarray) -> np.ndarray:
    """Plane-strain C^-1 S = (S - lambda/(2(lambda+mu)) tr(S) I) / (2 mu)."""
    beta = lam / (2.0 * (lam + mu))
    return (S - beta * np.trace(S) * np.eye(2)) / (2.0 * mu)


def compliance_dlam(lam: float, mu: float, S: np.ndarray) -> np.ndarray:
    """d/dlambda of compliance(lam, mu, S): -(dbeta/dlam) tr(S) I / (2 mu),
    dbeta/dlam = mu / (2 (lam+mu)^2)."""
    dbeta = mu / (2.0 * (lam + mu) ** 2)
    return -dbeta * np.trace(S) * np.eye(2) / (2.0 * mu)


def compliance_dmu(lam: float, mu: float, S: np.ndarray) -> np.ndarray:
    """d/dmu of compliance(lam, mu, S), dbeta/dmu = -lam / (2 (lam+mu)^2)."""
    beta = lam / (2.0 * (lam + mu))
    dbeta = -lam / (2.0 * (lam + mu) ** 2)
    return -dbeta * np.trace(S) * np.eye(2) / (2.0 * mu) - (S - beta * np.trace(S) * np.eye(2)) / (2.0 * mu ** 2)


def sym_grad_coef(c: int, d: int, q: int) -> float:
    """grad_sym(phi e_d) : E_c = sum_q coef * d_q phi; returns the coef for q."""
    G = np.zeros((2, 2))
    G[d, q] = 1.0                     # grad(phi e_d) = e_d (x) grad(phi)
    return float(np.sum(0.5 * (G + G.T) * E_BASIS[c]))


class System:
    """Global blocks M, K_T, K_TF, K_FT, K_F and the DOF maps."""

    def __init__(self, mesh: mmesh.Mesh, k: int, rho, lam, mu, kappa,
                 eta_f: float = 0.8, eta_s: float = 1.5, stab_speed: str = "cp",
                 tau_over_k: bool = False, tau_override=None):
        if k < 1 or k > 3:
            raise ValueError("k must be 1, 2 or 3")
        self.mesh = mesh
        self.k = k
        self.n = n_cell(k)
        self.f = n_face(k)
        self.exps = exponents(k)
        nc = mesh.n_cells
        self.rho = np.asarray(rho, dtype=np.float64)
        self.lam = np.asarray(lam, dtype=np.float64)
        self.mu = np.asarray(mu, dtype=np.float64)
        self.kappa = np.asarray(kappa, dtype=np.float64)
        dom = mesh.cell_domain
        # stabilisation weights (Sec. 3.3, alpha = 0; eta weights of Sec. 5.1)
        tau = np.empty(nc)
        for c in range(nc):
            if dom[c] == mmesh.FLUID:
                cp = np.sqrt(self.kappa[c] / self.rho[c])
                tau[c] = eta_f / (self.rho[c] * cp)
            else:
                if stab_speed == "cp":
                    cs = np.sqrt((self.lam[c] + 2.0 * self.mu[c]) / self.rho[c])
                elif stab_speed == "cs":
                    cs = np.sqrt(self.mu[c] / self.rho[c])
                else:
                    raise ValueError("stab_speed must be 'cp' or 'cs'")
                tau[c] = eta_s * self.rho[c] * cs
            if tau_over_k:
                tau[c] /= k
        if tau_override is not None:
            # stabilisation weights given explicitly (held fixed, e.g. while
            # differentiating with respect to the materials)
            tau = np.array(tau_override, dtype=np.float64)
        self.tau = tau
        self.tau_fixed = tau_override is not None
        self.stab_speed = stab_speed

        n, f = self.n, self.f
        self.cell_off = np.zeros(nc + 1, dtype=np.int64)
        for c in range(nc):
            self.cell_off[c + 1] = self.cell_off[c] + (3 if dom[c] == mmesh.FLUID else 5) * n
        self.nT = int(self.cell_off[-1])
        ft = mesh.face_type
        self.face_off = np.zeros(mesh.n_faces + 1, dtype=np.int64)
        for F in range(mesh.n_faces):
            size = {0: f, 1: 2 * f, 2: 3 * f, 3: 0, 4: 0}[int(ft[F])]
            self.face_off[F + 1] = self.face_off[F] + size
        self.nF = int(self.face_off[-1])
        self._assemble()

    # ---- DOF index helpers -------------------------------------------------
    def idx_m(self, c, comp, i):
        return self.cell_off[c] + comp * self.n + i

    def idx_p(self, c, i):
        return self.cell_off[c] + 2 * self.n + i

    def idx_s(self, c, comp, i):
        return self.cell_off[c] + comp * self.n + i

    def idx_v(self, c, comp, i):
        return self.cell_off[c] + (3 + comp) * self.n + i

    def idx_pF(self, F, l):
        return self.face_off[F] + l

    def idx_vF(self, F, comp, l):
        base = self.face_off[F] + (self.f if self.mesh.face_type[F] == mmesh.FT_IFACE else 0)
        return base + comp * self.f + l

    # ---- local integrals ---------------------------------------------------
    def cell_frame(self, c):
        m = self.mesh
        return m.cell_centroid[c, 0], m.cell_centroid[c, 1], m.cell_diam[c]

    def local_cell_integrals(self, c):
        """M0[i,j] = (phi_j, phi_i)_T and D[q][i,j] = (d_q phi_j, phi_i)_T."""
        m = self.mesh
        xT, yT, h = self.cell_frame(c)
        vs = mmesh.cell_vertices(m, c)
        X = [(m.xy[v, 0] - xT) / h for v in vs]
        Y = [(m.xy[v, 1] - yT) / h for v in vs]
        cache = {}

        def I(a, b):
            if (a, b) not in cache:
                cache[(a, b)] = h * h * polygon_monomial(X, Y, a, b)
            return cache[(a, b)]
        n = self.n
        M0 = np.zeros((n, n))
        Dx = np.zeros((n, n))
        Dy = np.zeros((n, n))
        for i, (ai, bi) in enumerate(self.exps):
            for j, (aj, bj) in enumerate(self.exps):
                M0[i, j] = I(ai + aj, bi + bj)
                if aj > 0:
                    Dx[i, j] = aj / h * I(ai + aj - 1, bi + bj)
                if bj > 0:
                    Dy[i, j] = bj / h * I(ai + aj, bi + bj - 1)
        return M0, (Dx, Dy)

    def local_face_integrals(self, F, c):
        """Face F seen from cell c: (PP, SP, SS, n_T) with
        PP[i,j] = (phi_j, phi_i)_F, SP[i,l] = (psi_l, phi_i)_F, SS[l,m] = (psi_m, psi_l)_F."""
        A, B, length, nT = mmesh.face_in_cell(self.mesh, F, c)
        xi, w = gauss_legendre(self.k + 2)
        W = w * length / 2.0
        pts = 0.5 * (A + B)[None, :] + xi[:, None] * (0.5 * (B - A))[None, :]
        xT, yT, h = self.cell_frame(c)
        phi = eval_cell_basis(self.k, xT, yT, h, pts[:, 0], pts[:, 1])      # (q, n)
        psi = np.stack([xi ** l for l in range(self.f)], axis=-1)          # (q, f)
        PP = phi.T @ (W[:, None] * phi)
        SP = phi.T @ (W[:, None] * psi)
        SS = psi.T @ (W[:, None] * psi)
        return PP, SP, SS, nT

    # ---- assembly ------------------------------------------------------------
    def _assemble(self):
        m = self.mesh
        n, f = self.n, self.f
        Mr, Mc, Mv = [], [], []
        Tr, Tc, Tv = [], [], []          # K_T
        TFr, TFc, TFv = [], [], []       # K_TF
        FTr, FTc, FTv = [], [], []       # K_FT
        Fr, Fc, Fv = [], [], []          # K_F
        self.M0 = []

        def add(r, cc, v, R, C, V):
            if v != 0.0:
                R.append(r)
                C.append(cc)
                V.append(v)

        for c in range(m.n_cells):
            M0, (Dx, Dy) = self.local_cell_integrals(c)
            self.M0.append(M0)
            Dq = (Dx, Dy)
            tau = self.tau[c]
            faces = m.cell_faces[c]
            finfo = [(F,) + self.local_face_integrals(F, c) for F in faces]
            if m.cell_domain[c] == mmesh.FLUID:
                rho, kap = self.rho[c], self.kappa[c]
                for comp in range(2):
                    for i in range(n):
                        for j in range(n):
                            add(self.idx_m(c, comp, i), self.idx_m(c, comp, j), rho * M0[i, j], Mr, Mc, Mv)
                for i in range(n):
                    for j in range(n):
                        add(self.idx_p(c, i), self.idx_p(c, j), M0[i, j] / kap, Mr, Mc, Mv)
                # G_T[(comp,i), j] = (d_comp phi_j, phi_i)_T - sum_F n_comp (phi_j, phi_i)_F
                G = [Dq[comp].copy() for comp in range(2)]
                SigT = np.zeros((n, n))
                for (F, PP, SP, SS, nT) in finfo:
                    for comp in range(2):
                        G[comp] -= nT[comp] * PP
                    SigT += tau * PP
                for comp in range(2):
                    for i in range(n):
                        for j in range(n):
                            add(self.idx_m(c, comp, i), self.idx_p(c, j), -G[comp][i, j], Tr, Tc, Tv)
                            add(self.idx_p(c, j), self.idx_m(c, comp, i), G[comp][i, j], Tr, Tc, Tv)
                for i in range(n):
                    for j in range(n):
                        add(self.idx_p(c, i), self.idx_p(c, j), SigT[i, j], Tr, Tc, Tv)
                for (F, PP, SP, SS, nT) in finfo:
                    if m.face_type[F] in (mmesh.FT_BND_FLUID, mmesh.FT_BND_SOLID):
                        continue
                    for l in range(f):
                        col = self.idx_pF(F, l)
                        for comp in range(2):
                            for i in range(n):
                                g = nT[comp] * SP[i, l]              # G_TF[(comp,i),(F,l)]
                                add(self.idx_m(c, comp, i), col, -g, TFr, TFc, TFv)
                                add(col, self.idx_m(c, comp, i), g, FTr, FTc, FTv)
                        for i in range(n):
                            s = -tau * SP[i, l]                      # Sigma_TF[i,(F,l)]
                            add(self.idx_p(c, i), col, s, TFr, TFc, TFv)
                            add(col, self.idx_p(c, i), s, FTr, FTc, FTv)
                        for l2 in range(f):
                            add(col, self.idx_pF(F, l2), tau * SS[l, l2], Fr, Fc, Fv)
            else:
                rho, lam, mu = self.rho[c], self.lam[c], self.mu[c]
                # (C^-1 s, b)_T = sum_{c,c'} s_c' b_c D[c, c'] (phi, phi)_T
                D = np.array([[np.sum(compliance(lam, mu, E_BASIS[cp]) * E_BASIS[cc]) for cp in range(3)]
                              for cc in range(3)])
                for cc in range(3):
                    for cp in range(3):
                        if D[cc, cp] == 0.0:
                            continue
                        for i in range(n):
                            for j in range(n):
                                add(self.idx_s(c, cc, i), self.idx_s(c, cp, j), D[cc, cp] * M0[i, j], Mr, Mc, Mv)
                for d in range(2):
                    for i in range(n):
                        for j in range(n):
                            add(self.idx_v(c, d, i), self.idx_v(c, d, j), rho * M0[i, j], Mr, Mc, Mv)
                # H_T[(cc,i),(d,j)] = (grad_sym(phi_j e_d), phi_i E_cc)_T - sum_F (E_cc n_T)_d (phi_j, phi_i)_F
                H = {}
                for cc in range(3):
                    for d in range(2):
                        Hm = np.zeros((n, n))
                        for q in range(2):
                            coef = sym_grad_coef(cc, d, q)
                            if coef != 0.0:
                                Hm += coef * Dq[q]
                        for (F, PP, SP, SS, nT) in finfo:
                            En = E_BASIS[cc] @ nT
                            Hm -= En[d] * PP
                        H[(cc, d)] = Hm
                SigT = np.zeros((n, n))
                for (F, PP, SP, SS, nT) in finfo:
                    SigT += tau * PP
                for cc in range(3):
                    for d in range(2):
                        Hm = H[(cc, d)]
                        for i in range(n):
                            for j in range(n):
                                add(self.idx_s(c, cc, i), self.idx_v(c, d, j), -Hm[i, j], Tr, Tc, Tv)
                                add(self.idx_v(c, d, j), self.idx_s(c, cc, i), Hm[i, j], Tr, Tc, Tv)
                for d in range(2):
                    for i in range(n):
                        for j in range(n):
                            add(self.idx_v(c, d, i), self.idx_v(c, d, j), SigT[i, j], Tr, Tc, Tv)
                for (F, PP, SP, SS, nT) in finfo:
                    if m.face_type[F] in (mmesh.FT_BND_FLUID, mmesh.FT_BND_SOLID):
                        continue
                    for d in range(2):
                        for l in range(f):
                            col = self.idx_vF(F, d, l)
                            for cc in range(3):
                                En = E_BASIS[cc] @ nT
                                for i in range(n):
                                    h_ = En[d] * SP[i, l]            # H_TF[(cc,i),(F,d,l)]
                                    add(self.idx_s(c, cc, i), col, -h_, TFr, TFc, TFv)
                                    add(col, self.idx_s(c, cc, i), h_, FTr, FTc, FTv)
                            for i in range(n):
                                s = -tau * SP[i, l]
                                add(self.idx_v(c, d, i), col, s, TFr, TFc, TFv)
                                add(col, self.idx_v(c, d, i), s, FTr, FTc, FTv)
                            for l2 in range(f):
                                add(col, self.idx_vF(F, d, l2), tau * SS[l, l2], Fr, Fc, Fv)
        # coupling block on interface faces: Q_F^T C V_F = (v_F . n_Gamma, q_F)_F
        for F in range(m.n_faces):
            if m.face_type[F] != mmesh.FT_IFACE:
                continue
            c0, c1 = m.face_cells[F]
            cs = c0 if m.cell_domain[c0] == mmesh.SOLID else c1
            _, _, SS, n_gamma = self.local_face_integrals(F, cs)      # outward of the solid cell
            for l in range(f):
                for d in range(2):
                    for l2 in range(f):
                        cval = n_gamma[d] * SS[l, l2]                   # C[(F,l),(F,d,l2)]
                        add(self.idx_pF(F, l), self.idx_vF(F, d, l2), cval, Fr, Fc, Fv)
                        add(self.idx_vF(F, d, l2), self.idx_pF(F, l), -cval, Fr, Fc, Fv)
        nT, nF = self.nT, self.nF
        self.M = sp.csc_matrix((Mv, (Mr, Mc)), shape=(nT, nT))
        self.KT = sp.csr_matrix((Tv, (Tr, Tc)), shape=(nT, nT))
        self.KTF = sp.csr_matrix((TFv, (TFr, TFc)), shape=(nT, nF))
        self.KFT = sp.csr_matrix((FTv, (FTr, FTc)), shape=(nF, nT))
        self.KF = sp.csc_matrix((Fv, (Fr, Fc)), shape=(nF, nF))

    # ---- dependence on the stabilisation weights -------------------------------
    def tau_material_derivatives(self):
        """d tau_c / d(rho, kappa, lambda, mu) per cell ([nc, 4]).

        tau^f = eta_f / (rho c_P) = eta_f (rho kappa)^(-1/2) in fluid cells and
        tau^s = eta_s rho c^s in solid cells, with c^s = c_P
        (tau^s = eta_s (rho (lambda + 2 mu))^(1/2)) or c_S
        (eta_s (rho mu)^(1/2)) (Sec. 3.3 with the eta weights of Sec. 5.1;
        the optional 1/k factor cancels in the logarithmic derivatives).
        Zero when the weights were given explicitly (tau_override)."""
        m = self.mesh
        d = np.zeros((m.n_cells, 4))
        if self.tau_fixed:
            return d
        for c in range(m.n_cells):
            t = self.tau[c]
            if m.cell_domain[c] == mmesh.FLUID:
                d[c, 0] = -0.5 * t / self.rho[c]
                d[c, 1] = -0.5 * t / self.kappa[c]
            elif self.stab_speed == "cp":
                l2m = self.lam[c] + 2.0 * self.mu[c]
                d[c, 0] = 0.5 * t / self.rho[c]
                d[c, 2] = 0.5 * t / l2m
                d[c, 3] = t / l2m
            else:
                d[c, 0] = 0.5 * t / self.rho[c]
                d[c, 3] = 0.5 * t / self.mu[c]
        return d

    def stab_form(self, c):
        """dK/dtau_c of the full system: the least-squares stabilisation of
        cell c without its weight (Eq. stab), sum over the faces F of c of
        (u_c|_F - u_F, w_c|_F - w_F)_F on the primal unknowns (p in a fluid
        cell, both components of v in a solid cell), u_F = 0 on boundary
        faces.  Sparse over the stacked vector [U_T; U_F] (nT + nF)."""
        m = self.mesh
        n, f, nT = self.n, self.f, self.nT
        R, C, V = [], [], []
        fluid = m.cell_domain[c] == mmesh.FLUID
        comps = [None] if fluid else [0, 1]
        for F in m.cell_faces[c]:
            PP, SP, SS, _ = self.local_face_integrals(F, c)
            bnd = m.face_type[F] in (mmesh.FT_BND_FLUID, mmesh.FT_BND_SOLID)
            for d in comps:
                cell = [self.idx_p(c, i) if fluid else self.idx_v(c, d, i) for i in range(n)]
                face = [] if bnd else [nT + (self.idx_pF(F, l) if fluid else self.idx_vF(F, d, l)) for l in range(f)]
                for i in range(n):
                    for j in range(n):
                        R.append(cell[i]); C.append(cell[j]); V.append(PP[i, j])
                for i in range(n if face else 0):
                    for l in range(len(face)):
                        R.append(cell[i]); C.append(face[l]); V.append(-SP[i, l])
                        R.append(face[l]); C.append(cell[i]); V.append(-SP[i, l])
                for l in range(len(face)):
                    for l2 in range(len(face)):
                        R.append(face[l]); C.append(face[l2]); V.append(SS[l, l2])
        N = nT + self.nF
        return sp.csr_matrix((V, (R, C)), shape=(N, N))

    # ---- sources -------------------------------------------------------------
    def point_load(self, x: float, y: float, direction=(0.0, 1.0), cell: int | None = None):
        """Load-vector pattern b of a unit point source at (x, y).

        In a solid cell: a point force (f^s, w)_T = w(x_s) . e_dir in the
        velocity equation.  In a fluid cell: (f^f, q)_T = q(x_s) in the
        pressure equation.  The caller multiplies by the wavelet w(t).
        """
        c = locate_cell(self.mesh, x, y) if cell is None else cell
        xT, yT, h = self.cell_frame(c)
        phi = eval_cell_basis(self.k, xT, yT, h, [x], [y])[0]
        b = np.zeros(self.nT)
        if self.mesh.cell_domain[c] == mmesh.SOLID:
            for d in range(2):
                for i in range(self.n):
                    b[self.idx_v(c, d, i)] += direction[d] * phi[i]
        else:
            for i in range(self.n):
                b[self.idx_p(c, i)] += phi[i]
        return b, c

    def quad_points(self, order: int):
        """Per-cell fan quadrature (points, weights) for smooth integrands."""
        out = []
        m = self.mesh
        for c in range(m.n_cells):
            vs = mmesh.cell_vertices(m, c)
            px = [m.xy[v, 0] for v in vs]
            py = [m.xy[v, 1] for v in vs]
            out.append(fan_rule(px, py, m.cell_centroid[c], order))
        return out

    def load_matrix(self, order: int = 8):
        """Sparse Q with F = Q @ [f^f at all points ; f^s_x ; f^s_y] for a distributed source.

        Returns (Q, xq, yq, dom_q) where the source values must be stacked as
        [ff(xq,yq) (fluid points, 0 elsewhere), fsx, fsy]."""
        qp = self.quad_points(order)
        xs, ys, ws, cells = [], [], [], []
        for c, (pts, wts) in enumerate(qp):
            xs.append(pts[:, 0]); ys.append(pts[:, 1]); ws.append(wts); cells.append(np.full(len(wts), c))
        xq = np.concatenate(xs); yq = np.concatenate(ys); wq = np.concatenate(ws); cq = np.concatenate(cells)
        nq = len(wq)
        R, C, V = [], [], []
        start = 0
        for c, (pts, wts) in enumerate(qp):
            xT, yT, h = self.cell_frame(c)
            phi = eval_cell_basis(self.k, xT, yT, h, pts[:, 0], pts[:, 1])
            for g in range(len(wts)):
                col = start + g
                for i in range(self.n):
                    val = wts[g] * phi[g, i]
                    if self.mesh.cell_domain[c] == mmesh.FLUID:
                        R.append(self.idx_p(c, i)); C.append(col); V.append(val)
                    else:
                        R.append(self.idx_v(c, 0, i)); C.append(nq + col); V.append(val)
                        R.append(self.idx_v(c, 1, i)); C.append(2 * nq + col); V.append(val)
            start += len(wts)
        Q = sp.csr_matrix((V, (R, C)), shape=(self.nT, 3 * nq))
        return Q, xq, yq, self.mesh.cell_domain[cq]

    def project(self, fields, order: int = 8):
        """L2 projection of analytic fields onto the cell spaces.

        ``fields(x, y, domain)`` returns an array [ncomp, len(x)]: 3 components
        (m_x, m_y, p) for fluid points, 5 (s_xx, s_yy, s_xy, v_x, v_y) for solid.
        """
        U = np.zeros(self.nT)
        m = self.mesh
        for c, (pts, wts) in enumerate(self.quad_points(order)):
            xT, yT, h = self.cell_frame(c)
            phi = eval_cell_basis(self.k, xT, yT, h, pts[:, 0], pts[:, 1])
            vals = np.asarray(fields(pts[:, 0], pts[:, 1], int(m.cell_domain[c])))
            rhs = phi.T @ (wts[:, None] * vals.T)          # (n, ncomp)
            coef = np.linalg.solve(self.M0[c], rhs)
            for comp in range(vals.shape[0]):
                for i in range(self.n):
                    U[self.cell_off[c] + comp * self.n + i] = coef[i, comp]
        return U


def point_in_polygon(px, py, x, y, tol=1e-12):
    """Inclusive point-in-polygon test (boundary counts as inside)."""
    nv = len(px)
    scale = max(max(px) - min(px), max(py) - min(py))
    for i in range(nv):
        j = (i + 1) % nv
        ex, ey = px[j] - px[i], py[j] - py[i]
        cr = ex * (y - py[i]) - ey * (x - px[i])
        if cr < -tol * scale * scale:
            return False            # strictly right of a CCW edge of a convex cell
    return True


def locate_cell(mesh: mmesh.Mesh, x: float, y: float) -> int:
    """Lowest-index cell containing (x, y) (convex cells; boundary inclusive)."""
    for c in range(mesh.n_cells):
        vs = mmesh.cell_vertices(mesh, c)
        if point_in_polygon([mesh.xy[v, 0] for v in vs], [mesh.xy[v, 1] for v in vs], x, y):
            return c
    raise ValueError("point (%g, %g) outside the mesh" % (x, y))
