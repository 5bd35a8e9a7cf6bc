"""Energy, dissipation and sensors (Sec. 5 of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``energy``: E^n = 1/2 |m|^2_rho + 1/2 |p|^2_(1/kappa) + 1/2 |v|^2_rho
  + 1/2 |s|^2_(C^-1) (Sec. 5.1), i.e. 1/2 U^T M U.
* ``dissipation``: U_T^T (K_T - K_TF K_F^-1 K_FT) U_T.  The skew parts
  (reconstruction and coupling) cancel in this quadratic form and what is left
  is sum_T tau_T |S_dT(U_T, U_dT)|^2_dT >= 0 (a consequence of Eq. rec,
  Eq. stab and the coupling block); the tests check that identity with an
  independent face quadrature.
* ``sensors``: point values of the cell polynomials, or of the face unknowns
  on an interface face (the interface sensor of Sec. 5.2).  Output per sensor:
  fluid [p, m_x, m_y, 0, 0]; solid [v_x, v_y, s_xx, s_yy, s_xy];
  interface [p_F, v_Fx, v_Fy, 0, 0].
"""
from __future__ import annotations

import numpy as np

from . import mesh as mmesh
from .assemble import locate_cell
from .spaces import eval_cell_basis


def energy(system, U) -> float:
    return 0.5 * float(U @ (system.M @ U))


def dissipation(stepper, U) -> float:
    sys_ = stepper.sys
    UF = stepper.face_solve(U)
    return float(U @ (sys_.KT @ U + sys_.KTF @ UF))


def find_interface_face(mesh, x, y, tol=1e-10):
    for F in range(mesh.n_faces):
        if mesh.face_type[F] != mmesh.FT_IFACE:
            continue
        A, B = mesh.face_ends[F]
        t = B - A
        L2 = float(t @ t)
        s = float((np.array([x, y]) - A) @ t) / L2
        if -tol <= s <= 1 + tol:
            d = abs(t[0] * (y - A[1]) - t[1] * (x - A[0])) / np.sqrt(L2)
            if d <= tol * np.sqrt(L2):
                return F, 2.0 * s - 1.0
    return None, None


def sensors(stepper, U, points):
    sys_ = stepper.sys
    m = sys_.mesh
    out = np.zeros((len(points), 5))
    UF = None
    for r, (x, y) in enumerate(points):
        F, xi = find_interface_face(m, x, y)
        if F is not None:
            if UF is None:
                UF = stepper.face_solve(U)
            psi = np.array([xi ** l for l in range(sys_.f)])
            out[r, 0] = psi @ UF[[sys_.idx_pF(F, l) for l in range(sys_.f)]]
            for d in range(2):
                out[r, 1 + d] = psi @ UF[[sys_.idx_vF(F, d, l) for l in range(sys_.f)]]
            continue
        c = locate_cell(m, x, y)
        xT, yT, h = sys_.cell_frame(c)
        phi = eval_cell_basis(sys_.k, xT, yT, h, [x], [y])[0]
        n = sys_.n
        base = sys_.cell_off[c]
        if m.cell_domain[c] == mmesh.FLUID:
            out[r, 0] = phi @ U[base + 2 * n: base + 3 * n]
            out[r, 1] = phi @ U[base: base + n]
            out[r, 2] = phi @ U[base + n: base + 2 * n]
        else:
            out[r, 0] = phi @ U[base + 3 * n: base + 4 * n]
            out[r, 1] = phi @ U[base + 4 * n: base + 5 * n]
            for comp in range(3):
                out[r, 2 + comp] = phi @ U[base + comp * n: base + (comp + 1) * n]
    return out


def l2_error(system, U, exact, order: int = 8, comps=None):
    """sqrt(sum_T int_T |u_h - u|^2) over the selected components.

    ``exact(x, y, domain)`` as in ``System.project``; ``comps`` maps domain ->
    list of component indices (default: all)."""
    m = system.mesh
    err = 0.0
    ref = 0.0
    for c, (pts, wts) in enumerate(system.quad_points(order)):
        d = int(m.cell_domain[c])
        xT, yT, h = system.cell_frame(c)
        phi = eval_cell_basis(system.k, xT, yT, h, pts[:, 0], pts[:, 1])
        vals = np.asarray(exact(pts[:, 0], pts[:, 1], d))
        sel = range(vals.shape[0]) if comps is None else comps[d]
        for comp in sel:
            coef = U[system.cell_off[c] + comp * system.n: system.cell_off[c] + (comp + 1) * system.n]
            diff = phi @ coef - vals[comp]
            err += float(wts @ diff ** 2)
            ref += float(wts @ vals[comp] ** 2)
    return np.sqrt(err), np.sqrt(ref)
