"""Closed-form solutions used to pin the oracle (not part of the oracle).

* ``Sinusoid``: the manufactured solution of Sec. 5.1 (Eq. non_poly_sol):
  u = x^2 sin(w pi x) sin(w pi y) sin(th pi t) in the fluid (0,1)^2,
  u_x = u_y = x^2 cos(w pi x / 2) sin(w pi y) cos(th pi t) in the solid
  (-1,0)x(0,1), with p = du/dt, m = grad u, v = du/dt, C^-1 s = grad_sym u,
  rho = kappa = 1 and lambda = mu = 1 (c_P = sqrt 3, c_S = 1).  The sources are
  f^f = (1/kappa) dp/dt - div m and f^s = rho dv/dt - div s, written out by hand
  below and checked against finite differences in the tests.
* ``plane_wave``: normal-incidence fluid/solid reflection and transmission
  (1D Riemann problem with impedances Z_f = rho_f c_f and Z_s = rho_s c_P).
"""
import numpy as np


class Sinusoid:
    def __init__(self, w=1.0, th=np.sqrt(2.0), lam=1.0, mu=1.0, rho=1.0, kappa=1.0):
        self.w, self.th, self.lam, self.mu, self.rho, self.kappa = w, th, lam, mu, rho, kappa

    # fluid ---------------------------------------------------------------
    def fluid_fields(self, x, y, t):
        W, T = self.w * np.pi, self.th * np.pi
        sx, cx, sy, cy = np.sin(W * x), np.cos(W * x), np.sin(W * y), np.cos(W * y)
        st, ct = np.sin(T * t), np.cos(T * t)
        p = T * x ** 2 * sx * sy * ct
        mx = (2 * x * sx + W * x ** 2 * cx) * sy * st
        my = W * x ** 2 * sx * cy * st
        return np.array([mx, my, p])

    def fluid_source(self, x, y, t):
        W, T = self.w * np.pi, self.th * np.pi
        sx, cx, sy = np.sin(W * x), np.cos(W * x), np.sin(W * y)
        st = np.sin(T * t)
        u = x ** 2 * sx * sy * st
        lap = (2 * sx + 4 * W * x * cx - W ** 2 * x ** 2 * sx) * sy * st - W ** 2 * x ** 2 * sx * sy * st
        # (1/kappa) d2u/dt2 - lap u with rho = 1 (m = grad u)
        return -(T ** 2) * u / self.kappa - lap

    # solid ---------------------------------------------------------------
    def _g(self, x):
        a = self.w * np.pi / 2
        g = x ** 2 * np.cos(a * x)
        g1 = 2 * x * np.cos(a * x) - a * x ** 2 * np.sin(a * x)
        g2 = 2 * np.cos(a * x) - 4 * a * x * np.sin(a * x) - a ** 2 * x ** 2 * np.cos(a * x)
        return g, g1, g2

    def solid_fields(self, x, y, t):
        W, T = self.w * np.pi, self.th * np.pi
        g, g1, _ = self._g(x)
        sy, cy = np.sin(W * y), np.cos(W * y)
        ct, st = np.cos(T * t), np.sin(T * t)
        exx = g1 * sy * ct
        eyy = g * W * cy * ct
        exy = 0.5 * (g * W * cy + g1 * sy) * ct
        lam, mu = self.lam, self.mu
        sxx = (lam + 2 * mu) * exx + lam * eyy
        syy = lam * exx + (lam + 2 * mu) * eyy
        sxy = 2 * mu * exy
        v = -T * g * sy * st
        return np.array([sxx, syy, sxy, v, v])

    def solid_source(self, x, y, t):
        W, T = self.w * np.pi, self.th * np.pi
        g, g1, g2 = self._g(x)
        sy, cy = np.sin(W * y), np.cos(W * y)
        ct = np.cos(T * t)
        lam, mu = self.lam, self.mu
        dx_exx = g2 * sy * ct
        dy_exx = g1 * W * cy * ct
        dx_eyy = g1 * W * cy * ct
        dy_eyy = -g * W ** 2 * sy * ct
        dx_exy = 0.5 * (g1 * W * cy + g2 * sy) * ct
        dy_exy = 0.5 * (-g * W ** 2 * sy + g1 * W * cy) * ct
        dx_sxx = (lam + 2 * mu) * dx_exx + lam * dx_eyy
        dy_syy = lam * dy_exx + (lam + 2 * mu) * dy_eyy
        dx_sxy = 2 * mu * dx_exy
        dy_sxy = 2 * mu * dy_exy
        dvdt = -(T ** 2) * g * sy * ct
        fx = self.rho * dvdt - (dx_sxx + dy_sxy)
        fy = self.rho * dvdt - (dx_sxy + dy_syy)
        return np.array([fx, fy])

    def fields(self, t):
        def f(x, y, dom):
            return self.fluid_fields(x, y, t) if dom == 0 else self.solid_fields(x, y, t)
        return f


def plane_wave(rho_f, c_f, rho_s, vp, vs, y0, sigma):
    """Downgoing Gaussian pulse p = g(y + c_f t), g(s) = exp(-((s - y0)/sigma)^2),
    hitting the interface y = 0 from the fluid (y > 0).  Returns
    fields(t) -> f(x, y, domain) and the coefficients (R, T) for the
    stress-like fields (p and s_yy)."""
    Zf = rho_f * c_f
    Zs = rho_s * vp
    R = (Zs - Zf) / (Zs + Zf)
    T = 2 * Zs / (Zs + Zf)
    mu = rho_s * vs * vs
    lam = rho_s * vp * vp - 2 * mu
    g = lambda s: np.exp(-((s - y0) / sigma) ** 2)

    def fields(t):
        def f(x, y, dom):
            z = np.zeros_like(np.asarray(x, dtype=float))
            if dom == 0:
                pin = g(y + c_f * t)
                pre = R * g(-y + c_f * t)
                p = pin + pre
                my = pin / Zf - pre / Zf
                return np.array([z, my, p])
            syy = T * g(c_f * (t + y / vp))
            sxx = lam / (lam + 2 * mu) * syy
            vy = syy / Zs
            return np.array([sxx, syy, z, z, vy])
        return f
    return fields, R, T
