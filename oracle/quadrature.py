"""Integration rules for the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``polygon_monomial``: exact integral of X^a Y^b over a polygon by Green's
  theorem, int_P X^a Y^b dX dY = sum over edges of int_e X^(a+1)/(a+1) Y^b dY,
  each edge integral done by Gauss-Legendre with enough points to be exact for
  the polynomial integrand.  This is how the oracle gets every cell integral
  of the paper's local operators (Eq. mass, Eq. rec, Eq. stab) exactly, up to
  rounding.
* ``gauss_legendre(q)``: nodes/weights on [-1, 1] (numpy's routine).
* ``fan_rule(px, py, order)``: quadrature for non-polynomial integrands
  (manufactured sources, initial data) on the fan of triangles from the
  centroid, with a collapsed (Duffy) Gauss-Legendre rule on each triangle.
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(q: int):
    x, w = np.polynomial.legendre.leggauss(q)
    return x, w


def polygon_monomial(X, Y, a: int, b: int) -> float:
    """Exact int over the CCW polygon with vertices (X_i, Y_i) of X^a Y^b dX dY."""
    nv = len(X)
    q = (a + b + 2) // 2 + 1
    s, w = gauss_legendre(q)
    t = 0.5 * (s + 1.0)          # map to [0, 1]
    wt = 0.5 * w
    total = 0.0
    for i in range(nv):
        j = (i + 1) % nv
        dX = X[j] - X[i]
        dY = Y[j] - Y[i]
        if dY == 0.0:
            continue
        xs = X[i] + t * dX
        ys = Y[i] + t * dY
        total += float(np.sum(wt * xs ** (a + 1) * ys ** b)) * dY / (a + 1)
    return total


def fan_rule(px, py, centre, order: int):
    """Points and weights integrating smooth functions over the polygon.

    Each fan triangle (centre, p_i, p_{i+1}) uses the collapsed map
    x = c + u (p_i - c) + u v (p_{i+1} - p_i), u, v in [0, 1], with Jacobian
    u * |det|; Gauss-Legendre with ``order`` points in u and v.
    """
    s, w = gauss_legendre(order)
    u = 0.5 * (s + 1.0)
    wu = 0.5 * w
    pts = []
    wts = []
    cx, cy = centre
    nv = len(px)
    for i in range(nv):
        j = (i + 1) % nv
        ax, ay = px[i] - cx, py[i] - cy
        bx, by = px[j] - px[i], py[j] - py[i]
        det = ax * by - ay * bx
        for iu in range(order):
            for iv in range(order):
                uu, vv = u[iu], u[iv]
                pts.append((cx + uu * ax + uu * vv * bx, cy + uu * ay + uu * vv * by))
                wts.append(wu[iu] * wu[iv] * uu * det)
    return np.array(pts), np.array(wts)
