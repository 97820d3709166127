"""Brute-force quadrature used only to pin the oracle: Duffy-transformed
Gauss-Legendre rules on a flat triangle, written independently of the oracle
(different rule, different parametrisation)."""
from __future__ import annotations

import numpy as np

_GL_CACHE = {}


def gauss_legendre(n, a=0.0, b=1.0):
    if n not in _GL_CACHE:
        _GL_CACHE[n] = np.polynomial.legendre.leggauss(n)
    x, w = _GL_CACHE[n]
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


# graded radial intervals: resolve the near-singular peak of an off-plane point
_U_BREAKS = [0.0, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 0.05, 0.2, 0.5, 1.0]


def triangle_integral(r, tri, func, n=24):
    """int_T func(rp, R) dS' for R = |r - rp|, by splitting T into three
    triangles with apex at the projection of r onto T's plane and a
    polar-like Duffy map in each (Jacobian proportional to the radius,
    which cancels a 1/R singularity).  func returns [..., m] arrays."""
    tri = np.asarray(tri, float).reshape(3, 3)
    nrm = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    nrm /= np.linalg.norm(nrm)
    r = np.asarray(r, float)
    rho = r - np.dot(r - tri[0], nrm) * nrm
    total = None
    for e in range(3):
        a, b = tri[e], tri[(e + 1) % 3]
        # signed area of (rho, a, b) relative to the triangle normal
        jac = np.dot(np.cross(a - rho, b - a), nrm)
        if abs(jac) < 1e-300:
            continue
        # the integrand peaks in v at the foot of the perpendicular from rho
        # onto the edge line: grade the v intervals geometrically towards it
        vs = float(np.clip(np.dot(rho - a, b - a) / np.dot(b - a, b - a), 0.0, 1.0))
        vb = {0.0, 1.0, vs}
        for g in (1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 0.03, 0.1, 0.3):
            vb.update(x for x in (vs - g, vs + g) if 0.0 < x < 1.0)
        vb = sorted(vb)
        parts = [gauss_legendre(n, v0, v1) for v0, v1 in zip(vb[:-1], vb[1:]) if v1 > v0]
        xv = np.concatenate([p[0] for p in parts])
        wv = np.concatenate([p[1] for p in parts])
        for u0, u1 in zip(_U_BREAKS[:-1], _U_BREAKS[1:]):
            xu, wu = gauss_legendre(n, u0, u1)
            U, V = np.meshgrid(xu, xv, indexing="ij")
            W = np.outer(wu, wv) * U * jac
            pts = rho[None, None, :] + U[..., None] * ((a - rho)[None, None, :]
                                                       + V[..., None] * (b - a)[None, None, :])
            R = np.linalg.norm(pts - r[None, None, :], axis=-1)
            val = func(pts, R)
            contrib = np.einsum("ij,ij...->...", W, val)
            total = contrib if total is None else total + contrib
    return total
