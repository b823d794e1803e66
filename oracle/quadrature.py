"""Conical-product Gauss rule on the reference tetrahedron (Stroud, 1971).

The unit cube (u, v, w) in [0,1]^3 is mapped onto the reference tetrahedron by
x = u, y = (1-u) v, z = (1-u)(1-v) w with Jacobian (1-u)^2 (1-v). With q
Gauss-Legendre points per direction the rule integrates polynomials of total
degree <= 2q - 3 exactly. Used only to pin the closed-form element integrals
and to measure L2 errors; the matrices themselves use exact monomial formulas.
"""

from __future__ import annotations

import numpy as np


def gauss01(q: int, a: float = 0.0, b: float = 1.0):
    x, w = np.polynomial.legendre.leggauss(q)
    return a + (b - a) * (x + 1.0) / 2.0, w * (b - a) / 2.0


def reference_tet_rule(q: int = 6, u_split: float | None = None):
    """Points (P, 4) as barycentric coordinates and weights (P,) summing to 1/6.

    lam_1 = x = u, so ``u_split`` lets the u-integral be split at a kink of an
    integrand that depends on lam_1 (the rule is then exact piecewise).
    """
    if u_split is None:
        us, wu = gauss01(q)
    else:
        u1, w1 = gauss01(q, 0.0, u_split)
        u2, w2 = gauss01(q, u_split, 1.0)
        us, wu = np.concatenate([u1, u2]), np.concatenate([w1, w2])
    vs, wv = gauss01(q)
    ws, ww = gauss01(q)
    U, V, Wc = np.meshgrid(us, vs, ws, indexing="ij")
    WU, WV, WW = np.meshgrid(wu, wv, ww, indexing="ij")
    x = U
    y = (1 - U) * V
    z = (1 - U) * (1 - V) * Wc
    weight = WU * WV * WW * (1 - U) ** 2 * (1 - V)
    lam = np.stack([1 - x - y - z, x, y, z], axis=-1).reshape(-1, 4)
    return lam, weight.ravel()
