"""Quadrature on the reference tetrahedron (oracle side).

The paper does not state its quadrature.  The reading used on both sides of the parity tests: a conical-product
(collapsed-coordinate) rule made of Gauss-Jacobi rules in each direction, with 3 points per direction (27 points,
exact for total degree 5).  It integrates the P2 mass matrix (degree 4) exactly and keeps one degree for the
variation of potentials.  Nodes and weights are produced here by Golub-Welsch (eigen-decomposition of the Jacobi
matrix of the orthogonal polynomials), independently of the CUDA side, which builds the same rule its own way.
"""
from __future__ import annotations

import math

import numpy as np


def gauss_jacobi(n: int, a: float, b: float):
    """n-point Gauss rule on [-1, 1] for the weight (1-t)^a (1+t)^b, by Golub-Welsch."""
    k = np.arange(n, dtype=np.float64)
    s = 2.0 * k + a + b
    alpha = np.empty(n)
    for i in range(n):
        if i == 0:
            alpha[i] = (b - a) / (a + b + 2.0)
        else:
            alpha[i] = (b * b - a * a) / (s[i] * (s[i] + 2.0))
    beta = np.empty(max(n - 1, 0))
    for i in range(1, n):
        si = 2.0 * i + a + b
        beta[i - 1] = 4.0 * i * (i + a) * (i + b) * (i + a + b) / (si * si * (si + 1.0) * (si - 1.0))
    T = np.diag(alpha) + np.diag(np.sqrt(beta), 1) + np.diag(np.sqrt(beta), -1)
    x, V = np.linalg.eigh(T)
    mu0 = 2.0 ** (a + b + 1.0) * math.gamma(a + 1.0) * math.gamma(b + 1.0) / math.gamma(a + b + 2.0)
    w = mu0 * V[0, :] ** 2
    return x, w


def gauss_jacobi01(n: int, a: float):
    """n-point rule on [0, 1] for the weight (1-x)^a."""
    t, w = gauss_jacobi(n, a, 0.0)
    return 0.5 * (1.0 + t), w * 2.0 ** (-a - 1.0)


def tet_rule(n: int = 3):
    """Conical-product rule on the reference tetrahedron {xi, eta, zeta >= 0, xi+eta+zeta <= 1}.

    Collapsed coordinates: xi = u, eta = v (1-u), zeta = w (1-u)(1-v), with Jacobian (1-u)^2 (1-v); u carries
    the weight (1-u)^2, v the weight (1-v), w none.  Returns (points [n^3, 3], weights [n^3]); weights sum to 1/6.
    """
    u, wu = gauss_jacobi01(n, 2.0)
    v, wv = gauss_jacobi01(n, 1.0)
    s, ws = gauss_jacobi01(n, 0.0)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                pts.append((u[i], v[j] * (1.0 - u[i]), s[k] * (1.0 - u[i]) * (1.0 - v[j])))
                wts.append(wu[i] * wv[j] * ws[k])
    return np.array(pts), np.array(wts)
