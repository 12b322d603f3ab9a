"""1D building blocks of the FR scheme (Sec. 3).

* Gauss-Legendre solution points and weights: roots of P_{p+1} by Newton's
  method on the three-term Legendre recurrence.
* Lagrange basis l_k of the solution points, its values at the element ends
  xi = -1, +1, and the derivative matrix D_ik = l_k'(xi_i).
* Correction functions: the Radau polynomials that make FR recover nodal DG
  (Sec. 3, "we employ the Radau polynomials to recover the nodal FR-DG
  method"):  g_L = (-1)^(p+1)/2 * (P_{p+1} - P_p)  (g_L(-1) = 1, g_L(1) = 0)
  and g_R(xi) = g_L(-xi); their derivatives at the solution points.

Pins (tests/test_oracle_basis.py): nodes/weights against NumPy's leggauss,
quadrature exactness, D applied to monomials, g_L'(-1) = -(p+1)^2/2 closed form,
end values of g_L / g_R.
"""
from __future__ import annotations

import numpy as np


def legendre(n: int, x):
    """P_n(x) and P_n'(x) from the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    # derivative: (1 - x^2) P_n' = n (P_{n-1} - x P_n); use the series form at |x| = 1
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    end = np.isclose(np.abs(x), 1.0)
    if np.any(end):
        dp = np.where(end, 0.5 * n * (n + 1) * np.sign(x) ** (n + 1), dp)
    return p1, dp


def gauss_legendre(npts: int):
    """Nodes (ascending) and weights of the npts-point Gauss-Legendre rule."""
    k = np.arange(npts)
    x = -np.cos(np.pi * (k + 0.75) / (npts + 0.5))
    for _ in range(100):
        pn, dpn = legendre(npts, x)
        dx = pn / dpn
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dpn = legendre(npts, x)
    w = 2.0 / ((1.0 - x * x) * dpn * dpn)
    return x, w


def lagrange_values(nodes, x):
    """Matrix L[m, k] = l_k(x_m) of the Lagrange basis on ``nodes``."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for k in range(n):
        for j in range(n):
            if j != k:
                L[:, k] *= (x - nodes[j]) / (nodes[k] - nodes[j])
    return L


def derivative_matrix(nodes):
    """D[i, k] = l_k'(x_i) from the product rule of the Lagrange basis."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    D = np.zeros((n, n))
    for i in range(n):
        for k in range(n):
            # l_k'(x) = sum_{m != k} 1/(x_k - x_m) prod_{j != k, m} (x - x_j)/(x_k - x_j)
            s = 0.0
            for m in range(n):
                if m == k:
                    continue
                prod = 1.0 / (nodes[k] - nodes[m])
                for j in range(n):
                    if j != k and j != m:
                        prod *= (nodes[i] - nodes[j]) / (nodes[k] - nodes[j])
                s += prod
            D[i, k] = s
    return D


def radau_gl(p: int, x):
    """Left correction function g_L (right Radau polynomial of degree p+1) and
    its derivative at x."""
    sgn = (-1.0) ** (p + 1)
    P1, dP1 = legendre(p + 1, x)
    P0, dP0 = legendre(p, x)
    return 0.5 * sgn * (P1 - P0), 0.5 * sgn * (dP1 - dP0)


def radau_gr(p: int, x):
    """Right correction function g_R(xi) = g_L(-xi) and its derivative."""
    x = np.asarray(x, dtype=np.float64)
    g, dg = radau_gl(p, -x)
    return g, -dg


class Basis:
    """All 1D tables of degree ``p`` on Gauss-Legendre solution points."""

    def __init__(self, p: int):
        self.p = p
        self.n = p + 1
        self.xi, self.w = gauss_legendre(p + 1)
        self.D = derivative_matrix(self.xi)
        ends = lagrange_values(self.xi, [-1.0, 1.0])
        self.lm = ends[0]          # l_k(-1)
        self.lp = ends[1]          # l_k(+1)
        self.dgL = radau_gl(p, self.xi)[1]  # g_L'(xi_i)
        self.dgR = radau_gr(p, self.xi)[1]  # g_R'(xi_i)
