"""Coefficient sets of the time integrators of Sec. 4.2-4.3.

The paper names its schemes but prints none of their coefficients:

* ROW2 = ROS2PR (3 stages, order 2), ROW3 = ROS34PW2 (4 stages, order 3),
  ROW4 = RODASP (6 stages, order 4), all stiffly accurate (Sec. 4.3);
* ESDIRK2 (3 stages, order 2), ESDIRK3 (4 stages, order 3), ESDIRK4
  (6 stages, order 4) with a_11 = 0 and a_ii = omega otherwise (Sec. 4.2).

ROS34PW2, RODASP, ESDIRK3 and ESDIRK4 are entered from their publications
(ESDIRK3/4 are the implicit parts of the ARK3(2)4L[2]SA / ARK4(3)6L[2]SA
additive schemes).  ESDIRK2 is the stiffly accurate L-stable 3-stage scheme
with gamma = 1 - sqrt(2)/2 and b = (sqrt2/4, sqrt2/4, gamma).  The ROS2PR
coefficients were not available, so ROW2 is constructed from the properties
the paper states (3 stages, order 2, stiffly accurate): W-order 2, stability
function matching exp(z) to third order (which fixes gamma as the root
0.43586652150845... of gamma^3 - 3 gamma^2 + 3/2 gamma - 1/6 = 0), and
stage 3 sampled at alpha_3j = b_j / (1 - gamma).

Every Rosenbrock set is stored in the Hairer-Wanner (alpha, Gamma, b) form and
converted to the form of Eq. Rosenbrock_General,
  (I/(omega dt) - dR/dq) Y_i = R(q^n + sum_j a_ij Y_j) + (1/dt) sum_j c_ij Y_j,
  q^{n+1} = q^n + sum_j m_j Y_j,
with omega = gamma, a = alpha Gamma^-1, c = diag(1/gamma) - Gamma^-1 and
m = b Gamma^-1 (Y_i = sum_j Gamma_ij k_j).  RODASP is entered directly in that
transformed form.

Pins (tests/test_oracle_tableaus.py): the Butcher / Rosenbrock order
conditions up to each scheme's order, stiff accuracy, L-stability
(R(infinity) = 0 and |R(iy)| <= 1), and the observed order on a nonlinear ODE.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class RowTableau:
    name: str
    order: int
    gamma: float          # omega of Eq. Rosenbrock_General
    a: np.ndarray         # (s, s) strictly lower
    c: np.ndarray         # (s, s) strictly lower
    m: np.ndarray         # (s,)

    @property
    def stages(self):
        return len(self.m)

    def alpha_form(self):
        """(alpha, Gamma, b) of the Hairer-Wanner form."""
        s = self.stages
        Ginv = np.diag(np.full(s, 1.0 / self.gamma)) - self.c
        G = np.linalg.inv(Ginv)
        return self.a @ G, G, self.m @ G


@dataclass(frozen=True)
class EsdirkTableau:
    name: str
    order: int
    A: np.ndarray         # (s, s) lower triangular, A[0,0] = 0, A[i,i] = omega
    b: np.ndarray

    @property
    def stages(self):
        return len(self.b)

    @property
    def omega(self):
        return float(self.A[1, 1])


def _from_alpha(name, order, alpha, G, b):
    alpha = np.asarray(alpha, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    g = G[0, 0]
    Ginv = np.linalg.inv(G)
    a = alpha @ Ginv
    c = np.diag(np.diag(Ginv)) - Ginv
    c = np.tril(c, -1)
    a = np.tril(a, -1)
    m = b @ Ginv
    return RowTableau(name, order, float(g), a, c, m)


def row2():
    """3-stage, order-2, stiffly accurate ROW (constructed; see module doc)."""
    # root of g^3 - 3 g^2 + 3/2 g - 1/6 in (0, 1) by Newton
    g = 0.4
    for _ in range(60):
        g -= (g ** 3 - 3 * g ** 2 + 1.5 * g - 1.0 / 6.0) / (3 * g ** 2 - 6 * g + 1.5)
    a21 = 2 * g
    b2 = (0.5 - g) / a21
    g21 = (g * g - g) / b2
    b3 = g
    b1 = 1.0 - b2 - b3
    a31 = b1 / (1.0 - g)
    a32 = b2 / (1.0 - g)
    alpha = np.array([[0, 0, 0], [a21, 0, 0], [a31, a32, 0]])
    G = np.array([[g, 0, 0], [g21, g, 0], [b1 - a31, b2 - a32, g]])
    return _from_alpha("ROW2", 2, alpha, G, [b1, b2, b3])


def ros34pw2():
    """ROS34PW2 of Rang & Angermann (2005): 4 stages, order 3."""
    g = 4.3586652150845900e-01
    alpha = np.zeros((4, 4))
    alpha[1, 0] = 8.7173304301691801e-01
    alpha[2, :2] = [8.4457060015369423e-01, -1.1299064236484185e-01]
    alpha[3, :3] = [0.0, 0.0, 1.0]
    G = np.eye(4) * g
    G[1, 0] = -8.7173304301691801e-01
    G[2, :2] = [-9.0338057013044082e-01, 5.4180672388095326e-02]
    G[3, :3] = [2.4212380706095346e-01, -1.2232505839045147e+00, 5.4526025533510214e-01]
    b = [2.4212380706095346e-01, -1.2232505839045147e+00, 1.5452602553351020e+00, g]
    return _from_alpha("ROW3", 3, alpha, G, b)


def rodasp():
    """RODASP of Steinebach (1995): 6 stages, order 4, transformed form."""
    s = 6
    a = np.zeros((s, s))
    c = np.zeros((s, s))
    a[1, 0] = 3.0
    a[2, :2] = [1.831036793486759, 0.4955183967433795]
    a[3, :3] = [2.304376582692669, -0.05249275245743001, -1.176798761832782]
    row5 = [-7.170454962423024, -4.741636671481785, -16.31002631330971, -1.062004044111401]
    a[4, :4] = row5
    a[5, :5] = row5 + [1.0]
    c[1, 0] = -12.0
    c[2, :2] = [-8.791795173947035, -2.207865586973518]
    c[3, :3] = [10.81793056857153, 6.780270611428266, 19.53485944642410]
    c[4, :4] = [34.19095006749676, 15.49671153725963, 54.74760875964130, 14.16005392148534]
    c[5, :5] = [34.62605830930532, 15.30084976114473, 56.99955578662667, 18.40807009793095,
                -5.714285714285717]
    m = np.array(row5 + [1.0, 1.0])
    return RowTableau("ROW4", 4, 0.25, a, c, m)


def esdirk2():
    g = 1.0 - math.sqrt(2.0) / 2.0
    r = math.sqrt(2.0) / 4.0
    A = np.array([[0.0, 0.0, 0.0], [g, g, 0.0], [r, r, g]])
    return EsdirkTableau("ESDIRK2", 2, A, A[-1].copy())


def esdirk3():
    g = 1767732205903 / 4055673282236
    A = np.array([
        [0.0, 0.0, 0.0, 0.0],
        [g, g, 0.0, 0.0],
        [2746238789719 / 10658868560708, -640167445237 / 6845629431997, g, 0.0],
        [1471266399579 / 7840856788654, -4482444167858 / 7529755066697,
         11266239266428 / 11593286722821, g]])
    return EsdirkTableau("ESDIRK3", 3, A, A[-1].copy())


def esdirk4():
    q = 0.25
    A = np.zeros((6, 6))
    A[1, :2] = [q, q]
    A[2, :3] = [8611 / 62500, -1743 / 31250, q]
    A[3, :4] = [5012029 / 34652500, -654441 / 2922500, 174375 / 388108, q]
    A[4, :5] = [15267082809 / 155376265600, -71443401 / 120774400, 730878875 / 902184768,
                2285395 / 8070912, q]
    A[5, :] = [82889 / 524892, 0.0, 15625 / 83664, 69875 / 102672, -2260 / 8211, q]
    return EsdirkTableau("ESDIRK4", 4, A, A[-1].copy())


ROW = {2: row2, 3: ros34pw2, 4: rodasp}
ESDIRK = {2: esdirk2, 3: esdirk3, 4: esdirk4}

# BDF2 of Eq. BDF: q^{n+1} = dt*omega*R(q^{n+1}) + a1 q^n + a2 q^{n-1}
BDF2_OMEGA = 2.0 / 3.0
BDF2_A = (4.0 / 3.0, -1.0 / 3.0)
