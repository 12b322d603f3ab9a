"""Isentropic vortex of Sec. 5.1 and the error norm of its accuracy study.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``VortexCase`` / ``exact_state``: the exact solution of Eq. VP_Solution.  A
  free stream (rho, u, v) = (1, u_inf, v_inf) with gas constant R = 1 carries a
  perturbation centred at (x0, y0) + (u_inf, v_inf) t:
      du = -alpha/(2 pi) (y - yc) exp(phi (1 - r^2)),
      dv =  alpha/(2 pi) (x - xc) exp(phi (1 - r^2)),
      dT = -alpha^2 (gamma - 1)/(16 phi gamma pi^2) exp(2 phi (1 - r^2)),
  with zero entropy change (p / rho^gamma fixed), r the Euclidean distance to
  the centre (the printed "r = (x-x0)^2 + (y-y0)^2" is read as the distance,
  so the exponent is phi (1 - r^2)).  The Mach number 0.5 is taken on the
  free-stream speed |V| = sqrt(u_inf^2 + v_inf^2), so
  T_inf = p_inf / rho_inf = |V|^2 / (gamma Ma^2) (= 40/7 for u = v = 1).
  On a periodic box the centre is taken at its nearest periodic image.
* ``l2_error``: the error of Sec. 5.1, Error(s) = sqrt( int (s_exact -
  s_num)^2 dV / V ), V the area of the domain, with the integral taken by the
  Gauss-Legendre rule of the solution points on every affine element
  (weights w_i w_j |J_e|, |J_e| = hx hy / 4).
* ``vortex_errors``: E(s) for s = rho, u, v, p of a conserved state against
  the exact vortex at time t.

Pins (tests/test_oracle_vortex.py): the exact state is isentropic and in
radial equilibrium (dp/dr = rho u_theta^2 / r, checked by differences of the
state itself), has Mach 0.5 and the closed-form peak swirl alpha / (2 pi),
returns to itself after one period; R(U_exact(t)) + dU_exact/dt tends to zero
under refinement at the rate of the FR truncation error (a wrong amplitude or
exponent would leave an O(1) remainder); the norm is exact for piecewise
polynomial errors that the quadrature integrates exactly, on jittered
meshes, and equals |c| for a constant error c.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .basis import Basis
from .fr2d import Mesh


@dataclass(frozen=True)
class VortexCase:
    """Parameters of the isentropic vortex (Sec. 5.1 and its free stream)."""
    alpha: float = 5.0
    phi: float = 0.5
    gamma: float = 1.4
    mach: float = 0.5
    rho_inf: float = 1.0
    u_inf: float = 1.0
    v_inf: float = 1.0
    x0: float = 0.0
    y0: float = 0.0
    box: tuple = (-10.0, 10.0, -10.0, 10.0)

    @property
    def t_inf(self) -> float:
        """Free-stream temperature from c = |V| / Ma and c^2 = gamma R T, R = 1."""
        speed2 = self.u_inf ** 2 + self.v_inf ** 2
        return speed2 / (self.gamma * self.mach ** 2)

    @property
    def p_inf(self) -> float:
        return self.rho_inf * self.t_inf


def point_coordinates(mesh: Mesh, basis: Basis):
    """Physical coordinates (x, y), each (Ne, Np), of the solution points:
    element ix + nx*iy, point i + (p+1)*j, xi_i along x and eta_j along y."""
    n = basis.n
    x = np.empty((mesh.ne, n * n))
    y = np.empty((mesh.ne, n * n))
    for iy in range(mesh.ny):
        for ix in range(mesh.nx):
            e = ix + mesh.nx * iy
            xa, xb = mesh.x_edges[ix], mesh.x_edges[ix + 1]
            ya, yb = mesh.y_edges[iy], mesh.y_edges[iy + 1]
            for j in range(n):
                for i in range(n):
                    x[e, i + n * j] = 0.5 * (xa + xb) + 0.5 * (xb - xa) * basis.xi[i]
                    y[e, i + n * j] = 0.5 * (ya + yb) + 0.5 * (yb - ya) * basis.xi[j]
    return x, y


def exact_primitive(case: VortexCase, x, y, t: float = 0.0):
    """(rho, u, v, p) of the advected vortex at the points (x, y) and time t."""
    lx = case.box[1] - case.box[0]
    ly = case.box[3] - case.box[2]
    # centre after advection by the free stream, nearest periodic image
    dx = x - (case.x0 + case.u_inf * t)
    dy = y - (case.y0 + case.v_inf * t)
    dx = dx - lx * np.floor(dx / lx + 0.5)
    dy = dy - ly * np.floor(dy / ly + 0.5)
    r2 = dx ** 2 + dy ** 2
    g = case.gamma
    bump = np.exp(case.phi * (1.0 - r2))
    du = -case.alpha / (2.0 * math.pi) * dy * bump
    dv = case.alpha / (2.0 * math.pi) * dx * bump
    dT = -(case.alpha ** 2) * (g - 1.0) / (16.0 * case.phi * g * math.pi ** 2) * bump ** 2
    T = case.t_inf + dT
    # dS = 0: p / rho^gamma = p_inf / rho_inf^gamma together with p = rho R T
    rho = case.rho_inf * (T / case.t_inf) ** (1.0 / (g - 1.0))
    p = rho * T
    return rho, case.u_inf + du, case.v_inf + dv, p


def conserved_from_primitive(rho, u, v, p, gamma):
    """Stack (rho, rho u, rho v, E) on axis 1, E = p/(gamma-1) + rho |u|^2 / 2 (Sec. 2)."""
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], axis=1)


def primitive_from_conserved(U, gamma):
    """(rho, u, v, p), each (Ne, Np), of a conserved state (Ne, 4, Np)."""
    rho = U[:, 0]
    u = U[:, 1] / rho
    v = U[:, 2] / rho
    p = (gamma - 1.0) * (U[:, 3] - 0.5 * rho * (u * u + v * v))
    return rho, u, v, p


def exact_state(case: VortexCase, mesh: Mesh, p: int, t: float = 0.0):
    """Conserved exact state (Ne, 4, Np) at the solution points at time t."""
    x, y = point_coordinates(mesh, Basis(p))
    return conserved_from_primitive(*exact_primitive(case, x, y, t), case.gamma)


def l2_error(s_num, s_exact, mesh: Mesh, p: int):
    """Error(s) of Sec. 5.1: sqrt(int (s_exact - s_num)^2 dV / V), the integral
    by Gauss-Legendre quadrature at the solution points of every element."""
    b = Basis(p)
    n = b.n
    total = 0.0
    volume = 0.0
    for iy in range(mesh.ny):
        for ix in range(mesh.nx):
            e = ix + mesh.nx * iy
            jac = mesh.hx[iy, ix] * mesh.hy[iy, ix] / 4.0   # |J_e| of the affine map
            volume += 4.0 * jac                             # the reference square has area 4
            for j in range(n):
                for i in range(n):
                    d = s_exact[e, i + n * j] - s_num[e, i + n * j]
                    total += b.w[i] * b.w[j] * jac * d * d
    return math.sqrt(total / volume)


def vortex_errors(U, case: VortexCase, mesh: Mesh, p: int, t: float):
    """E(rho), E(u), E(v), E(p) of the conserved state U against the exact vortex."""
    x, y = point_coordinates(mesh, Basis(p))
    exact = exact_primitive(case, x, y, t)
    num = primitive_from_conserved(U, case.gamma)
    return {name: l2_error(sn, se, mesh, p) for name, sn, se in zip(("rho", "u", "v", "p"), num, exact)}
