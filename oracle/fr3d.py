"""3D Navier-Stokes FR residual on periodic axis-aligned hexahedra, and the
Taylor-Green kinetic-energy dissipation rate (Sec. 3 and Sec. 5, Taylor-Green
vortex).  Test infrastructure: only tests, the smoke check and the benchmark's
CPU baseline use it.

The scheme is the tensor-product extension of ``fr2d`` / ``ns2d`` to three
reference directions (xi, eta, zeta) on an element of size hx x hy x hz:

* state q = (rho, rho u, rho v, rho w, E), p = (gamma - 1)(E - rho |v|^2 / 2);
* inviscid flux along direction d:  (rho v_d, rho u v_d + p delta_d1,
  rho v v_d + p delta_d2, rho w v_d + p delta_d3, v_d (E + p))  (Sec. 2);
* viscous flux along d:  (0, tau_d1, tau_d2, tau_d3, sum_j v_j tau_dj + kappa dT/dx_d)
  with tau = mu (grad v + grad v^T - 2/3 (div v) I), kappa = mu Cp / Pr,
  T = p / (rho R), R = 1; gradients of the conserved variables are turned
  into grad v and grad T by the chain rule;
* common solution q_com = (q- + q+)/2 (Eq. com_q), BR2 common gradient
  (Eq. com_grad_q) with the lifting r = |grad xi| g'(+-1) (q_com - q_face) n,
  g'(+-1) = +-(P+1)(P+2)/2, corrected gradient at the solution points
  grad q + sum over the faces of (q_com - q_face) grad g;
* Rusanov common inviscid flux, common viscous flux f_vis(q_com, grad q_com) . n;
* corrected divergence of the total flux F - F_vis along each direction as in
  Sec. 3: sum_k D_ik F_k + (F^num_L - F^l_L) g_L'(xi_i) + (F^num_R - F^l_R) g_R'(xi_i),
  with the local flux polynomial evaluated at the element ends.  On an
  axis-aligned hexahedron |J| = hx hy hz / 8 and the transformed flux along
  xi is (hy hz / 4) f (Eq. trans_detail), so R = -(2/hx dF/dxi + 2/hy dG/deta
  + 2/hz dH/dzeta) with the physical fluxes: the same numbers, written
  without the metric factors that cancel.

Layout: U[Ne][5][Np], Np = (p+1)^3, point index i + n j + n^2 k (i along x),
element index ix + nx (iy + ny iz).

Dissipation rate (Sec. 5, Taylor-Green vortex): eps = eps1 + eps2 + eps3 with
eps1 = 2 mu / rho0 <S^d : S^d>, eps2 = mu_v / rho0 <(div v)^2> = 0 (mu_v = 0),
eps3 = -1 / rho0 <p div v>, <.> the volume average.  The paper does not say
how the velocity gradient is evaluated; here the velocity at the solution
points is differentiated as the element's degree-p interpolant (no
correction), and <.> is Gauss-Legendre quadrature at the solution points.

Pins (tests/test_oracle_fr3d.py): free stream is preserved on uniform and
stretched meshes; discrete conservation; a state that does not depend on z
with w = 0 gives the 2D Navier-Stokes residual and R_rhow = 0; a cyclic
permutation of the axes permutes the residual; FD Jv and element blocks
against a brute-force Jacobian; the dissipation rate and kinetic energy of
the Taylor-Green initial field against their closed forms (sympy).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .basis import Basis


class Mesh3D:
    """Periodic tensor-product mesh of axis-aligned hexahedra."""

    def __init__(self, x_edges, y_edges, z_edges):
        self.x_edges = np.asarray(x_edges, dtype=np.float64)
        self.y_edges = np.asarray(y_edges, dtype=np.float64)
        self.z_edges = np.asarray(z_edges, dtype=np.float64)
        self.nx = len(self.x_edges) - 1
        self.ny = len(self.y_edges) - 1
        self.nz = len(self.z_edges) - 1
        if min(self.nx, self.ny, self.nz) < 2:
            raise ValueError("a periodic mesh needs at least 2 elements per direction")
        self.ne = self.nx * self.ny * self.nz
        self.hx = np.diff(self.x_edges)
        self.hy = np.diff(self.y_edges)
        self.hz = np.diff(self.z_edges)

    @property
    def volume(self):
        return self.hx.sum() * self.hy.sum() * self.hz.sum()


@dataclass(frozen=True)
class Gas3D:
    mu: float = 0.0
    prandtl: float = 0.71
    gamma: float = 1.4
    gas_r: float = 1.0

    @property
    def kappa(self):
        cp = self.gamma * self.gas_r / (self.gamma - 1.0)
        return self.mu * cp / self.prandtl


def as_grid(U, mesh: Mesh3D, p):
    """(Ne, 5, Np) -> (5, nz, ny, nx, n[k], n[j], n[i])."""
    n = p + 1
    return np.asarray(U, dtype=np.float64).reshape(mesh.nz, mesh.ny, mesh.nx, 5, n, n, n).transpose(3, 0, 1, 2, 4, 5, 6)


def from_grid(Q, mesh: Mesh3D, p):
    n = p + 1
    return Q.transpose(1, 2, 3, 0, 4, 5, 6).reshape(mesh.ne, 5, n ** 3)


def pressure(q, gamma):
    rho, ru, rv, rw, E = q
    return (gamma - 1.0) * (E - 0.5 * (ru * ru + rv * rv + rw * rw) / rho)


def inviscid_flux(q, d, gamma):
    """Inviscid flux along direction d (0: x, 1: y, 2: z), variable on axis 0."""
    rho = q[0]
    vd = q[1 + d] / rho
    p = pressure(q, gamma)
    f = [q[0] * vd, q[1] * vd, q[2] * vd, q[3] * vd, vd * (q[4] + p)]
    f[1 + d] = f[1 + d] + p
    return np.stack(f)


def rusanov(qm, qp, d, gamma):
    """Rusanov common flux along +x_d from the (-) and (+) states."""
    fm, fp = inviscid_flux(qm, d, gamma), inviscid_flux(qp, d, gamma)
    cm = np.sqrt(gamma * pressure(qm, gamma) / qm[0])
    cp = np.sqrt(gamma * pressure(qp, gamma) / qp[0])
    lam = np.maximum(np.abs(qm[1 + d] / qm[0]) + cm, np.abs(qp[1 + d] / qp[0]) + cp)
    return 0.5 * (fm + fp) - 0.5 * lam * (qp - qm)


def viscous_flux(q, grads, d, gas: Gas3D):
    """Viscous flux along d from q and its three gradients grads[0..2]."""
    rho = q[0]
    vel = [q[1] / rho, q[2] / rho, q[3] / rho]
    e = q[4] / rho
    # derivative of (u, v, w) and of T along each direction c
    dvel = [[(grads[c][1 + m] - vel[m] * grads[c][0]) / rho for m in range(3)] for c in range(3)]
    dT = [(gas.gamma - 1.0) / gas.gas_r * ((grads[c][4] - e * grads[c][0]) / rho
                                          - sum(vel[m] * dvel[c][m] for m in range(3))) for c in range(3)]
    div = dvel[0][0] + dvel[1][1] + dvel[2][2]
    # tau_dm = mu (d v_m / d x_d + d v_d / d x_m) - 2/3 mu div delta_dm
    tau = [gas.mu * (dvel[d][m] + dvel[m][d]) for m in range(3)]
    tau[d] = tau[d] - 2.0 / 3.0 * gas.mu * div
    energy = sum(vel[m] * tau[m] for m in range(3)) + gas.kappa * dT[d]
    return np.stack([np.zeros_like(rho), tau[0], tau[1], tau[2], energy])


def _deriv(A, D, axis):
    """Apply the 1D derivative matrix along one of the last three axes
    (axis -1: xi, -2: eta, -3: zeta)."""
    return np.moveaxis(np.tensordot(np.moveaxis(A, axis, -1), D, axes=([-1], [1])), -1, axis)


def _trace(A, c, axis):
    """Evaluate along one of the last three axes with coefficients c (the
    Lagrange values at an element end); that axis is removed."""
    return np.tensordot(np.moveaxis(A, axis, -1), c, axes=([-1], [0]))


_AX = (-1, -2, -3)          # point axis of reference direction d
_EL = (3, 2, 1)             # element axis of direction d in the grid form


def residual3d(U, mesh: Mesh3D, p, gas: Gas3D, basis: Basis | None = None):
    """R(q) of the 3D Navier-Stokes equations (Euler when mu = 0)."""
    b = basis or Basis(p)
    g = gas.gamma
    Q = as_grid(U, mesh, p)
    cbr2 = (p + 1) * (p + 2) / 2.0
    hs = [mesh.hx[None, None, None, :, None, None, None],
          mesh.hy[None, None, :, None, None, None, None],
          mesh.hz[None, :, None, None, None, None, None]]
    s = [2.0 / h for h in hs]                                 # |grad xi_d|
    sf = [x[..., 0] for x in s]                               # same, on a face array
    # traces of q on the low (L) and high (R) face of every direction
    qL = [_trace(Q, b.lm, _AX[d]) for d in range(3)]
    qR = [_trace(Q, b.lp, _AX[d]) for d in range(3)]
    # neighbour traces: the low face of an element meets the high face of its low neighbour
    nL = [np.roll(qR[d], 1, axis=_EL[d]) for d in range(3)]
    nR = [np.roll(qL[d], -1, axis=_EL[d]) for d in range(3)]
    cL = [0.5 * (qL[d] + nL[d]) for d in range(3)]
    cR = [0.5 * (qR[d] + nR[d]) for d in range(3)]

    def expand(F, d):   # a face array back onto the points (insert the removed axis)
        return np.expand_dims(F, _AX[d])

    def along(c, d):    # 1D coefficients c broadcast along the point axis of d
        shape = [1, 1, 1]
        shape[2 - d] = len(c)
        return np.asarray(c).reshape(shape)

    # own (uncorrected) physical gradient and the FR-corrected gradient
    g_loc = [s[d] * _deriv(Q, b.D, _AX[d]) for d in range(3)]
    g_cor = [s[d] * (_deriv(Q, b.D, _AX[d])
                     + expand(cL[d] - qL[d], d) * along(b.dgL, d)
                     + expand(cR[d] - qR[d], d) * along(b.dgR, d)) for d in range(3)]
    # BR2: own gradient traces plus the lifting in the face-normal component
    cgL, cgR = [], []
    for d in range(3):
        oL = [_trace(g_loc[c], b.lm, _AX[d]) for c in range(3)]
        oR = [_trace(g_loc[c], b.lp, _AX[d]) for c in range(3)]
        rL = -sf[d] * cbr2 * (cL[d] - qL[d])    # normal +x_d: the low face has n . grad xi_d < 0
        rR = sf[d] * cbr2 * (cR[d] - qR[d])
        oL[d] = oL[d] + rL
        oR[d] = oR[d] + rR
        cgL.append([0.5 * (oL[c] + np.roll(oR[c], 1, axis=_EL[d])) for c in range(3)])
        cgR.append([0.5 * (oR[c] + np.roll(oL[c], -1, axis=_EL[d])) for c in range(3)])
    # corrected divergence of the total flux along each direction
    R = np.zeros_like(Q)
    for d in range(3):
        F = inviscid_flux(Q, d, g) - viscous_flux(Q, g_cor, d, gas)
        FlL = _trace(F, b.lm, _AX[d])
        FlR = _trace(F, b.lp, _AX[d])
        FnL = rusanov(nL[d], qL[d], d, g) - viscous_flux(cL[d], cgL[d], d, gas)
        FnR = rusanov(qR[d], nR[d], d, g) - viscous_flux(cR[d], cgR[d], d, gas)
        dF = (_deriv(F, b.D, _AX[d]) + expand(FnL - FlL, d) * along(b.dgL, d)
              + expand(FnR - FlR, d) * along(b.dgR, d))
        R = R - s[d] * dF
    return from_grid(R, mesh, p)


class Problem3D:
    """What the oracle steppers need: R(q), the DOF count and the element
    blocks of the 3D residual."""

    def __init__(self, mesh: Mesh3D, p: int, gas: Gas3D = Gas3D()):
        self.mesh = mesh
        self.p = p
        self.np = (p + 1) ** 3
        self.nb = 5 * self.np
        self.basis = Basis(p)
        self.gas = gas
        self.gamma = gas.gamma
        self.viscous = None
        self.n_residuals = 0

    @property
    def ndof(self):
        return self.mesh.ne * self.nb

    def R(self, U):
        self.n_residuals += 1
        return residual3d(U, self.mesh, self.p, self.gas, self.basis)

    def element_jacobians(self, U, elements=None, eps_rel=1e-7):
        """J_ee = dR_e/dq_e (all other elements' DOFs held fixed) by forward
        differences with eps_j = eps_rel (1 + |q_j|).  R_e depends only on
        the element and its six face neighbours, so the elements of one
        colour of a 3D checkerboard are perturbed together (even nx, ny, nz)."""
        m = self.mesh
        if m.nx % 2 or m.ny % 2 or m.nz % 2:
            raise ValueError("checkerboard colouring needs even nx, ny and nz")
        nb = self.nb
        U = np.asarray(U, dtype=np.float64)
        flat = U.reshape(m.ne, nb)
        R0 = self.R(U).reshape(m.ne, nb)
        e = np.arange(m.ne)
        ix, iy, iz = e % m.nx, (e // m.nx) % m.ny, e // (m.nx * m.ny)
        colour = (ix + iy + iz) % 2
        J = np.zeros((m.ne, nb, nb))
        for c in (0, 1):
            sel = np.nonzero(colour == c)[0]
            for col in range(nb):
                Up = flat.copy()
                eps = eps_rel * (1.0 + np.abs(flat[sel, col]))
                Up[sel, col] += eps
                Rp = self.R(Up.reshape(U.shape)).reshape(m.ne, nb)
                J[sel, :, col] = (Rp[sel] - R0[sel]) / eps[:, None]
        return J if elements is None else J[np.asarray(elements)]


def dissipation_rate(U, mesh: Mesh3D, p, gas: Gas3D, rho0=1.0, basis: Basis | None = None):
    """(eps1, eps3, kinetic energy) of the Taylor-Green study, Sec. 5:
    eps1 = 2 mu/rho0 <S^d:S^d>, eps3 = -<p div v>/rho0, k = <rho |v|^2/2>/rho0."""
    b = basis or Basis(p)
    Q = as_grid(U, mesh, p)
    rho = Q[0]
    vel = [Q[1 + m] / rho for m in range(3)]
    pr = pressure(Q, gas.gamma)
    hs = [mesh.hx[None, None, :, None, None, None],
          mesh.hy[None, :, None, None, None, None],
          mesh.hz[:, None, None, None, None, None]]
    # G[m][c] = d v_m / d x_c from the element's interpolant of v_m
    G = [[(2.0 / hs[c]) * _deriv(vel[m], b.D, _AX[c]) for c in range(3)] for m in range(3)]
    div = G[0][0] + G[1][1] + G[2][2]
    SdSd = np.zeros_like(rho)
    for m in range(3):
        for c in range(3):
            S = 0.5 * (G[m][c] + G[c][m]) - (div / 3.0 if m == c else 0.0)
            SdSd = SdSd + S * S
    w3 = b.w[:, None, None] * b.w[None, :, None] * b.w[None, None, :]
    vol = (hs[0] * hs[1] * hs[2]) / 8.0

    def mean(f):
        return float(np.sum(f * w3 * vol) / mesh.volume)
    ke = 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    return 2.0 * gas.mu / rho0 * mean(SdSd), -mean(pr * div) / rho0, mean(ke) / rho0
