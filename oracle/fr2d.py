"""FR/CPR residual R(q) of the 2D Euler equations on affine quadrilaterals.

Follows Sec. 3 of the paper step by step:

1. Pointwise inviscid fluxes f, g of Sec. 2 (Eq. ns_equation in 2D) at every
   solution point, transformed to F = |J| f xi_x, G = |J| g eta_y
   (Eq. trans_detail; for an axis-aligned element of size hx x hy,
   |J| = hx*hy/4, xi_x = 2/hx, eta_y = 2/hy).
2. Solution traces q(+-1, eta_j), q(xi_i, +-1) and local-flux traces
   F^l(+-1), G^l(+-1) by evaluating the degree-p Lagrange polynomials at the
   element ends (the local flux polynomial is evaluated at the boundary).
3. Common normal flux at every face point.  The paper uses Roe (Eq. invis_com);
   the workload here uses the Rusanov (local Lax-Friedrichs) flux
   f_n = (f_n(q-) + f_n(q+))/2 - lambda/2 (q+ - q-),
   lambda = max(|u_n-| + c-, |u_n+| + c+), q- the element on the side the unit
   normal n points away from.  F^num = |J| |grad xi| f_n sign(n . grad xi)
   (Eq. norm_num_f); for vertical faces n = +x and |J||grad xi| = hy/2, for
   horizontal faces n = +y and |J||grad eta| = hx/2.
4. Divergence of the reconstructed flux at the solution points,
   dF~/dxi_i = sum_k D_ik F_k + (F^num_L - F^l_L) g_L'(xi_i) + (F^num_R - F^l_R) g_R'(xi_i),
   same along eta, and R = -(dF~/dxi + dG~/deta)/|J| (Eq. discrete_ns written
   as dq/dt = R(q), Eq. simplified_ode).

The residual is split into ``traces`` (per element) and ``local_residual``
(one element given the traces its four neighbours present to it) so that the
element-Jacobi blocks can be formed with the neighbours frozen.

Pins (tests/test_oracle_fr.py): free-stream preservation on uniform and
jittered meshes, discrete conservation, p=0 reduces to the textbook
first-order Rusanov finite-volume scheme, spatial order p+1 on a translating
density wave, hand-computed single-point flux values.
"""
from __future__ import annotations

import numpy as np

from .basis import Basis

GAMMA = 1.4


class Mesh:
    """Periodic tensor-product mesh of axis-aligned quads.

    Element ``ix + Nx*iy`` spans [x_edges[ix], x_edges[ix+1]] x
    [y_edges[iy], y_edges[iy+1]].
    """

    def __init__(self, x_edges, y_edges, wall_y: bool = False):
        self.wall_y = bool(wall_y)   # isothermal no-slip walls at the y ends (viscous residual)
        self.x_edges = np.asarray(x_edges, dtype=np.float64)
        self.y_edges = np.asarray(y_edges, dtype=np.float64)
        self.nx = len(self.x_edges) - 1
        self.ny = len(self.y_edges) - 1
        if self.nx < 2 or self.ny < 2:
            raise ValueError("a periodic mesh needs at least 2 elements per direction")
        self.ne = self.nx * self.ny
        hx = np.diff(self.x_edges)
        hy = np.diff(self.y_edges)
        # per-element sizes, shape (ny, nx)
        self.hx = np.broadcast_to(hx[None, :], (self.ny, self.nx)).copy()
        self.hy = np.broadcast_to(hy[:, None], (self.ny, self.nx)).copy()


# ---------------------------------------------------------------- physics --

def pressure(q, gamma=GAMMA):
    """p = (gamma-1) (E - rho |u|^2 / 2); q has the variable on axis 0."""
    rho, ru, rv, E = q
    return (gamma - 1.0) * (E - 0.5 * (ru * ru + rv * rv) / rho)


def flux_x(q, gamma=GAMMA):
    """Inviscid flux f = F_inv,1 of Sec. 2 in 2D."""
    rho, ru, rv, E = q
    u = ru / rho
    p = pressure(q, gamma)
    return np.stack([ru, ru * u + p, rv * u, u * (E + p)])


def flux_y(q, gamma=GAMMA):
    """Inviscid flux g = F_inv,2 of Sec. 2 in 2D."""
    rho, ru, rv, E = q
    v = rv / rho
    p = pressure(q, gamma)
    return np.stack([rv, ru * v, rv * v + p, v * (E + p)])


def rusanov(qm, qp, direction, gamma=GAMMA):
    """Rusanov common flux along +x (direction 0) or +y (direction 1)."""
    flux = flux_x if direction == 0 else flux_y
    fm, fp = flux(qm, gamma), flux(qp, gamma)
    unm = qm[1 + direction] / qm[0]
    unp = qp[1 + direction] / qp[0]
    cm = np.sqrt(gamma * pressure(qm, gamma) / qm[0])
    cp = np.sqrt(gamma * pressure(qp, gamma) / qp[0])
    lam = np.maximum(np.abs(unm) + cm, np.abs(unp) + cp)
    return 0.5 * (fm + fp) - 0.5 * lam * (qp - qm)


def roe(qm, qp, direction, gamma=GAMMA):
    """Roe's approximate Riemann flux (the paper's common flux, Sec. 3) along
    +x (direction 0) or +y (direction 1), without entropy fix:
    F = (f(qm) + f(qp))/2 - sum_k |lambda_k| alpha_k r_k / 2 with the
    eigen-decomposition of the flux Jacobian at the Roe average (density
    weights sqrt(rho): velocity and total enthalpy H = (E + p)/rho averaged,
    a^2 = (gamma - 1)(H - |u|^2/2)).  Waves: u_n - a, the entropy and the
    shear wave (both u_n), u_n + a."""
    flux = flux_x if direction == 0 else flux_y
    fm, fp = flux(qm, gamma), flux(qp, gamma)
    rm, rp = qm[0], qp[0]
    um, vm, up, vp = qm[1] / rm, qm[2] / rm, qp[1] / rp, qp[2] / rp
    pm, pp = pressure(qm, gamma), pressure(qp, gamma)
    Hm, Hp = (qm[3] + pm) / rm, (qp[3] + pp) / rp
    sm, sp = np.sqrt(rm), np.sqrt(rp)
    w = 1.0 / (sm + sp)
    u = (sm * um + sp * up) * w
    v = (sm * vm + sp * vp) * w
    H = (sm * Hm + sp * Hp) * w
    rho = sm * sp
    a2 = (gamma - 1.0) * (H - 0.5 * (u * u + v * v))
    a = np.sqrt(a2)
    un, dun = (u, up - um) if direction == 0 else (v, vp - vm)
    dut = (vp - vm) if direction == 0 else (up - um)
    drho, dp = rp - rm, pp - pm
    al1 = (dp - rho * a * dun) / (2.0 * a2)
    al2 = drho - dp / a2
    al3 = rho * dut
    al4 = (dp + rho * a * dun) / (2.0 * a2)
    l1, l2, l4 = np.abs(un - a), np.abs(un), np.abs(un + a)
    one = np.ones_like(u)
    zero = np.zeros_like(u)
    if direction == 0:
        r1 = np.stack([one, u - a, v, H - u * a])
        r3 = np.stack([zero, zero, one, v])
        r4 = np.stack([one, u + a, v, H + u * a])
    else:
        r1 = np.stack([one, u, v - a, H - v * a])
        r3 = np.stack([zero, one, zero, u])
        r4 = np.stack([one, u, v + a, H + v * a])
    r2 = np.stack([one, u, v, 0.5 * (u * u + v * v)])
    diss = l1 * al1 * r1 + l2 * al2 * r2 + l2 * al3 * r3 + l4 * al4 * r4
    return 0.5 * (fm + fp) - 0.5 * diss


def common_flux(qm, qp, direction, gamma=GAMMA, riemann="rusanov"):
    if riemann == "roe":
        return roe(qm, qp, direction, gamma)
    return rusanov(qm, qp, direction, gamma)


# ----------------------------------------------------------- FR residual --

def as_grid(U, mesh: Mesh, p: int):
    """(Ne, 4, Np) -> (4, ny, nx, p+1 [j], p+1 [i])."""
    n = p + 1
    return np.asarray(U, dtype=np.float64).reshape(mesh.ny, mesh.nx, 4, n, n).transpose(2, 0, 1, 3, 4)


def from_grid(Q, mesh: Mesh, p: int):
    n = p + 1
    return np.ascontiguousarray(Q.transpose(1, 2, 0, 3, 4).reshape(mesh.ne, 4, n * n))


def traces(Q, b: Basis):
    """Solution traces of each element on its four faces.

    Q: (4, ..., p+1 [j], p+1 [i]).  Returns qW, qE (shape (4, ..., p+1) over j)
    at xi = -1, +1 and qS, qN (over i) at eta = -1, +1.
    """
    qW = np.einsum("...jk,k->...j", Q, b.lm)
    qE = np.einsum("...jk,k->...j", Q, b.lp)
    qS = np.einsum("...kj,k->...j", Q, b.lm)
    qN = np.einsum("...kj,k->...j", Q, b.lp)
    return qW, qE, qS, qN


def local_residual(Q, hx, hy, nW, nE, nS, nN, b: Basis, gamma=GAMMA, riemann="rusanov"):
    """R on elements given their own state Q (4, E..., n, n) and the traces the
    neighbours present on each face (nW: the west neighbour's east trace,
    etc., each (4, E..., n)).  hx, hy broadcast against E...."""
    hx = np.asarray(hx)[None, ..., None, None]
    hy = np.asarray(hy)[None, ..., None, None]
    # step 1: transformed fluxes at solution points
    F = 0.5 * hy * flux_x(Q, gamma)
    G = 0.5 * hx * flux_y(Q, gamma)
    # step 2: own traces and local-flux traces
    qW, qE, qS, qN = traces(Q, b)
    FlW = np.einsum("...jk,k->...j", F, b.lm)
    FlE = np.einsum("...jk,k->...j", F, b.lp)
    GlS = np.einsum("...kj,k->...j", G, b.lm)
    GlN = np.einsum("...kj,k->...j", G, b.lp)
    # step 3: common fluxes; q- is the element the +x / +y normal leaves
    hy_f = hy[..., 0]
    hx_f = hx[..., 0]
    FnW = 0.5 * hy_f * common_flux(nW, qW, 0, gamma, riemann)
    FnE = 0.5 * hy_f * common_flux(qE, nE, 0, gamma, riemann)
    GnS = 0.5 * hx_f * common_flux(nS, qS, 1, gamma, riemann)
    GnN = 0.5 * hx_f * common_flux(qN, nN, 1, gamma, riemann)
    # step 4: divergence of the corrected flux
    dF = (np.einsum("ik,...jk->...ji", b.D, F)
          + (FnW - FlW)[..., :, None] * b.dgL[None, :]
          + (FnE - FlE)[..., :, None] * b.dgR[None, :])
    dG = (np.einsum("jk,...ki->...ji", b.D, G)
          + (GnS - GlS)[..., None, :] * b.dgL[:, None]
          + (GnN - GlN)[..., None, :] * b.dgR[:, None])
    detJ = 0.25 * hx * hy
    return -(dF + dG) / detJ


def neighbour_traces(Q, b: Basis):
    """Traces each element sees from its periodic neighbours."""
    qW, qE, qS, qN = traces(Q, b)            # (4, ny, nx, n)
    nW = np.roll(qE, 1, axis=2)              # east trace of element ix-1
    nE = np.roll(qW, -1, axis=2)             # west trace of element ix+1
    nS = np.roll(qN, 1, axis=1)              # north trace of element iy-1
    nN = np.roll(qS, -1, axis=1)             # south trace of element iy+1
    return nW, nE, nS, nN


def residual(U, mesh: Mesh, p: int, basis: Basis | None = None, gamma=GAMMA, riemann="rusanov"):
    """R(q) for the whole periodic mesh; U and the result are (Ne, 4, Np)."""
    b = basis or Basis(p)
    Q = as_grid(U, mesh, p)
    nW, nE, nS, nN = neighbour_traces(Q, b)
    R = local_residual(Q, mesh.hx, mesh.hy, nW, nE, nS, nN, b, gamma, riemann)
    return from_grid(R, mesh, p)
