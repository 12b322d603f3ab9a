"""Viscous (Navier-Stokes) FR residual with BR2 common gradients, Sec. 2-3.

Builds on the inviscid residual of ``fr2d``:

* viscous flux of Sec. 2 in 2D: tau_xx = mu (2 u_x - 2/3 (u_x + v_y)),
  tau_yy = mu (2 v_y - 2/3 (u_x + v_y)), tau_xy = mu (u_y + v_x), heat flux
  K = -kappa grad T with kappa = mu Cp / Pr, Cp = gamma R / (gamma - 1),
  T = p / (rho R);  f_vis = (0, tau_xx, tau_xy, u tau_xx + v tau_xy - K_x),
  g_vis = (0, tau_xy, tau_yy, u tau_xy + v tau_yy - K_y);
* gradients of the conserved variables, converted to grad u, grad v,
  grad T by the chain rule (the paper averages "primitive variables" but its
  Eq. com_q is written in q: conserved variables are taken);
* common solution q_com = (q- + q+)/2 (Eq. com_q);
* corrected gradient at the solution points: the FR derivative of q with
  the correction (q_com - q_face) g'(xi) along each direction;
* BR2 common gradient (Eq. com_grad_q): (grad q- + r- + grad q+ + r+)/2 with
  grad q the face trace of the element's own (uncorrected) polynomial
  gradient and r = gamma_BR2 (q_com - q_face) n, gamma_BR2 = |grad xi|
  g'(+-1) sign(n . grad xi), g'(+-1) = +-(P+1)(P+2)/2 (the text writes
  "g(+-1)"; the derivative is meant);
* the total flux F = F_inv - F_vis is corrected and differentiated as in
  ``fr2d``; the common viscous flux is f_vis(q_com, grad q_com) . n;
* isothermal no-slip walls at the y ends when ``mesh.wall_y``: boundary
  state q_b = (rho_int, 0, 0, rho_int R T_w / (gamma - 1)); inviscid wall
  flux g(q_b); q_com = q_b; grad q_com = grad q_int + r_int; the paper does
  not give its wall treatment, this is the reading used on both sides;
* a body force per unit mass (gx, 0): source (0, rho gx, 0, rho u gx).

Pins (tests/test_oracle_ns.py): uniform state on a periodic mesh gives
R = 0; discrete conservation on a periodic mesh; Poiseuille flow between
walls at p = 4 gives R_rho = R_rhou = R_rhov = 0 and R_E = mu (du/dy)^2
pointwise (the closed form of viscous heating); mu = 0 reduces to the
inviscid residual.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .basis import Basis
from .fr2d import as_grid, flux_x, flux_y, from_grid, pressure, rusanov, traces


@dataclass(frozen=True)
class Viscous:
    mu: float = 0.0
    prandtl: float = 0.72
    gas_r: float = 1.0
    gamma: float = 1.4
    gx: float = 0.0          # body force per unit mass along x
    t_wall: float = 1.0

    @property
    def kappa(self):
        cp = self.gamma * self.gas_r / (self.gamma - 1.0)
        return self.mu * cp / self.prandtl


def primitive_gradients(q, qx, qy, ph: Viscous):
    """(u, v, T) and their x/y derivatives from q and the gradients of q."""
    rho, ru, rv, E = q
    u = ru / rho
    v = rv / rho
    T = (ph.gamma - 1.0) / ph.gas_r * (E / rho - 0.5 * (u * u + v * v))
    out = []
    for d in (qx, qy):
        drho, dru, drv, dE = d
        du = (dru - u * drho) / rho
        dv = (drv - v * drho) / rho
        dT = (ph.gamma - 1.0) / ph.gas_r * ((dE - E / rho * drho) / rho - (u * du + v * dv))
        out.append((du, dv, dT))
    return (u, v, T), out[0], out[1]


def viscous_fluxes(q, qx, qy, ph: Viscous):
    """f_vis and g_vis of Sec. 2 in 2D (variable on axis 0)."""
    (u, v, T), (ux, vx, Tx), (uy, vy, Ty) = primitive_gradients(q, qx, qy, ph)
    div = ux + vy
    txx = ph.mu * (2 * ux - 2.0 / 3.0 * div)
    tyy = ph.mu * (2 * vy - 2.0 / 3.0 * div)
    txy = ph.mu * (uy + vx)
    zero = np.zeros_like(u)
    fv = np.stack([zero, txx, txy, u * txx + v * txy + ph.kappa * Tx])
    gv = np.stack([zero, txy, tyy, u * txy + v * tyy + ph.kappa * Ty])
    return fv, gv


def wall_state(q, ph: Viscous):
    """Isothermal no-slip boundary state from the interior trace."""
    rho = q[0]
    zero = np.zeros_like(rho)
    return np.stack([rho, zero, zero, rho * ph.gas_r * ph.t_wall / (ph.gamma - 1.0)])


def ns_residual(U, mesh, p, ph: Viscous, basis: Basis | None = None):
    """R(q) for the 2D Navier-Stokes equations; U and R are (Ne, 4, Np)."""
    b = basis or Basis(p)
    n = p + 1
    g = ph.gamma
    Q = as_grid(U, mesh, p)                                  # (4, ny, nx, n[j], n[i])
    hx = mesh.hx[None, :, :, None, None]
    hy = mesh.hy[None, :, :, None, None]
    wall = getattr(mesh, "wall_y", False)
    cbr2 = (p + 1) * (p + 2) / 2.0
    # ---- traces and their neighbours
    qW, qE, qS, qN = traces(Q, b)                             # (4, ny, nx, n)
    nW = np.roll(qE, 1, axis=2)
    nE = np.roll(qW, -1, axis=2)
    nS = np.roll(qN, 1, axis=1)
    nN = np.roll(qS, -1, axis=1)
    # ---- common solution (walls: boundary state)
    cW, cE = 0.5 * (qW + nW), 0.5 * (qE + nE)
    cS, cN = 0.5 * (qS + nS), 0.5 * (qN + nN)
    if wall:
        cS[:, 0] = wall_state(qS[:, 0], ph)
        cN[:, -1] = wall_state(qN[:, -1], ph)
    # ---- own (uncorrected) polynomial gradient at points, and corrected gradient
    dxi = np.einsum("ik,...jk->...ji", b.D, Q)               # d/dxi along rows
    deta = np.einsum("jk,...ki->...ji", b.D, Q)              # d/deta along columns
    sx = 2.0 / hx
    sy = 2.0 / hy
    gx_loc = sx * dxi
    gy_loc = sy * deta
    gx_cor = sx * (dxi + (cW - qW)[..., :, None] * b.dgL[None, :] + (cE - qE)[..., :, None] * b.dgR[None, :])
    gy_cor = sy * (deta + (cS - qS)[..., None, :] * b.dgL[:, None] + (cN - qN)[..., None, :] * b.dgR[:, None])
    # ---- face traces of the own gradients
    def tr_x(A):  # traces of a point field on W/E faces (over j)
        return np.einsum("...jk,k->...j", A, b.lm), np.einsum("...jk,k->...j", A, b.lp)

    def tr_y(A):  # on S/N faces (over i)
        return np.einsum("...kj,k->...j", A, b.lm), np.einsum("...kj,k->...j", A, b.lp)
    gxW, gxE = tr_x(gx_loc)
    gyW, gyE = tr_x(gy_loc)
    gxS, gxN = tr_y(gx_loc)
    gyS, gyN = tr_y(gy_loc)
    sx_f = sx[..., 0]
    sy_f = sy[..., 0]
    # BR2 liftings r = |grad xi| g'(+-1) (q_com - q_face) n with n = +x / +y
    rW = -sx_f * cbr2 * (cW - qW)     # x-component on the west face
    rE = sx_f * cbr2 * (cE - qE)
    rS = -sy_f * cbr2 * (cS - qS)     # y-component on the south face
    rN = sy_f * cbr2 * (cN - qN)
    # neighbour quantities across each face
    def nbx(A, shift):
        return np.roll(A, shift, axis=2)

    def nby(A, shift):
        return np.roll(A, shift, axis=1)
    # x-faces: west face of (iy, ix) is shared with the east face of (iy, ix-1)
    cgx_W = 0.5 * (gxW + rW + nbx(gxE + rE, 1))
    cgy_W = 0.5 * (gyW + nbx(gyE, 1))
    cgx_E = 0.5 * (gxE + rE + nbx(gxW + rW, -1))
    cgy_E = 0.5 * (gyE + nbx(gyW, -1))
    cgx_S = 0.5 * (gxS + nby(gxN, 1))
    cgy_S = 0.5 * (gyS + rS + nby(gyN + rN, 1))
    cgx_N = 0.5 * (gxN + nby(gxS, -1))
    cgy_N = 0.5 * (gyN + rN + nby(gyS + rS, -1))
    if wall:
        cgx_S[:, 0] = gxS[:, 0]
        cgy_S[:, 0] = gyS[:, 0] + rS[:, 0]
        cgx_N[:, -1] = gxN[:, -1]
        cgy_N[:, -1] = gyN[:, -1] + rN[:, -1]
    # ---- pointwise total fluxes F = (hy/2)(f - f_vis), G = (hx/2)(g - g_vis)
    fv, gv = viscous_fluxes(Q, gx_cor, gy_cor, ph)
    F = 0.5 * hy * (flux_x(Q, g) - fv)
    G = 0.5 * hx * (flux_y(Q, g) - gv)
    FlW = np.einsum("...jk,k->...j", F, b.lm)
    FlE = np.einsum("...jk,k->...j", F, b.lp)
    GlS = np.einsum("...kj,k->...j", G, b.lm)
    GlN = np.einsum("...kj,k->...j", G, b.lp)
    # ---- common total fluxes
    fvW, _ = viscous_fluxes(cW, cgx_W, cgy_W, ph)
    fvE, _ = viscous_fluxes(cE, cgx_E, cgy_E, ph)
    _, gvS = viscous_fluxes(cS, cgx_S, cgy_S, ph)
    _, gvN = viscous_fluxes(cN, cgx_N, cgy_N, ph)
    fiW = rusanov(nW, qW, 0, g)
    fiE = rusanov(qE, nE, 0, g)
    giS = rusanov(nS, qS, 1, g)
    giN = rusanov(qN, nN, 1, g)
    if wall:
        giS[:, 0] = flux_y(cS[:, 0], g)
        giN[:, -1] = flux_y(cN[:, -1], g)
    hy_f = hy[..., 0]
    hx_f = hx[..., 0]
    FnW = 0.5 * hy_f * (fiW - fvW)
    FnE = 0.5 * hy_f * (fiE - fvE)
    GnS = 0.5 * hx_f * (giS - gvS)
    GnN = 0.5 * hx_f * (giN - gvN)
    dF = (np.einsum("ik,...jk->...ji", b.D, F)
          + (FnW - FlW)[..., :, None] * b.dgL[None, :]
          + (FnE - FlE)[..., :, None] * b.dgR[None, :])
    dG = (np.einsum("jk,...ki->...ji", b.D, G)
          + (GnS - GlS)[..., None, :] * b.dgL[:, None]
          + (GnN - GlN)[..., None, :] * b.dgR[:, None])
    R = -(dF + dG) / (0.25 * hx * hy)
    if ph.gx != 0.0:
        R[1] = R[1] + Q[0] * ph.gx
        R[3] = R[3] + Q[1] * ph.gx
    return from_grid(R, mesh, p)


def ns_element_jacobians(U, mesh, p, ph: Viscous, elements=None, eps_rel=1e-7, basis=None):
    """J_ee = dR_e/dq_e (all other elements' DOFs held fixed) by forward
    differences with eps_j = eps_rel (1 + |q_j|): the diagonal blocks of the
    global Jacobian.  Elements of one checkerboard colour are perturbed
    together (their residuals do not see each other: R_e depends only on
    the element and its four face neighbours), which gives exactly the
    per-element quotients; this needs an even nx (periodic x)."""
    b = basis or Basis(p)
    if mesh.nx % 2 or (mesh.ny % 2 and not mesh.wall_y):
        raise ValueError("checkerboard colouring needs even nx (and even ny unless walls)")
    nb = 4 * (p + 1) ** 2
    U = np.asarray(U, dtype=np.float64)
    R0 = ns_residual(U, mesh, p, ph, b)
    iy, ix = np.divmod(np.arange(mesh.ne), mesh.nx)
    colour = (ix + iy) % 2
    J = np.zeros((mesh.ne, nb, nb))
    flat = U.reshape(mesh.ne, nb)
    for c in (0, 1):
        sel = np.nonzero(colour == c)[0]
        for col in range(nb):
            Up = flat.copy()
            eps = eps_rel * (1.0 + np.abs(flat[sel, col]))
            Up[sel, col] += eps
            Rp = ns_residual(Up.reshape(U.shape), mesh, p, ph, b).reshape(mesh.ne, nb)
            J[sel, :, col] = (Rp[sel] - R0.reshape(mesh.ne, nb)[sel]) / eps[:, None]
    if elements is not None:
        return J[np.asarray(elements)]
    return J
