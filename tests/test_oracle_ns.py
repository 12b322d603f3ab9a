"""Pins of the viscous BR2 residual (oracle/ns2d.py)."""
import numpy as np
import pytest

import synthetic as S
from oracle.basis import Basis
from oracle.fr2d import Mesh, flux_x, flux_y, residual, rusanov
from oracle.ns2d import Viscous, ns_residual, viscous_fluxes


def test_zero_viscosity_is_the_inviscid_residual():
    p = 3
    xe, ye = S.stretched_mesh(5, 4, seed=1)
    X, Y = S.point_coords(xe, ye, p)
    U = S.smooth_random_state(X, Y, seed=3, amp=0.1)
    m = Mesh(xe, ye)
    assert np.array_equal(ns_residual(U, m, p, Viscous(mu=0.0)), residual(U, m, p))


@pytest.mark.parametrize("p", [2, 3, 4])
def test_uniform_state_periodic(p):
    xe, ye = S.stretched_mesh(5, 4, seed=p)
    X, _ = S.point_coords(xe, ye, p)
    one = np.ones_like(X)
    U = S.conserved(1.2 * one, 0.3 * one, -0.2 * one, 2.0 * one)
    assert np.max(np.abs(ns_residual(U, Mesh(xe, ye), p, Viscous(mu=0.05)))) < 1e-12


@pytest.mark.parametrize("p", [2, 3, 4])
def test_discrete_conservation_periodic(p):
    xe, ye = S.stretched_mesh(6, 5, seed=2)
    X, Y = S.point_coords(xe, ye, p)
    U = S.smooth_random_state(X, Y, seed=7, amp=0.1)
    m = Mesh(xe, ye)
    R = ns_residual(U, m, p, Viscous(mu=0.05))
    b = Basis(p)
    w2 = np.outer(b.w, b.w).reshape(-1)
    detJ = (0.25 * m.hx * m.hy).reshape(-1)
    tot = np.einsum("evp,p,e->v", R, w2, detJ)
    scale = np.einsum("evp,p,e->v", np.abs(R), w2, detJ)
    assert np.all(np.abs(tot) < 1e-13 * np.maximum(scale, 1.0))


def test_poiseuille_viscous_heating_closed_form():
    """Plane Poiseuille flow u = Uc 4y(H-y)/H^2, uniform rho and T, driven by
    the body force rho gx = 8 mu Uc / H^2 between isothermal walls: the exact
    semi-discrete residual is zero in mass and momentum and mu (du/dy)^2 in
    energy (viscous heating).  At p = 4 every field involved is a polynomial
    the scheme represents exactly."""
    p = 4
    xe = np.linspace(0.0, 2.0, 4)
    ye = S.channel_y_edges(6, first=0.05, ratio=1.3)
    m = Mesh(xe, ye, wall_y=True)
    X, Y = S.point_coords(xe, ye, p)
    Uc, H, mu, rho, T = 1.0, 1.0, 0.002, 1.0, 17.857
    u = Uc * 4 * Y * (H - Y) / H ** 2
    U = S.conserved(rho * np.ones_like(X), u, np.zeros_like(X), rho * T * np.ones_like(X))
    R = ns_residual(U, m, p, Viscous(mu=mu, gx=8 * mu * Uc / H ** 2 / rho, t_wall=T))
    dudy = Uc * 4 * (H - 2 * Y) / H ** 2
    heat = mu * dudy ** 2
    assert np.max(np.abs(R[:, 0])) < 1e-11
    assert np.max(np.abs(R[:, 1])) < 1e-11
    assert np.max(np.abs(R[:, 2])) < 1e-10
    assert np.max(np.abs(R[:, 3] - heat)) < 1e-9
    # the heating term is really there (not zero)
    assert np.max(heat) > 1e-2


def test_p0_is_two_point_finite_volume_navier_stokes():
    """With p = 0 the BR2 common gradient of a face is
    (q+ - q-)(1/h- + 1/h+)/2 along its normal (the two-point difference) and
    zero along it, so the scheme is textbook first-order FV: Rusanov
    inviscid flux minus the viscous flux of the face average."""
    xe, ye = S.stretched_mesh(5, 4, seed=8)
    X, Y = S.point_coords(xe, ye, 0)
    U = S.smooth_random_state(X, Y, seed=4, amp=0.2)
    m = Mesh(xe, ye)
    ph = Viscous(mu=0.03)
    R = ns_residual(U, m, 0, ph)
    Q = U[:, :, 0].reshape(m.ny, m.nx, 4)
    hx, hy = np.diff(xe), np.diff(ye)
    zero = np.zeros(4)
    expect = np.zeros_like(Q)
    for iy in range(m.ny):
        for ix in range(m.nx):
            def fx(a, b, ha, hb):
                qc = 0.5 * (a + b)
                gx = (b - a) * (1.0 / ha + 1.0 / hb) / 2.0
                fv, _ = viscous_fluxes(qc[:, None], gx[:, None], zero[:, None], ph)
                return rusanov(a, b, 0) - fv[:, 0]

            def gy(a, b, ha, hb):
                qc = 0.5 * (a + b)
                gyv = (b - a) * (1.0 / ha + 1.0 / hb) / 2.0
                _, gv = viscous_fluxes(qc[:, None], zero[:, None], gyv[:, None], ph)
                return rusanov(a, b, 1) - gv[:, 0]
            c = Q[iy, ix]
            ixm, ixp = (ix - 1) % m.nx, (ix + 1) % m.nx
            iym, iyp = (iy - 1) % m.ny, (iy + 1) % m.ny
            fe = fx(c, Q[iy, ixp], hx[ix], hx[ixp])
            fw = fx(Q[iy, ixm], c, hx[ixm], hx[ix])
            gn = gy(c, Q[iyp, ix], hy[iy], hy[iyp])
            gs = gy(Q[iym, ix], c, hy[iym], hy[iy])
            expect[iy, ix] = -(fe - fw) / hx[ix] - (gn - gs) / hy[iy]
    assert np.allclose(R[:, :, 0], expect.reshape(-1, 4), rtol=1e-12, atol=1e-12)


def test_ns_element_blocks_match_brute_force_jacobian():
    from oracle.jfnk import Problem, brute_jacobian
    from oracle.ns2d import ns_element_jacobians
    p = 2
    xe, ye = S.stretched_mesh(2, 2, seed=6)
    m = Mesh(xe, ye)
    ph = Viscous(mu=0.05)
    X, Y = S.point_coords(xe, ye, p)
    U = S.smooth_random_state(X, Y, seed=13, amp=0.1)

    class NS(Problem):
        def R(self, V):
            return ns_residual(V, m, p, ph)
    J = brute_jacobian(NS(m, p), U)
    Je = ns_element_jacobians(U, m, p, ph)
    nb = 4 * (p + 1) ** 2
    scale = np.max(np.abs(J))
    for e in range(m.ne):
        assert np.max(np.abs(Je[e] - J[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb])) < 1e-5 * scale
