"""Pins of the 3D Navier-Stokes FR residual and the Taylor-Green dissipation
rate (oracle/fr3d.py)."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle.basis import Basis
from oracle.fr2d import Mesh
from oracle.fr3d import Gas3D, Mesh3D, Problem3D, as_grid, dissipation_rate, from_grid, residual3d
from oracle.jfnk import brute_jacobian, diagonal_blocks, fd_jv
from oracle.ns2d import Viscous, ns_residual


def _mean(R, mesh, p):
    """Quadrature of each variable of R over the domain, and of |R|."""
    b = Basis(p)
    w3 = np.einsum("k,j,i->kji", b.w, b.w, b.w).reshape(-1)
    vol = np.einsum("z,y,x->zyx", mesh.hz, mesh.hy, mesh.hx).reshape(-1) / 8.0
    return np.einsum("evp,p,e->v", R, w3, vol), np.einsum("evp,p,e->v", np.abs(R), w3, vol)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["uniform", "stretched"])
def test_free_stream_preserved(p, kind):
    edges = S.uniform_mesh3d(3) if kind == "uniform" else S.stretched_mesh3d(3, 2, 4, seed=p)
    X, _, _ = S.point_coords3d(*edges, p)
    one = np.ones_like(X)
    U = S.conserved3d(1.3 * one, 0.4 * one, -0.9 * one, 0.2 * one, 2.2 * one)
    R = residual3d(U, Mesh3D(*edges), p, Gas3D(mu=0.05))
    assert np.max(np.abs(R)) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_discrete_conservation(p):
    edges = S.stretched_mesh3d(3, 4, 2, seed=5)
    X, Y, Z = S.point_coords3d(*edges, p)
    U = S.smooth_random_state3d(X, Y, Z, seed=2, amp=0.1)
    m = Mesh3D(*edges)
    tot, scale = _mean(residual3d(U, m, p, Gas3D(mu=0.03)), m, p)
    assert np.all(np.abs(tot) < 1e-13 * np.maximum(scale, 1.0))


@pytest.mark.parametrize("mu", [0.0, 0.04])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_z_invariant_state_reduces_to_the_2d_residual(p, mu):
    """A state that does not depend on z and has w = 0: the mass, x/y
    momentum and energy residuals are the 2D Navier-Stokes residual.  R_rhow
    is zero without viscosity; with it, tau_zz = -2/3 mu div v enters the zeta
    correction (BR2 takes the broken gradient on the z faces, the points the
    corrected one), so R_rhow is odd in zeta and integrates to zero."""
    n = p + 1
    xe, ye = S.stretched_mesh(4, 3, seed=9, box=(-math.pi, math.pi, -math.pi, math.pi))
    ze = np.array([-1.0, 0.3, 2.0])
    X, Y = S.point_coords(xe, ye, p)
    U2 = S.smooth_random_state(X, Y, seed=4, amp=0.1, box=(-math.pi, math.pi, -math.pi, math.pi))
    R2 = ns_residual(U2, Mesh(xe, ye), p, Viscous(mu=mu, prandtl=0.71))
    nz, ne2 = len(ze) - 1, U2.shape[0]
    U3 = np.zeros((nz, ne2, 5, n, n * n))
    U3[:, :, [0, 1, 2, 4]] = U2[None, :, :, None, :]
    U3 = U3.reshape(nz * ne2, 5, n ** 3)
    R3 = residual3d(U3, Mesh3D(xe, ye, ze), p, Gas3D(mu=mu, prandtl=0.71)).reshape(nz, ne2, 5, n, n * n)
    scale = np.max(np.abs(R2))
    assert np.max(np.abs(R3[:, :, [0, 1, 2, 4]] - R2[None, :, :, None, :])) < 1e-12 * scale
    Rw = R3[:, :, 3].reshape(nz, ne2, n, n * n)                 # [.., k, j*n + i]
    if mu == 0.0:
        assert np.max(np.abs(Rw)) < 1e-12 * scale
    else:
        assert np.max(np.abs(Rw + Rw[:, :, ::-1])) < 1e-12 * scale
        assert np.max(np.abs(Rw)) > 1e-6 * scale


@pytest.mark.parametrize("p", [1, 2])
def test_cyclic_permutation_of_the_axes(p):
    """Relabelling (x, y, z) -> (z, x, y) (a rotation) maps the state and its
    residual the same way: (u, v, w) -> (w, u, v) and the grid axes with them."""
    edges = S.stretched_mesh3d(3, 2, 4, seed=3)
    X, Y, Z = S.point_coords3d(*edges, p)
    UA = S.smooth_random_state3d(X, Y, Z, seed=8, amp=0.1)
    gas = Gas3D(mu=0.05)
    mA = Mesh3D(*edges)
    RA = residual3d(UA, mA, p, gas)

    def rotate(U, mesh):
        Q = as_grid(U, mesh, p)                 # (var, iz, iy, ix, k, j, i)
        # new x' = old y, y' = old z, z' = old x
        Qb = Q.transpose(0, 3, 1, 2, 6, 4, 5)[[0, 2, 3, 1, 4]]
        return Qb
    mB = Mesh3D(edges[1], edges[2], edges[0])
    UB = from_grid(rotate(UA, mA), mB, p)
    RB = residual3d(UB, mB, p, gas)
    expect = from_grid(rotate(RA, mA), mB, p)
    assert np.max(np.abs(RB - expect)) < 1e-12 * np.max(np.abs(RA))


def _tiny(p=1, mu=0.05, seed=1):
    edges = S.stretched_mesh3d(2, 2, 2, seed=seed)
    X, Y, Z = S.point_coords3d(*edges, p)
    U = S.smooth_random_state3d(X, Y, Z, seed=seed, amp=0.1)
    return Problem3D(Mesh3D(*edges), p, Gas3D(mu=mu)), U


def test_fd_jv_matches_brute_force_jacobian():
    prob, U = _tiny()
    J = brute_jacobian(prob, U)
    z = S.random_vector(U.shape, seed=3)
    R0 = prob.R(U)
    y = fd_jv(prob, U, R0, z, shift=2.5)
    expect = 2.5 * z.reshape(-1) - J @ z.reshape(-1)
    assert np.linalg.norm(y.reshape(-1) - expect) / np.linalg.norm(expect) < 1e-6


def test_element_blocks_match_brute_force_diagonal_blocks():
    prob, U = _tiny(seed=4)
    J = brute_jacobian(prob, U)
    B = diagonal_blocks(prob, U)
    nb = prob.nb
    for e in range(prob.mesh.ne):
        Je = J[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb]
        assert np.linalg.norm(B[e] - Je) / np.linalg.norm(Je) < 2e-6


def test_degree3_element_block_matches_brute_force_columns():
    """The 320-row blocks of degree 3: element 0's block against central
    differences of the full residual in element 0's DOFs only (every other
    element unperturbed, so the rows of element 0 are dR_0/dq_0)."""
    prob, U = _tiny(p=3, seed=5)
    nb = prob.nb
    u = U.reshape(-1)
    J00 = np.zeros((nb, nb))
    for j in range(nb):
        h = 1e-6 * max(1.0, abs(u[j]))
        up = u.copy(); up[j] += h
        um = u.copy(); um[j] -= h
        d = (prob.R(up.reshape(U.shape)) - prob.R(um.reshape(U.shape))).reshape(-1)
        J00[:, j] = d[:nb] / (2 * h)
    B = diagonal_blocks(prob, U)
    assert np.linalg.norm(B[0] - J00) / np.linalg.norm(J00) < 2e-6


def _tgv_closed_forms():
    """<S:S> and <rho |v|^2 / 2> / rho0 of the Taylor-Green initial field
    (rho0 = V0 = L = 1, p0 from Ma = 0.1), integrated exactly."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    u = sp.sin(x) * sp.cos(y) * sp.cos(z)
    v = -sp.cos(x) * sp.sin(y) * sp.cos(z)
    w = sp.Integer(0)
    vel, X = (u, v, w), (x, y, z)
    SS = sum((sp.diff(vel[m], X[c]) + sp.diff(vel[c], X[m])) ** 2 / 4 for m in range(3) for c in range(3))
    p0 = sp.Rational(1) / (sp.Rational(14, 10) * sp.Rational(1, 100))
    pr = p0 + sp.Rational(1, 16) * (sp.cos(2 * x) + sp.cos(2 * y)) * (sp.cos(2 * z) + 2)
    ke = pr / p0 * (u ** 2 + v ** 2) / 2

    def mean(f):
        I = sp.integrate(sp.expand(sp.expand_trig(f)), (x, -sp.pi, sp.pi), (y, -sp.pi, sp.pi), (z, -sp.pi, sp.pi))
        return float(I / (2 * sp.pi) ** 3)
    return mean(SS), mean(ke)


def test_taylor_green_dissipation_rate_and_energy_closed_forms():
    """At t = 0 the Taylor-Green velocity is solenoidal: eps1 = 2 mu <S:S>,
    eps3 = 0, and the kinetic energy has a closed form; the quadrature of the
    interpolated field converges to them as the mesh is refined."""
    SS, ke = _tgv_closed_forms()
    tg = S.TaylorGreen()
    gas = Gas3D(mu=tg.mu, prandtl=tg.prandtl)
    errs = []
    for n in (4, 8):
        p = 3
        edges = S.uniform_mesh3d(n)
        X, Y, Z = S.point_coords3d(*edges, p)
        U = tg.state(X, Y, Z)
        e1, e3, k = dissipation_rate(U, Mesh3D(*edges), p, gas, tg.rho0)
        errs.append((abs(e1 / (2 * tg.mu * SS) - 1), abs(e3) / (2 * tg.mu * SS), abs(k / ke - 1)))
    # eps1 converges at order p + 1 (the velocity derivative of a degree-p
    # interpolant); eps3 vanishes by the field's symmetry; the energy is a
    # quadrature of exact point values
    assert errs[1][0] < 5e-4 and errs[1][0] < errs[0][0] / 12
    assert errs[0][1] < 1e-10 and errs[1][1] < 1e-10
    assert errs[0][2] < 1e-12 and errs[1][2] < 1e-12
    assert abs(SS - 0.375) < 1e-14   # <S:S> = 3/8 for this field


def test_ssprk3_step_on_the_3d_problem():
    """The oracle steppers accept the 3D problem: one SSPRK3 step of the
    Taylor-Green field conserves mass, momentum and energy to round-off."""
    from oracle.steppers import step_ssprk3
    tg = S.TaylorGreen()
    p = 2
    edges = S.uniform_mesh3d(3)
    X, Y, Z = S.point_coords3d(*edges, p)
    U = tg.state(X, Y, Z)
    prob = Problem3D(Mesh3D(*edges), p, Gas3D(mu=tg.mu, prandtl=tg.prandtl))
    U1 = step_ssprk3(prob, 0.01, U)
    t0, s0 = _mean(U, prob.mesh, p)
    t1, _ = _mean(U1, prob.mesh, p)
    assert np.all(np.abs(t1 - t0) < 1e-12 * np.maximum(s0, 1.0))
    assert np.max(np.abs(U1 - U)) > 1e-6


def _rk4_density_wave_3d(n, p, t_end=0.3, cfl=0.2):
    """L2 density error of a density wave rho = 1 + 0.2 sin(x + y + z)
    translated by v = (1, 1, 1) at constant pressure (an exact solution of
    the Euler equations) after classical RK4 steps small enough that the
    spatial error dominates."""
    edges = S.uniform_mesh3d(n)
    X, Y, Z = S.point_coords3d(*edges, p)

    def exact(t):
        one = np.ones_like(X)
        return S.conserved3d(1.0 + 0.2 * np.sin((X - t) + (Y - t) + (Z - t)), one, one, one, one)
    U = exact(0.0)
    m, b = Mesh3D(*edges), Basis(p)
    h = 2 * math.pi / n
    dt0 = cfl * h / ((p + 1) ** 2 * 3.0)
    nsteps = int(math.ceil(t_end / dt0))
    dt = t_end / nsteps
    f = lambda u: residual3d(u, m, p, Gas3D(), b)
    for _ in range(nsteps):
        k1 = f(U)
        k2 = f(U + 0.5 * dt * k1)
        k3 = f(U + 0.5 * dt * k2)
        k4 = f(U + dt * k3)
        U = U + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    w3 = np.einsum("k,j,i->kji", b.w, b.w, b.w).reshape(-1)
    err2 = np.einsum("ep,p->", (U[:, 0] - exact(t_end)[:, 0]) ** 2, w3) * h ** 3 / 8
    return math.sqrt(err2 / (2 * math.pi) ** 3)


def test_spatial_order_on_a_3d_density_wave():
    """Order p + 1 = 2 at p = 1 under h-refinement along a wave that crosses
    all three directions, and a smaller error at p = 2 on the same mesh."""
    e4, e8 = _rk4_density_wave_3d(4, 1), _rk4_density_wave_3d(8, 1)
    assert math.log2(e4 / e8) > 2 - 0.3
    assert _rk4_density_wave_3d(4, 2) < e4 / 4


def test_viscous_shear_flow_closed_form():
    """w = A sin x with rho = 1, u = v = 0 and constant pressure: a closed
    form of the viscous terms along z (the direction the 2D reduction does
    not reach).  The continuous residual is R_rhow = -mu A sin x, R_E =
    mu A^2 cos 2x and zero otherwise.  R_rho and R_rhov vanish to round-off;
    R_rhow converges to the closed form at about order p in the maximum norm
    (the residual is a second derivative of the interpolated state); R_rhou
    is the BR2 broken-gradient term on the z faces and vanishes at the same
    order; R_E, whose heat flux differentiates the chain-rule temperature
    gradient once more, converges at about order p - 1."""
    A, mu, p = 0.3, 0.05, 3
    errs = []
    for n in (8, 16):
        ex, e2 = S.uniform_edges(n, -math.pi, math.pi), S.uniform_edges(2, -math.pi, math.pi)
        X, Y, Z = S.point_coords3d(ex, e2, e2, p)
        one = np.ones_like(X)
        U = S.conserved3d(one, 0 * one, 0 * one, A * np.sin(X), 2.0 * one)
        R = residual3d(U, Mesh3D(ex, e2, e2), p, Gas3D(mu=mu))
        assert np.max(np.abs(R[:, [0, 2]])) < 1e-13
        errs.append((np.max(np.abs(R[:, 3] + mu * A * np.sin(X))),
                     np.max(np.abs(R[:, 1])),
                     np.max(np.abs(R[:, 4] - mu * A * A * np.cos(2 * X)))))
    order = [math.log2(errs[0][c] / errs[1][c]) for c in range(3)]
    assert order[0] > p - 0.5 and order[1] > p - 0.5 and order[2] > p - 1.5
    assert errs[1][0] < 0.01 * mu * A
