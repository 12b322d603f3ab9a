"""Pins of the oracle's Roe flux (oracle/fr2d.py, Sec. 3 Eq. invis_com): the
defining property of Roe's linearisation checked against an independent
eigen-decomposition, consistency, exact resolution of a stationary contact,
full upwinding for supersonic flow, and the FR residual with Roe fluxes
(free stream, conservation, spatial order)."""
import numpy as np
import pytest

import synthetic as S
from oracle.fr2d import Mesh, flux_x, flux_y, pressure, residual, roe, rusanov

G = 1.4


def _q(rho, u, v, p):
    return np.array([rho, rho * u, rho * v, p / (G - 1.0) + 0.5 * rho * (u * u + v * v)])


def _jacobian(u, v, H, direction):
    """Analytic flux Jacobian of the 2D Euler flux along x or y at (u, v, H),
    written out from f(q) (test-side, independent of the oracle's waves)."""
    g1 = G - 1.0
    k = 0.5 * (u * u + v * v)
    if direction == 0:
        return np.array([
            [0.0, 1.0, 0.0, 0.0],
            [g1 * k - u * u, (3.0 - G) * u, -g1 * v, g1],
            [-u * v, v, u, 0.0],
            [u * (g1 * k - H), H - g1 * u * u, -g1 * u * v, G * u]])
    return np.array([
        [0.0, 0.0, 1.0, 0.0],
        [-u * v, v, u, 0.0],
        [g1 * k - v * v, -g1 * u, (3.0 - G) * v, g1],
        [v * (g1 * k - H), -g1 * u * v, H - g1 * v * v, G * v]])


def _roe_average(qa, qb):
    ra, rb = qa[0], qb[0]
    ua, va, ub, vb = qa[1] / ra, qa[2] / ra, qb[1] / rb, qb[2] / rb
    Ha = (qa[3] + pressure(qa, G)) / ra
    Hb = (qb[3] + pressure(qb, G)) / rb
    sa, sb = np.sqrt(ra), np.sqrt(rb)
    w = lambda a, b: (sa * a + sb * b) / (sa + sb)
    return w(ua, ub), w(va, vb), w(Ha, Hb)


@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_roe_equals_abs_jacobian_decomposition(direction, seed):
    """F = (f(qm) + f(qp))/2 - |A| (qp - qm)/2 with A the flux Jacobian at the
    Roe average and |A| = V |Lambda| V^-1 from a numerical eigen-solver; and
    Roe's property f(qp) - f(qm) = A (qp - qm)."""
    rng = np.random.default_rng(seed)
    qm = _q(rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.5, 3))
    qp = _q(rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.5, 3))
    flux = flux_x if direction == 0 else flux_y
    u, v, H = _roe_average(qm, qp)
    A = _jacobian(u, v, H, direction)
    assert np.allclose(flux(qp, G) - flux(qm, G), A @ (qp - qm), rtol=1e-12, atol=1e-12)
    lam, V = np.linalg.eig(A)
    absA = (V @ np.diag(np.abs(lam)) @ np.linalg.inv(V)).real
    want = 0.5 * (flux(qm, G) + flux(qp, G)) - 0.5 * absA @ (qp - qm)
    assert np.allclose(roe(qm, qp, direction, G), want, rtol=1e-11, atol=1e-11)


def test_roe_consistency_contact_and_upwinding():
    q = _q(1.3, 0.4, -0.2, 2.0)
    for d, flux in ((0, flux_x), (1, flux_y)):
        assert np.allclose(roe(q, q, d, G), flux(q, G), rtol=1e-14, atol=1e-14)
    # stationary contact: equal pressure, no velocity, different densities
    qa, qb = _q(1.0, 0.0, 0.0, 1.0), _q(0.125, 0.0, 0.0, 1.0)
    assert np.allclose(roe(qa, qb, 0, G), [0.0, 1.0, 0.0, 0.0], atol=1e-14)
    assert np.linalg.norm(rusanov(qa, qb, 0, G) - [0.0, 1.0, 0.0, 0.0]) > 0.1  # Rusanov smears it
    # supersonic to the right: every Roe wave speed positive -> the left flux
    qa, qb = _q(1.0, 3.0, 0.2, 1.0), _q(0.9, 2.8, 0.1, 0.8)
    assert np.allclose(roe(qa, qb, 0, G), flux_x(qa, G), rtol=1e-12, atol=1e-12)


def test_fr_residual_with_roe_free_stream_and_conservation():
    p = 3
    xe, ye = S.stretched_mesh(6, 5, seed=1)
    X, Y = S.point_coords(xe, ye, p)
    m = Mesh(xe, ye)
    U = _q(1.0, 0.7, -0.4, 2.0)[None, :, None] * np.ones((m.ne, 4, (p + 1) ** 2))
    assert np.max(np.abs(residual(U, m, p, riemann="roe"))) < 1e-12
    U = S.smooth_random_state(X, Y, seed=5, amp=0.1)
    R = residual(U, m, p, riemann="roe")
    w = np.polynomial.legendre.leggauss(p + 1)[1]
    w2 = np.outer(w, w).reshape(-1)
    detJ = (m.hx * m.hy).reshape(-1) / 4.0
    tot = np.einsum("evp,p,e->v", R, w2, detJ)
    assert np.all(np.abs(tot) < 1e-12)


def _rk4_wave_error(n, p, t_end, cfl=0.1):
    from oracle.basis import Basis
    xe, ye = S.uniform_mesh(n)
    X, Y = S.point_coords(xe, ye, p)
    U = S.density_wave_state(X, Y, 0.0)
    m, b = Mesh(xe, ye), Basis(p)
    h = 10.0 / n
    nsteps = int(np.ceil(t_end / (cfl * h / ((p + 1) ** 2 * 3.0))))
    dt = t_end / nsteps
    f = lambda u: residual(u, m, p, b, riemann="roe")
    for _ in range(nsteps):  # classical fourth-order Runge-Kutta
        k1 = f(U)
        k2 = f(U + 0.5 * dt * k1)
        k3 = f(U + 0.5 * dt * k2)
        k4 = f(U + dt * k3)
        U = U + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    exact = S.density_wave_state(X, Y, t_end)
    w2 = np.outer(b.w, b.w).reshape(-1)
    return np.sqrt(np.einsum("ep,p->", (U[:, 0] - exact[:, 0]) ** 2, w2) * (h * h / 4) / 100.0)


def test_fr_with_roe_spatial_order_p_plus_1():
    """Translating density wave with Roe fluxes: solution error of order
    p + 1 (the FR/DG order) after RK4 time integration."""
    p = 2
    e = [_rk4_wave_error(n, p, 1.0) for n in (4, 8, 16)]
    assert e[0] > e[1] > e[2]
    assert np.log2(e[1] / e[2]) > p + 1 - 0.3, e
