"""Pins of the oracle FR residual (oracle/fr2d.py)."""
import math
import os

import numpy as np
import pytest

import synthetic as S
from oracle.basis import Basis
from oracle.fr2d import Mesh, flux_x, flux_y, residual, rusanov

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mesh(kind, nx, ny, seed=0):
    if kind == "uniform":
        return S.uniform_mesh(nx, ny=ny)
    return S.stretched_mesh(nx, ny, seed=seed)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("kind", ["uniform", "stretched"])
def test_free_stream_preserved(p, kind):
    xe, ye = _mesh(kind, 5, 4, seed=p)
    X, _ = S.point_coords(xe, ye, p)
    one = np.ones_like(X)
    U = S.conserved(1.3 * one, 0.4 * one, -0.9 * one, 2.2 * one)
    R = residual(U, Mesh(xe, ye), p)
    assert np.max(np.abs(R)) < 1e-13 * 10


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_discrete_conservation(p):
    xe, ye = S.stretched_mesh(6, 5, seed=3)
    X, Y = S.point_coords(xe, ye, p)
    U = S.smooth_random_state(X, Y, seed=11, amp=0.1)
    m = Mesh(xe, ye)
    R = residual(U, m, p)
    b = Basis(p)
    w2 = np.outer(b.w, b.w).reshape(-1)
    detJ = (0.25 * m.hx * m.hy).reshape(-1)
    total = np.einsum("evp,p,e->v", R, w2, detJ)
    scale = np.einsum("evp,p,e->v", np.abs(R), w2, detJ)
    assert np.all(np.abs(total) < 1e-13 * np.maximum(scale, 1.0))


def test_rusanov_golden_sod():
    vals = np.loadtxt(os.path.join(GOLDEN, "rusanov_sod.txt"))
    qL = np.array([1.0, 0.0, 0.0, 2.5])
    qR = np.array([0.125, 0.0, 0.0, 0.25])
    assert np.allclose(rusanov(qL, qR, 0), vals, rtol=0, atol=1e-15)
    # rotate the states: same physics along y
    qLy = np.array([1.0, 0.0, 0.0, 2.5])
    qRy = np.array([0.125, 0.0, 0.0, 0.25])
    fy = rusanov(qLy, qRy, 1)
    assert np.allclose(fy[[0, 2, 1, 3]], vals, rtol=0, atol=1e-15)


def test_rusanov_consistent():
    q = np.array([1.1, 0.3, -0.2, 3.0])
    assert np.allclose(rusanov(q, q, 0), flux_x(q), atol=1e-15)
    assert np.allclose(rusanov(q, q, 1), flux_y(q), atol=1e-15)


def test_p0_is_first_order_rusanov_finite_volume():
    """With p = 0 the FR scheme is the textbook first-order FV scheme
    dU/dt = -(F_{i+1/2} - F_{i-1/2})/hx - (G_{j+1/2} - G_{j-1/2})/hy."""
    xe, ye = S.stretched_mesh(5, 4, seed=5)
    X, Y = S.point_coords(xe, ye, 0)
    U = S.smooth_random_state(X, Y, seed=2, amp=0.2)
    m = Mesh(xe, ye)
    R = residual(U, m, 0)
    Q = U[:, :, 0].reshape(m.ny, m.nx, 4)
    hx, hy = np.diff(xe), np.diff(ye)
    expect = np.zeros_like(Q)
    for iy in range(m.ny):
        for ix in range(m.nx):
            qc = Q[iy, ix]
            fe = rusanov(qc, Q[iy, (ix + 1) % m.nx], 0)
            fw = rusanov(Q[iy, ix - 1], qc, 0)
            gn = rusanov(qc, Q[(iy + 1) % m.ny, ix], 1)
            gs = rusanov(Q[iy - 1, ix], qc, 1)
            expect[iy, ix] = -(fe - fw) / hx[ix] - (gn - gs) / hy[iy]
    assert np.allclose(R[:, :, 0], expect.reshape(-1, 4), rtol=1e-13, atol=1e-13)


def _rk4_density_wave(n, p, t_end, cfl=0.1):
    xe, ye = S.uniform_mesh(n)
    X, Y = S.point_coords(xe, ye, p)
    U = S.density_wave_state(X, Y, 0.0)
    m = Mesh(xe, ye)
    b = Basis(p)
    h = 10.0 / n
    dt0 = cfl * h / ((p + 1) ** 2 * 3.0)
    nsteps = int(math.ceil(t_end / dt0))
    dt = t_end / nsteps
    f = lambda u: residual(u, m, p, b)
    for _ in range(nsteps):             # classical fourth-order Runge-Kutta
        k1 = f(U)
        k2 = f(U + 0.5 * dt * k1)
        k3 = f(U + 0.5 * dt * k2)
        k4 = f(U + dt * k3)
        U = U + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    exact = S.density_wave_state(X, Y, t_end)
    w2 = np.outer(b.w, b.w).reshape(-1)
    err = np.sqrt(np.einsum("ep,p->", (U[:, 0] - exact[:, 0]) ** 2, w2) * (h * h / 4) / 100.0)
    return err


@pytest.mark.parametrize("p", [1, 2])
def test_spatial_order_p_plus_1_density_wave(p):
    e1 = _rk4_density_wave(4, p, 1.0)
    e2 = _rk4_density_wave(8, p, 1.0)
    e3 = _rk4_density_wave(16, p, 1.0)
    o2 = math.log2(e2 / e3)
    assert e1 > e2 > e3
    assert o2 > p + 1 - 0.3, (e1, e2, e3)
