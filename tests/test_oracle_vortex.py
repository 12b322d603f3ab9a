"""Pins of the oracle's isentropic vortex and error norm (Sec. 5.1,
Eq. VP_Solution and the error definition that follows it)."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle.basis import Basis
from oracle.fr2d import Mesh, residual
from oracle.vortex import (VortexCase, exact_primitive, exact_state, l2_error, point_coordinates,
                           vortex_errors)


def test_free_stream_mach_and_far_field():
    c = VortexCase()
    # c = sqrt(gamma p / rho) at the free stream; Ma on |V| = sqrt(2)
    assert math.sqrt(2.0) / math.sqrt(c.gamma * c.p_inf / c.rho_inf) == pytest.approx(0.5, rel=1e-15)
    assert c.p_inf == pytest.approx(40.0 / 7.0, rel=1e-15)
    rho, u, v, p = exact_primitive(c, np.array([9.5]), np.array([-9.5]))
    assert abs(rho[0] - 1.0) < 1e-15 and abs(u[0] - 1.0) < 1e-15 and abs(v[0] - 1.0) < 1e-15
    assert abs(p[0] - 40.0 / 7.0) < 1e-13


def test_isentropic_everywhere():
    c = VortexCase()
    x, y = np.meshgrid(np.linspace(-4, 4, 41), np.linspace(-4, 4, 37))
    rho, _, _, p = exact_primitive(c, x, y)
    s = p / rho ** c.gamma
    assert np.max(np.abs(s / (c.p_inf / c.rho_inf ** c.gamma) - 1.0)) < 1e-13


def test_radial_equilibrium_by_differences():
    """A steady vortex in the frame moving with the free stream balances the
    radial pressure gradient with the centripetal force: dp/dr = rho u_theta^2 / r.
    Checked along the ray y = 0 with central differences of the state itself,
    so a wrong amplitude, exponent or (gamma - 1) factor in dT fails."""
    c = VortexCase()
    r = np.linspace(0.2, 3.0, 15)
    h = 1e-4
    zero = np.zeros_like(r)
    _, _, _, pp = exact_primitive(c, r + h, zero)
    _, _, _, pm = exact_primitive(c, r - h, zero)
    rho, _, v, _ = exact_primitive(c, r, zero)
    dpdr = (pp - pm) / (2 * h)
    u_theta = v - c.v_inf                       # on y = 0 the swirl is along +y
    rhs = rho * u_theta ** 2 / r
    assert np.max(np.abs(dpdr - rhs) / np.abs(rhs)) < 1e-6


def test_peak_swirl_closed_form():
    """u_theta(r) = alpha/(2 pi) r exp(phi(1 - r^2)) peaks at r = 1/sqrt(2 phi) = 1
    with the value alpha / (2 pi)."""
    c = VortexCase()
    _, _, v, _ = exact_primitive(c, np.array([0.99, 1.0, 1.01]), np.zeros(3))
    sw = v - c.v_inf
    assert sw[1] == pytest.approx(c.alpha / (2 * math.pi), rel=1e-14)
    assert sw[0] < sw[1] and sw[2] < sw[1]


def test_one_period_returns_to_start():
    c = VortexCase()
    xe = np.linspace(-10, 10, 9)
    m = Mesh(xe, xe)
    a = exact_state(c, m, 3, 0.0)
    b = exact_state(c, m, 3, 20.0)
    assert np.max(np.abs(a - b)) < 1e-12
    # half a period: the centre sits at (10, 10) = the corner (image of the origin's opposite)
    h = exact_state(c, m, 3, 10.0)
    assert np.max(np.abs(h - a)) > 0.1


def test_input_generator_matches_oracle_vortex():
    """The seeded generator the GPU path and the oracle both read places the
    same vortex (pins the shared input against the oracle's restatement)."""
    xe, ye = S.uniform_mesh(12, box=(-10.0, 10.0, -10.0, 10.0))
    X, Y = S.point_coords(xe, ye, 3)
    for t in (0.0, 1.7):
        Ug = S.Vortex().state(X, Y, t=t, box=(-10.0, 10.0, -10.0, 10.0))
        Uo = exact_state(VortexCase(), Mesh(xe, ye), 3, t)
        assert np.max(np.abs(Ug - Uo)) < 1e-12
    xe, ye = S.uniform_mesh(8)
    X, Y = S.point_coords(xe, ye, 2)
    Ug = S.Vortex().state(X, Y, t=0.4)
    Uo = exact_state(VortexCase(box=(-5.0, 5.0, -5.0, 5.0)), Mesh(xe, ye), 2, 0.4)
    assert np.max(np.abs(Ug - Uo)) < 1e-12


@pytest.mark.parametrize("p", [2, 3])
def test_exact_vortex_is_a_discrete_steady_state_up_to_truncation(p):
    """R(U_exact(t)) + dU_exact/dt -> 0 under refinement on [-10,10]^2 (no
    periodic floor) at the FR truncation rate (order p for the pointwise
    residual of an interpolated smooth solution); an error in the vortex
    leaves an O(1) remainder instead (a doubled dT stalls at ~5e-2)."""
    c = VortexCase()
    t, d = 0.3, 1e-5
    errs = []
    for n in (10, 20, 40):
        xe = np.linspace(-10, 10, n + 1)
        m = Mesh(xe, xe)
        U = exact_state(c, m, p, t)
        dUdt = (exact_state(c, m, p, t + d) - exact_state(c, m, p, t - d)) / (2 * d)
        r = residual(U, m, p) - dUdt
        errs.append(max(l2_error(r[:, k], np.zeros_like(r[:, k]), m, p) for k in range(4)))
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1])
    order = math.log2(errs[-2] / errs[-1])
    assert order > p - 0.3, (errs, order)


def test_norm_equals_constant_error():
    xe = np.array([-1.0, -0.2, 0.5, 3.0])
    ye = np.array([0.0, 0.1, 1.0, 1.5, 4.0])
    m = Mesh(xe, ye)
    n = (3 + 1) ** 2
    s = np.full((m.ne, n), 2.0)
    assert l2_error(s, s + 0.37, m, 3) == pytest.approx(0.37, rel=1e-14)


def _poly_square_integral(coef, a, b, c, d):
    """Exact integral over [a,b] x [c,d] of (sum_kl coef[k,l] x^k y^l)^2."""
    sq = {}
    for (k1, l1), c1 in np.ndenumerate(coef):
        for (k2, l2), c2 in np.ndenumerate(coef):
            key = (k1 + k2, l1 + l2)
            sq[key] = sq.get(key, 0.0) + c1 * c2
    tot = 0.0
    for (k, l), cc in sq.items():
        tot += cc * (b ** (k + 1) - a ** (k + 1)) / (k + 1) * (d ** (l + 1) - c ** (l + 1)) / (l + 1)
    return tot


@pytest.mark.parametrize("p", [1, 2, 4])
def test_norm_exact_for_polynomial_error_on_jittered_mesh(p):
    """An error that is a polynomial of degree <= p in x and in y has a square
    of degree <= 2p, which the (p+1)-point Gauss-Legendre rule integrates
    exactly on every affine element; E then equals the closed-form value."""
    xe, ye = S.stretched_mesh(5, 4, seed=3, box=(-2.0, 3.0, -1.0, 2.0))
    m = Mesh(xe, ye)
    x, y = point_coordinates(m, Basis(p))
    rng = np.random.default_rng(7)
    coef = rng.uniform(-1, 1, size=(p + 1, p + 1))
    err = sum(coef[k, l] * x ** k * y ** l for k in range(p + 1) for l in range(p + 1))
    base = np.sin(x) * np.cos(y)
    got = l2_error(base + err, base, m, p)
    V = (xe[-1] - xe[0]) * (ye[-1] - ye[0])
    want = math.sqrt(_poly_square_integral(coef, xe[0], xe[-1], ye[0], ye[-1]) / V)
    assert got == pytest.approx(want, rel=1e-12)


def test_vortex_errors_zero_on_exact_and_linear_in_offset():
    c = VortexCase(box=(-5.0, 5.0, -5.0, 5.0))
    xe = np.linspace(-5, 5, 7)
    m = Mesh(xe, xe)
    U = exact_state(c, m, 2, 0.8)
    e0 = vortex_errors(U, c, m, 2, 0.8)
    assert max(e0.values()) < 1e-14
    V = U.copy()
    V[:, 0] += 1e-3                  # density up by 1e-3, momenta and energy kept
    e1 = vortex_errors(V, c, m, 2, 0.8)
    assert e1["rho"] == pytest.approx(1e-3, rel=1e-12)
