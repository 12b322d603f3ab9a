"""Pins of the 1D FR tables (oracle/basis.py) against facts the mathematics fixes."""
import numpy as np
import pytest

from oracle.basis import Basis, derivative_matrix, gauss_legendre, lagrange_values, radau_gl, radau_gr


@pytest.mark.parametrize("p", range(0, 8))
def test_gauss_legendre_matches_library(p):
    x, w = gauss_legendre(p + 1)
    xr, wr = np.polynomial.legendre.leggauss(p + 1)
    assert np.allclose(x, xr, atol=1e-15, rtol=0)
    assert np.allclose(w, wr, atol=1e-14, rtol=0)


@pytest.mark.parametrize("p", range(0, 7))
def test_quadrature_exact_to_degree_2p_plus_1(p):
    x, w = gauss_legendre(p + 1)
    for k in range(2 * p + 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("p", range(1, 7))
def test_derivative_matrix_exact_on_polynomials(p):
    b = Basis(p)
    for k in range(p + 1):
        d = b.D @ b.xi ** k
        exact = k * b.xi ** (k - 1) if k > 0 else np.zeros_like(b.xi)
        assert np.max(np.abs(d - exact)) < 1e-12


@pytest.mark.parametrize("p", range(1, 7))
def test_lagrange_end_values_extrapolate_polynomials(p):
    b = Basis(p)
    poly = np.polynomial.Polynomial(np.random.default_rng(p).standard_normal(p + 1))
    f = poly(b.xi)
    assert abs(b.lm @ f - poly(-1.0)) < 1e-12
    assert abs(b.lp @ f - poly(1.0)) < 1e-12
    L = lagrange_values(b.xi, b.xi)
    assert np.allclose(L, np.eye(p + 1), atol=1e-14)


@pytest.mark.parametrize("p", range(0, 7))
def test_radau_correction_end_values_and_slope(p):
    gl, dgl = radau_gl(p, np.array([-1.0, 1.0]))
    gr, dgr = radau_gr(p, np.array([-1.0, 1.0]))
    assert np.allclose(gl, [1.0, 0.0], atol=1e-14)
    assert np.allclose(gr, [0.0, 1.0], atol=1e-14)
    # closed form of the Radau (g_DG) end slope: g_L'(-1) = -(p+1)^2/2
    assert abs(dgl[0] + (p + 1) ** 2 / 2.0) < 1e-12
    assert abs(dgr[1] - (p + 1) ** 2 / 2.0) < 1e-12


@pytest.mark.parametrize("p", range(1, 7))
def test_radau_g_dg_orthogonal_to_degree_p_minus_1(p):
    """g_L is the right Radau polynomial: orthogonal to P_{p-1} and below."""
    xq, wq = np.polynomial.legendre.leggauss(p + 4)
    g, _ = radau_gl(p, xq)
    for k in range(p):
        assert abs(np.dot(wq, g * xq ** k)) < 1e-13


@pytest.mark.parametrize("p", range(1, 7))
def test_fr_dg_identity(p):
    """With g_DG on Gauss points the FR correction equals the DG lifting:
    sum_i w_i l_m(x_i) g_L'(x_i) = -l_m(-1) for every basis function."""
    b = Basis(p)
    lhs = b.w * b.dgL          # w_i g_L'(x_i) against l_m(x_i) = delta_mi
    assert np.allclose(lhs, -b.lm, atol=1e-13)
    assert np.allclose(b.w * b.dgR, b.lp, atol=1e-13)
