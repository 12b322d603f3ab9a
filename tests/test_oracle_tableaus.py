"""Pins of the ROW / ESDIRK / BDF2 coefficient sets (oracle/tableaus.py).

Order conditions are written from the rooted-tree expansions (Butcher trees
for Runge-Kutta; Hairer & Wanner's Rosenbrock conditions with
beta_ij = alpha_ij + gamma_ij).  The empirical-order tests on an ODE check the
same facts by a route that shares nothing with those formulas."""
import json
import math
import os

import numpy as np
import pytest

from oracle.tableaus import BDF2_A, BDF2_OMEGA, ESDIRK, ROW

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rk_residuals(A, b):
    c = A.sum(1)
    return [b.sum() - 1,
            b @ c - 1 / 2,
            b @ c ** 2 - 1 / 3, b @ (A @ c) - 1 / 6,
            b @ c ** 3 - 1 / 4, (b * c) @ (A @ c) - 1 / 8, b @ (A @ c ** 2) - 1 / 12,
            b @ (A @ (A @ c)) - 1 / 24]


def ros_residuals(alpha, G, b):
    g = G[0, 0]
    beta = alpha + np.tril(G, -1)
    al = alpha.sum(1)
    bp = beta.sum(1)
    return [b.sum() - 1,
            b @ bp - (0.5 - g),
            b @ al ** 2 - 1 / 3, b @ (beta @ bp) - (1 / 6 - g + g * g),
            b @ al ** 3 - 1 / 4, (b * al) @ (alpha @ bp) - (1 / 8 - g / 3),
            b @ (beta @ al ** 2) - (1 / 12 - g / 3),
            b @ (beta @ (beta @ bp)) - (1 / 24 - g / 2 + 1.5 * g * g - g ** 3)]


NCOND = {1: 1, 2: 2, 3: 4, 4: 8}


@pytest.mark.parametrize("order", [2, 3, 4])
def test_esdirk_order_conditions_and_structure(order):
    t = ESDIRK[order]()
    res = rk_residuals(t.A, t.b)
    assert np.max(np.abs(res[:NCOND[order]])) < 1e-13
    if order < 4:
        assert np.max(np.abs(res[NCOND[order]:NCOND[order + 1]])) > 1e-6
    assert t.A[0, 0] == 0.0
    assert np.allclose(np.diag(t.A)[1:], t.omega)
    assert np.allclose(t.b, t.A[-1])            # stiffly accurate
    assert np.allclose(np.triu(t.A, 1), 0.0)
    stages = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))["esdirk_stages"]
    assert t.stages == stages[t.name]


@pytest.mark.parametrize("order", [2, 3, 4])
def test_row_order_conditions_and_structure(order):
    t = ROW[order]()
    alpha, G, b = t.alpha_form()
    res = ros_residuals(alpha, G, b)
    assert np.max(np.abs(res[:NCOND[order]])) < 1e-13
    assert np.allclose(np.diag(G), t.gamma)
    # stiffly accurate: last stage at t + dt and b equal to its beta row
    assert abs(alpha[-1].sum() - 1.0) < 1e-13
    beta_last = alpha[-1] + G[-1]
    assert np.allclose(b, beta_last, atol=1e-12)
    stages = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))["row_stages"]
    assert t.stages == stages[t.name]


def _stability(B, b, z):
    s = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * B, np.ones(s))


@pytest.mark.parametrize("kind,order", [(k, o) for k in ("row", "esdirk") for o in (2, 3, 4)])
def test_l_stability(kind, order):
    if kind == "row":
        alpha, G, b = ROW[order]().alpha_form()
        B = alpha + G
    else:
        t = ESDIRK[order]()
        B, b = t.A, t.b
    assert abs(_stability(B, b, -1e9)) < 1e-6
    for y in np.linspace(0.0, 200.0, 401):
        assert abs(_stability(B, b, 1j * y)) <= 1.0 + 1e-12
    for z in (-0.5, -3.0, -50.0, -2 + 5j):
        assert abs(_stability(B, b, z)) <= 1.0 + 1e-12


def test_bdf2_coefficients_from_paper():
    gold = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))["bdf2"]
    assert BDF2_OMEGA == pytest.approx(gold["omega"], abs=1e-16)
    assert BDF2_A[0] == pytest.approx(gold["a1"], abs=1e-16)
    assert BDF2_A[1] == pytest.approx(gold["a2"], abs=1e-16)
    # exact for quadratics: q(t) = 1 + 2t + 3t^2 on t = 0, h, 2h
    h = 0.1
    q = lambda t: 1 + 2 * t + 3 * t * t
    dq = lambda t: 2 + 6 * t
    lhs = q(2 * h)
    rhs = h * BDF2_OMEGA * dq(2 * h) + BDF2_A[0] * q(h) + BDF2_A[1] * q(0.0)
    assert abs(lhs - rhs) < 1e-14


# ---------------------------------------------------------- ODE orders --
def _vdp(y, mu=2.0):
    return np.array([y[1], mu * (1 - y[0] ** 2) * y[1] - y[0]])


def _vdp_jac(y, mu=2.0):
    return np.array([[0.0, 1.0], [-2 * mu * y[0] * y[1] - 1.0, mu * (1 - y[0] ** 2)]])


def _row_ode(t, y, h, n):
    for _ in range(n):
        J = _vdp_jac(y)
        W = np.eye(2) / (t.gamma * h) - J
        Y = []
        for i in range(t.stages):
            yi = y + sum(t.a[i, j] * Y[j] for j in range(i))
            rhs = _vdp(yi) + sum(t.c[i, j] * Y[j] for j in range(i)) / h
            Y.append(np.linalg.solve(W, rhs))
        y = y + sum(t.m[j] * Y[j] for j in range(t.stages))
    return y


def _esdirk_ode(t, y, h, n):
    for _ in range(n):
        K = [_vdp(y)]
        yi = y
        for i in range(1, t.stages):
            base = y + h * sum(t.A[i, j] * K[j] for j in range(i))
            for _ in range(50):                     # Newton on the stage
                F = yi - base - h * t.omega * _vdp(yi)
                Jf = np.eye(2) - h * t.omega * _vdp_jac(yi)
                d = np.linalg.solve(Jf, -F)
                yi = yi + d
                if np.max(np.abs(d)) < 1e-15:
                    break
            K.append(_vdp(yi))
        y = y + h * sum(t.b[i] * K[i] for i in range(t.stages))
    return y


@pytest.mark.parametrize("kind,order", [(k, o) for k in ("row", "esdirk") for o in (2, 3, 4)])
def test_observed_order_on_nonlinear_ode(kind, order):
    y0 = np.array([2.0, 0.0])
    T = 1.0
    t = ROW[order]() if kind == "row" else ESDIRK[order]()
    run = _row_ode if kind == "row" else _esdirk_ode
    ref = run(t, y0, T / 2048, 2048)
    errs = [np.linalg.norm(run(t, y0, T / n, n) - ref) for n in (16, 32, 64)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(rates[-1] - order) < 0.3, (errs, rates)
